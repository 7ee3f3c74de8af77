"""B-spline bases on open knot vectors, evaluated with the Cox-de Boor recursion.

The discrete spaces follow Sec. 2.2 (spline edge elements of the IGA framework):
per direction, the H^1 factor uses the degree-p B-splines N_i on the knot vector
t; the edge factor in the component's own direction uses

    D_i = p / (t_{i+p+1} - t_{i+1}) * N_{i+1, p-1},   i = 0 .. n-2,

so that dN_i/dx = D_{i-1} - D_i (the derivative identity that makes the discrete
gradient the +-1 incidence matrix of the control mesh, used by the tree gauge of
Sec. 3).  Plain definitions, written for clarity not speed.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(q: int):
    """q-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return x, w


def basis_all_degrees(t: np.ndarray, p: int, x: np.ndarray):
    """All B-splines of degree 0..p on knot vector t at points x.

    Returns a list ``B[k]`` of arrays of shape (len(t)-k-1, len(x)).  Points must not
    coincide with knots (quadrature points never do).
    """
    t = np.asarray(t, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    m = len(t)
    B0 = ((t[:-1, None] <= x[None, :]) & (x[None, :] < t[1:, None])).astype(np.float64)
    out = [B0]
    for k in range(1, p + 1):
        prev = out[-1]
        nk = m - k - 1
        Bk = np.zeros((nk, len(x)))
        for i in range(nk):
            d1 = t[i + k] - t[i]
            d2 = t[i + k + 1] - t[i + 1]
            if d1 > 0:
                Bk[i] += (x - t[i]) / d1 * prev[i]
            if d2 > 0:
                Bk[i] += (t[i + k + 1] - x) / d2 * prev[i + 1]
        out.append(Bk)
    return out


def h1_and_edge(t: np.ndarray, p: int, x: np.ndarray):
    """Values at x of N_i (degree p), dN_i/dx, and the edge functions D_i.

    Shapes: N (n, X), dN (n, X), D (n-1, X) with n = len(t) - p - 1.
    """
    B = basis_all_degrees(t, p, x)
    N = B[p]
    n = N.shape[0]
    Bm = B[p - 1]
    D = np.zeros((n - 1, len(x)))
    for i in range(n - 1):
        D[i] = p / (t[i + p + 1] - t[i + 1]) * Bm[i + 1]
    # derivative of N_i: p/(t_{i+p}-t_i) N_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}
    dN = np.zeros_like(N)
    for i in range(n):
        d1 = t[i + p] - t[i]
        d2 = t[i + p + 1] - t[i + 1]
        if d1 > 0:
            dN[i] += p / d1 * Bm[i]
        if d2 > 0:
            dN[i] -= p / d2 * Bm[i + 1]
    return N, dN, D


def element_quadrature(t: np.ndarray, p: int, q: int):
    """Gauss points/weights of every non-empty knot span (element) of t.

    Returns (x, w, el) with x, w of shape (E, q) and the knot-span start index per
    element; element e covers [t[p+e], t[p+e+1]].
    """
    g, gw = gauss_legendre(q)
    n_el = len(t) - 2 * p - 1
    lo = t[p:p + n_el]
    hi = t[p + 1:p + n_el + 1]
    x = lo[:, None] + (hi - lo)[:, None] * (g[None, :] + 1.0) * 0.5
    w = (hi - lo)[:, None] * gw[None, :] * 0.5
    return x, w
