"""Pins of the oracle's spline bases against library routines and identities."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import basis_all_degrees, h1_and_edge, element_quadrature, gauss_legendre


def _knots(n_el, p, graded=False):
    inner = np.arange(1, n_el) / n_el
    if graded:
        inner = inner ** 1.3
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("graded", [False, True])
def test_basis_matches_scipy_design_matrix(p, graded):
    t = _knots(5, p, graded)
    x = np.linspace(0.013, 0.987, 41)
    N = basis_all_degrees(t, p, x)[p]
    ref = BSpline.design_matrix(x, t, p).toarray().T
    assert np.abs(N - ref).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3])
def test_partition_of_unity_and_edge_identity(p):
    t = _knots(6, p, graded=True)
    x = np.linspace(0.01, 0.99, 57)
    N, dN, D = h1_and_edge(t, p, x)
    assert np.abs(N.sum(0) - 1).max() < 1e-14
    # derivative identity dN_i = D_{i-1} - D_i (zero-padded), independent check by
    # central differences of the basis itself
    h = 1e-6
    Np, _, _ = h1_and_edge(t, p, x + h)
    Nm, _, _ = h1_and_edge(t, p, x - h)
    fd = (Np - Nm) / (2 * h)
    assert np.abs(fd - dN).max() < 1e-6 * max(1.0, np.abs(dN).max())
    Dpad = np.vstack([np.zeros((1, len(x))), D, np.zeros((1, len(x)))])
    assert np.abs(dN - (Dpad[:-1] - Dpad[1:])).max() < 1e-12
    # the edge functions integrate to one: int D_i = 1 for the Curry-Schoenberg scaling
    xq, wq = element_quadrature(t, p, p + 2)
    _, _, Dq = h1_and_edge(t, p, xq.ravel())
    assert np.abs(Dq @ wq.ravel() - 1).max() < 1e-13


def test_gauss_rule_exactness():
    for q in range(1, 7):
        x, w = gauss_legendre(q)
        for k in range(2 * q):
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert abs(np.sum(w * x ** k) - exact) < 1e-13
