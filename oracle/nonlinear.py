"""Nonlinear reluctivity nu(|B|) resolved by Newton's method in every implicit-Euler
step (test infrastructure: only tests, the smoke check and the bench's CPU
baseline use this package).

The paper keeps the material linear and notes that nonlinear behaviour is a plain
extension of its method (Sec. 2, after Eq. (3)).  The extension built here: in the
conducting elements (sigma > 0) the reluctivity follows the exponential law

    nu(s) = nu0 (k1 exp(k2 s) + k3),   s = |B|^2 = |curl A|^2,

elsewhere it stays the given per-element constant.  The step of Eq. (11) becomes the
nonlinear system (on the free, gauged unknowns)

    R(a) = M (a - a^l) + dt (K_lin a + N(a)) - dt j = 0,
    N(a)_i = int_{Omega_C} nu(|B|^2) B . curl w_i,          B = curl(sum_k a_k w_k),

whose Jacobian is  J(a) = M + dt (K_lin + K_t(a))  with
    K_t(a)_ik = int_{Omega_C} nu(s) curl w_k . curl w_i + 2 nu'(s) (B . curl w_k)(B . curl w_i).
R is the gradient of the energy
    E(a) = 1/2 a.M a - a.M a^l + dt (1/2 a.K_lin a + int_{Omega_C} 1/2 Phi(|B|^2) - j.a),
    Phi(s) = int_0^s nu = nu0 (k1 (exp(k2 s) - 1) / k2 + k3 s),
so both R and J can be checked against finite differences of E.  Newton: a_0 = a^l,
J(a_k) d_k = -R(a_k), a_{k+1} = a_k + d_k, stop when ||d_k|| <= tol ||a_{k+1}||.
Linear solves: SuperLU (library routine) on the assembled global matrices.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assembly import Assembled, PatchEval
from .gauge import CLS_E, Gauge


class Reluctivity:
    """nu(s) = nu0 (k1 exp(k2 s) + k3) as a function of s = |B|^2."""

    def __init__(self, nu0=1.0, k1=0.5, k2=2.0, k3=0.5):
        self.nu0, self.k1, self.k2, self.k3 = float(nu0), float(k1), float(k2), float(k3)

    def nu(self, s):
        return self.nu0 * (self.k1 * np.exp(self.k2 * s) + self.k3)

    def dnu(self, s):
        """d nu / d s."""
        return self.nu0 * self.k1 * self.k2 * np.exp(self.k2 * s)

    def Phi(self, s):
        """int_0^s nu(t) dt (twice the magnetic energy density as a function of s)."""
        if self.k1 == 0.0:
            return self.nu0 * self.k3 * s
        return self.nu0 * (self.k1 * np.expm1(self.k2 * s) / self.k2 + self.k3 * s)


class NewtonProblem:
    """Gauged implicit-Euler step with the nonlinear reluctivity in the conducting
    elements, on the free (r and p) edges, assembled globally."""

    def __init__(self, prob, model: Reluctivity | None = None, gauge_kw=None):
        self.prob = prob
        self.model = model if model is not None else Reluctivity(**prob.reluctivity)
        # linear part: the given nu everywhere except the conducting elements
        nu_lin = prob.nu_el.copy()
        self.nl_mask = prob.sigma_el > 0
        nu_lin[self.nl_mask] = 0.0
        lin = _with_nu(prob, nu_lin)
        self.asm = Assembled(lin)
        self.gauge = Gauge(prob, self.asm.lat, **(gauge_kw or {}))
        L = self.asm.lat
        self.free = np.nonzero(self.gauge.cls != CLS_E)[0]
        fidx = -np.ones(L.n_edges, dtype=np.int64)
        fidx[self.free] = np.arange(len(self.free))
        self.fidx = fidx
        n = len(self.free)
        Kg = sp.csr_matrix((n, n))
        Mg = sp.csr_matrix((n, n))
        self.R = []
        for s in range(prob.n_patches):
            g = self.asm.l2g[s]
            keep = np.nonzero(self.gauge.cls[g] != CLS_E)[0]
            Rs = sp.csr_matrix((np.ones(len(keep)), (fidx[g[keep]], keep)), shape=(n, len(g)))
            self.R.append(Rs)
            Kg = Kg + Rs @ self.asm.K[s] @ Rs.T
            Mg = Mg + Rs @ self.asm.M[s] @ Rs.T
        self.K_lin = Kg.tocsr()
        self.M = Mg.tocsr()
        self.n = n
        # nonlinear elements: U = DF c_hat (= det curl w) at every point, weights, det
        self.nl = []
        off = 0
        for s in range(prob.n_patches):
            E = int(np.prod(prob.patch_n_el(s)))
            mask = self.nl_mask[off:off + E]
            off += E
            if not mask.any():
                continue
            pe = PatchEval(prob, s)
            U = np.einsum("eqij,eqaj->eqai", pe.DF, pe.chat)[mask]   # (E', Q, nloc, 3)
            self.nl.append(dict(s=s, U=U, w=pe.w[mask], det=pe.det[mask], loc=pe.loc[mask]))

    # ------------------------------------------------------------------ fields
    def _patch_coeffs(self, a_free, item):
        g = self.asm.l2g[item["s"]]
        a_glob = np.zeros(self.asm.lat.n_edges)
        a_glob[self.free] = a_free
        return a_glob[g][item["loc"]]                      # (E', nloc)

    def _B(self, a_free, item):
        """curl A at the points of the nonlinear elements: (E', Q, 3)."""
        c = self._patch_coeffs(a_free, item)
        return np.einsum("ea,eqai->eqi", c, item["U"]) / item["det"][:, :, None]

    def _scatter(self, item, ve):
        """Element vectors (E', nloc) -> free-DOF vector."""
        s = item["s"]
        out = np.zeros(self.asm.K[s].shape[0])
        np.add.at(out, item["loc"].ravel(), ve.ravel())
        return self.R[s] @ out

    def N(self, a_free):
        """N(a)_i = sum_q w det nu(|B|^2) B . curl w_i = sum_q w nu B . U_i."""
        out = np.zeros(self.n)
        for it in self.nl:
            B = self._B(a_free, it)
            s2 = np.einsum("eqi,eqi->eq", B, B)
            ve = np.einsum("eq,eqi,eqai->ea", it["w"] * self.model.nu(s2), B, it["U"])
            out += self._scatter(it, ve)
        return out

    def K_t(self, a_free):
        """Tangent of N: sum_q (w / det) (nu U_i.U_k + 2 nu' (B.U_i)(B.U_k))."""
        rows, cols, vals = [], [], []
        for it in self.nl:
            s = it["s"]
            B = self._B(a_free, it)
            s2 = np.einsum("eqi,eqi->eq", B, B)
            c = it["w"] / it["det"]
            BU = np.einsum("eqi,eqai->eqa", B, it["U"])
            Ke = (np.einsum("eq,eqai,eqbi->eab", c * self.model.nu(s2), it["U"], it["U"])
                  + 2.0 * np.einsum("eq,eqa,eqb->eab", c * self.model.dnu(s2), BU, BU))
            nl = it["loc"].shape[1]
            r = np.repeat(it["loc"][:, :, None], nl, axis=2)
            cc = np.repeat(it["loc"][:, None, :], nl, axis=1)
            n_s = self.asm.K[s].shape[0]
            Kp = sp.coo_matrix((Ke.ravel(), (r.ravel(), cc.ravel())), shape=(n_s, n_s)).tocsr()
            Rs = self.R[s]
            rows.append(Rs @ Kp @ Rs.T)
        out = sp.csr_matrix((self.n, self.n))
        for m in rows:
            out = out + m
        return out.tocsr()

    def energy_nl(self, a_free):
        """sum over nonlinear elements of int 1/2 Phi(|B|^2)."""
        e = 0.0
        for it in self.nl:
            B = self._B(a_free, it)
            s2 = np.einsum("eqi,eqi->eq", B, B)
            e += 0.5 * np.sum(it["w"] * it["det"] * self.model.Phi(s2))
        return e

    # ------------------------------------------------------------------ step
    def rhs_vectors(self, a_prev_glob, j_glob):
        return self.M @ a_prev_glob[self.free], j_glob[self.free]

    def residual(self, a, a_prev, jf):
        """R(a) on the free DOFs (a, a_prev, jf free-DOF vectors)."""
        dt = self.prob.dt
        return self.M @ (a - a_prev) + dt * (self.K_lin @ a + self.N(a)) - dt * jf

    def jacobian(self, a):
        dt = self.prob.dt
        return (self.M + dt * (self.K_lin + self.K_t(a))).tocsc()

    def energy(self, a, a_prev, jf):
        dt = self.prob.dt
        return (0.5 * a @ (self.M @ a) - a @ (self.M @ a_prev)
                + dt * (0.5 * a @ (self.K_lin @ a) + self.energy_nl(a) - jf @ a))

    def step(self, a_prev_glob, j_glob, tol=1e-10, max_it=50):
        """One implicit-Euler step by Newton; returns the global state and the
        relative update norms ||d_k|| / ||a_{k+1}||."""
        a_prev = a_prev_glob[self.free]
        jf = j_glob[self.free]
        a = a_prev.copy()
        hist = []
        fn = np.linalg.norm(self.M @ a_prev + self.prob.dt * jf)
        self.last_residuals = []       # ||R(a_k)|| / ||M a^l + dt j|| before every update
        for _ in range(max_it):
            R = self.residual(a, a_prev, jf)
            self.last_residuals.append(np.linalg.norm(R) / fn)
            d = spla.spsolve(self.jacobian(a), -R)
            a = a + d
            rel = np.linalg.norm(d) / max(np.linalg.norm(a), 1e-300)
            hist.append(rel)
            if rel <= tol:
                break
        out = np.zeros(self.asm.lat.n_edges)
        out[self.free] = a
        return out, hist

    def run(self, n_steps, tol=1e-10):
        a = np.zeros(self.asm.lat.n_edges)
        out, its = [], []
        j = self.asm_load()
        for _ in range(n_steps):
            a, hist = self.step(a, j, tol)
            out.append(a)
            its.append(len(hist))
        return out, its

    def asm_load(self):
        return self.asm.j_global


def _with_nu(prob, nu_el):
    """A shallow copy of the problem with another per-element reluctivity."""
    import copy
    q = copy.copy(prob)
    q.nu_el = np.asarray(nu_el, dtype=float)
    return q
