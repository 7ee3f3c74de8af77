"""The gauged implicit-Euler system of Eq. (11) on the unique global unknowns.

With a_e = 0 and the interface copies identified, Eq. (11) (equivalently the
system after Eq. (12), of which the dual-primal form is an exact rewrite) is the
assembled sparse system  W_g a = M_g a^l + dt j  over the r and p edges, with
W_g = sum_s R_s^T (M_s + dt K_s) R_s.  Solved with SuperLU (library routine).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .gauge import CLS_E


class Monolithic:
    def __init__(self, prob, asm, gauge):
        self.prob = prob
        L = asm.lat
        self.free = np.nonzero(gauge.cls != CLS_E)[0]
        fidx = -np.ones(L.n_edges, dtype=np.int64)
        fidx[self.free] = np.arange(len(self.free))
        n = len(self.free)
        Wg = sp.csr_matrix((n, n))
        Mg = sp.csr_matrix((n, n))
        for s in range(prob.n_patches):
            g = asm.l2g[s]
            keep = np.nonzero(gauge.cls[g] != CLS_E)[0]
            R = sp.csr_matrix((np.ones(len(keep)), (fidx[g[keep]], keep)), shape=(n, len(g)))
            Ws = asm.M[s] + prob.dt * asm.K[s]
            Wg = Wg + R @ Ws @ R.T
            Mg = Mg + R @ asm.M[s] @ R.T
        self.W = Wg.tocsc()
        self.M = Mg.tocsr()
        self.n_edges = L.n_edges
        self._lu = None

    def factor(self):
        if self._lu is None:
            self._lu = spla.splu(self.W)
        return self._lu

    def rhs(self, a_global, j_global):
        return self.M @ a_global[self.free] + self.prob.dt * j_global[self.free]

    def step(self, a_global, j_global):
        x = self.factor().solve(self.rhs(a_global, j_global))
        out = np.zeros(self.n_edges)
        out[self.free] = x
        return out

    def residual(self, a_next, a_prev, j_global):
        """||f - W a_next|| / ||f|| for a candidate solution."""
        f = self.rhs(a_prev, j_global)
        r = f - self.W @ a_next[self.free]
        return np.linalg.norm(r) / np.linalg.norm(f)
