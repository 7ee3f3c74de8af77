"""Implicit-Euler time loop of Eq. (11): a^0 = 0, f^{l+1} = M a^l + dt j^{l+1}."""
from __future__ import annotations

import numpy as np

from .assembly import Assembled
from .gauge import Gauge
from .ietidp import Decomposition, IETIDP, gather_global, local_rhs, PRECOND_DIRICHLET
from .monolithic import Monolithic


class OracleProblem:
    """Everything the oracle derives from a problem description."""

    def __init__(self, prob, with_load=True, **gauge_kw):
        self.prob = prob
        self.asm = Assembled(prob, with_load=with_load)
        self.gauge = Gauge(prob, self.asm.lat, **gauge_kw)
        self._mono = None
        self._dec = None
        self._ieti = {}

    @property
    def mono(self):
        if self._mono is None:
            self._mono = Monolithic(self.prob, self.asm, self.gauge)
        return self._mono

    @property
    def dec(self):
        if self._dec is None:
            self._dec = Decomposition(self.prob, self.asm, self.gauge)
        return self._dec

    def ietidp(self, precond=PRECOND_DIRICHLET, deflation=False):
        key = (precond, bool(deflation))
        if key not in self._ieti:
            self._ieti[key] = IETIDP(self.dec, precond, deflation=deflation)
        return self._ieti[key]

    def run_monolithic(self, n_steps, j_of_step=None, a0=None):
        a = np.zeros(self.asm.lat.n_edges) if a0 is None else a0.copy()
        out = []
        for l in range(n_steps):
            j = self.asm.j_global if j_of_step is None else j_of_step(l + 1)
            a = self.mono.step(a, j)
            out.append(a)
        return out

    def run_ietidp(self, n_steps, tol, precond=PRECOND_DIRICHLET, j_of_step=None, a0=None, deflation=False):
        I = self.ietidp(precond, deflation)
        a = np.zeros(self.asm.lat.n_edges) if a0 is None else a0.copy()
        out, its = [], []
        for l in range(n_steps):
            j = self.asm.j_global if j_of_step is None else j_of_step(l + 1)
            a_loc, lam, it, res = I.solve(local_rhs(self.dec, a, j), tol)
            a = gather_global(self.dec, a_loc)
            out.append(a)
            its.append(it)
        return out, its
