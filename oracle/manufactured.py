"""Manufactured solutions and error norms (Sec. 4).

Sec. 4 prescribes A = e^{-t} (sin x cos y cos z, -2 cos x sin y cos z,
cos x cos y sin z) with inhomogeneous data.  The pins here use a field with the
same structure that already has zero tangential trace on the unit cube, so the
homogeneous PEC condition of Sec. 2 holds without lifting:

    A*(x) = (sin(pi y) sin(pi z), sin(pi z) sin(pi x), sin(pi x) sin(pi y)),
    div A* = 0,  curl curl A* = 2 pi^2 A*.

With A(x, t) = e^{-t} A*(x) and constant sigma, nu per region, Eq. (5) gives the
source J = e^{-t} (2 pi^2 nu - sigma) A*.  Errors follow the paper's measures:
eps_B for B = curl A on Omega and eps_E for E_C = -dA/dt on Omega_C (relative L2,
the reading of the cited definition that we use).
"""
from __future__ import annotations

import numpy as np

from .assembly import PatchEval

PI = np.pi


def A_star(x):
    sx, sy, sz = np.sin(PI * x[..., 0]), np.sin(PI * x[..., 1]), np.sin(PI * x[..., 2])
    return np.stack([sy * sz, sz * sx, sx * sy], axis=-1)


def curl_A_star(x):
    sx, sy, sz = np.sin(PI * x[..., 0]), np.sin(PI * x[..., 1]), np.sin(PI * x[..., 2])
    cx, cy, cz = np.cos(PI * x[..., 0]), np.cos(PI * x[..., 1]), np.cos(PI * x[..., 2])
    # curl (Ax, Ay, Az) = (dAz/dy - dAy/dz, dAx/dz - dAz/dx, dAy/dx - dAx/dy)
    return PI * np.stack([sx * cy - sx * cz, sy * cz - cx * sy, cx * sz - cy * sz], axis=-1)


class FieldEval:
    """Values and curls of a discrete field at all quadrature points of all patches."""

    def __init__(self, prob, asm):
        self.pe = [PatchEval(prob, s) for s in range(prob.n_patches)]
        self.asm = asm
        self.prob = prob
        self.vals = [pe.phys_values() for pe in self.pe]
        self.curls = [pe.phys_curls() for pe in self.pe]

    def load(self, field):
        out = np.zeros(self.asm.lat.n_edges)
        for s, pe in enumerate(self.pe):
            np.add.at(out, self.asm.l2g[s], pe.load_from_field(field))
        return out

    def errors(self, a_global, A_fn, curlA_fn, region_sigma_positive=True):
        """(||A - A_h||_{L2(Omega_C)}/||A||, ||curl A - curl A_h||_{L2(Omega)}/||curl A||)."""
        eA = nA = eB = nB = 0.0
        for s, pe in enumerate(self.pe):
            c = a_global[self.asm.l2g[s]][pe.loc]                         # (E, nloc)
            Ah = np.einsum("ea,eqai->eqi", c, self.vals[s])
            Bh = np.einsum("ea,eqai->eqi", c, self.curls[s])
            A = A_fn(pe.F)
            B = curlA_fn(pe.F)
            wq = pe.w * pe.det
            cond = (self.prob.patch_sigma(s).reshape(-1) > 0)[:, None]
            eA += np.sum(wq * cond * np.sum((A - Ah) ** 2, -1))
            nA += np.sum(wq * cond * np.sum(A ** 2, -1))
            eB += np.sum(wq * np.sum((B - Bh) ** 2, -1))
            nB += np.sum(wq * np.sum(B ** 2, -1))
        return np.sqrt(eA / max(nA, 1e-300)), np.sqrt(eB / nB)
