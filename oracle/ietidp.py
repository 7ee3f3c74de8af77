"""Dual-primal tearing and interconnecting for one implicit-Euler step (Sec. 3).

The step system is Eq. (11): [W, dt B^T; dt B, 0][a; m] = [f; 0] with W = M + dt K
and f = M a^l + dt j^{l+1}.  Splitting a into e / p / r (``gauge``) and writing
a_p = N p gives the unnumbered system after Eq. (12):

    [ W_rr      W_rp N     dt B_rr^T ] [a_r]   [ f_r      ]
    [ N^T W_pr  N^T W_pp N  0        ] [ p ] = [ N^T f_p  ]      (a_e = 0)
    [ dt B_rr   0           0        ] [m_r]   [ 0        ]

solved, as the paper does after Farhat et al. (2001), by two sequential Schur
complements: the local r-blocks (one Cholesky per patch), then the primal coarse
block S_c = sum_s A_s^T (W_pp - W_pr W_rr^{-1} W_rp) A_s, leaving the dual problem
F lambda = d, solved by PCG with the Dirichlet preconditioner (Sec. 4: "without
scaling"; the scaled variants of the outlook are options).  The factor dt of the
constraint rows is absorbed into lambda (lambda = dt m_r), which changes neither
a nor the CG iterates' residual ratios.

Readings: one multiplier per pair of copies of a shared r-DOF (fully redundant;
sign +1 on the lower patch id, as B = [R_C, -R_I]); the load of a DOF shared by k
patches is split 1/k per patch (any split gives the same assembled system); PCG
starts from lambda = 0 and stops when ||r_k|| <= tol ||d||.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .gauge import CLS_E, CLS_P, CLS_R

PRECOND_NONE, PRECOND_DIRICHLET, PRECOND_MULT, PRECOND_STIFF = 0, 1, 2, 3


class Decomposition:
    """Index sets of every patch, multipliers B_s and primal maps A_s."""

    def __init__(self, prob, asm, gauge):
        self.prob = prob
        self.asm = asm
        self.gauge = gauge
        L = asm.lat
        cls = gauge.cls
        self.n_patches = prob.n_patches
        self.i_loc, self.b_loc, self.p_loc = [], [], []
        copies = []                          # (global edge, patch, position in b)
        for s in range(self.n_patches):
            g = asm.l2g[s]
            c = cls[g]
            sh = L.n_share[g] >= 2
            i_loc = np.nonzero((c == CLS_R) & ~sh)[0]
            b_loc = np.nonzero((c == CLS_R) & sh)[0]
            p_loc = np.nonzero(c == CLS_P)[0]
            self.i_loc.append(i_loc); self.b_loc.append(b_loc); self.p_loc.append(p_loc)
            for k, lid in enumerate(b_loc):
                copies.append((int(g[lid]), s, k))
        copies.sort()
        # fully redundant multipliers, ordered by (edge, lower patch, upper patch)
        self.lam = []                        # (edge, s, pos_s, t, pos_t)
        i = 0
        while i < len(copies):
            j = i
            while j < len(copies) and copies[j][0] == copies[i][0]:
                j += 1
            grp = copies[i:j]
            for a in range(len(grp)):
                for b in range(a + 1, len(grp)):
                    self.lam.append((grp[a][0], grp[a][1], grp[a][2], grp[b][1], grp[b][2]))
            i = j
        self.m = len(self.lam)
        # coarse numbering: primal edges in ascending id
        prim = np.nonzero(cls == CLS_P)[0]
        self.n_coarse = len(prim)
        cidx = -np.ones(L.n_edges, dtype=np.int64)
        cidx[prim] = np.arange(len(prim))
        self.A = [cidx[asm.l2g[s][self.p_loc[s]]] for s in range(self.n_patches)]
        # B_s acting on the b-part of patch s
        self.B = []
        for s in range(self.n_patches):
            rows, cols, vals = [], [], []
            for q, (g, s1, k1, s2, k2) in enumerate(self.lam):
                if s1 == s:
                    rows.append(q); cols.append(k1); vals.append(1.0)
                if s2 == s:
                    rows.append(q); cols.append(k2); vals.append(-1.0)
            self.B.append(sp.csr_matrix((vals, (rows, cols)), shape=(self.m, len(self.b_loc[s]))))
        # load split weights (1/k for a DOF shared by k patches)
        self.load_w = [1.0 / L.n_share[asm.l2g[s]] for s in range(self.n_patches)]

    def pair_space(self):
        """U (m x k, sparse): one column per pair of patches (s < t) joined by at least one
        multiplier, the indicator of that pair's multipliers.  U^T lambda are the
        patch-pair sums of lambda, the deflation space of the balanced preconditioner
        (Sec. 5 recommends deflation in the Dirichlet preconditioner; this is that
        recommendation's reading, see IETIDP)."""
        pairs = sorted({(s1, s2) for (_, s1, _, s2, _) in self.lam})
        col = {p: j for j, p in enumerate(pairs)}
        cols = [col[(s1, s2)] for (_, s1, _, s2, _) in self.lam]
        return sp.csr_matrix((np.ones(self.m), (np.arange(self.m), cols)), shape=(self.m, len(pairs)))

    def scaled_B(self, W_diag, mode):
        """B_D,s: entry of the copy in s for the multiplier (s,t) times delta_t^dagger."""
        if mode in (PRECOND_NONE, PRECOND_DIRICHLET):
            return self.B
        L = self.asm.lat
        rho_sum = {}
        rho = []
        for s in range(self.n_patches):
            g = self.asm.l2g[s][self.b_loc[s]]
            r = np.ones(len(g)) if mode == PRECOND_MULT else W_diag[s][self.b_loc[s]]
            rho.append(r)
            for gg, rr in zip(g, r):
                rho_sum[int(gg)] = rho_sum.get(int(gg), 0.0) + rr
        out = []
        for s in range(self.n_patches):
            rows, cols, vals = [], [], []
            for q, (g, s1, k1, s2, k2) in enumerate(self.lam):
                if s1 == s:
                    rows.append(q); cols.append(k1); vals.append(rho[s2][k2] / rho_sum[g])
                if s2 == s:
                    rows.append(q); cols.append(k2); vals.append(-rho[s1][k1] / rho_sum[g])
            out.append(sp.csr_matrix((vals, (rows, cols)), shape=(self.m, len(self.b_loc[s]))))
        return out


class IETIDP:
    """FETI-DP operators for W_s = M_s + dt K_s (dense local blocks, LAPACK).

    deflation=True (or an explicit U) wraps the preconditioner M in the balancing form
        M_bal = (I - P) M (I - P)^T + U E^{-1} U^T,  P = U E^{-1} U^T F,  E = U^T F U,
    with U the patch-pair space of ``Decomposition.pair_space``: Sec. 5 recommends
    "deflation in the Dirichlet preconditioner" without fixing its form; this is the
    balancing (projector) form of a deflation space for dual-primal methods, which
    keeps M_bal symmetric so plain PCG applies and leaves the solution unchanged."""

    def __init__(self, dec: Decomposition, precond=PRECOND_DIRICHLET, deflation=False, U=None):
        self.dec = dec
        asm = dec.asm
        dt = dec.prob.dt
        self.precond = precond
        self.Wrr_f, self.Wrp, self.Wpp, self.Wbb_S, self.nr, self.nb, self.ni = [], [], [], [], [], [], []
        self.Phi = []
        n_c = dec.n_coarse
        Sc = np.zeros((n_c, n_c))
        W_diag = []
        self.W = []
        for s in range(dec.n_patches):
            W = (asm.M[s] + dt * asm.K[s]).toarray()
            self.W.append(W)
            W_diag.append(np.diag(W).copy())
            r = np.concatenate([dec.i_loc[s], dec.b_loc[s]])
            p = dec.p_loc[s]
            Wrr = W[np.ix_(r, r)]
            Wrp = W[np.ix_(r, p)]
            Wpp = W[np.ix_(p, p)]
            cf = sla.cho_factor(Wrr, lower=True)
            Phi = sla.cho_solve(cf, Wrp)
            Cs = Wpp - Wrp.T @ Phi
            A = dec.A[s]
            Sc[np.ix_(A, A)] += Cs
            self.Wrr_f.append(cf); self.Wrp.append(Wrp); self.Wpp.append(Wpp); self.Phi.append(Phi)
            ni, nb = len(dec.i_loc[s]), len(dec.b_loc[s])
            self.ni.append(ni); self.nb.append(nb); self.nr.append(ni + nb)
            # Dirichlet preconditioner block: S_bb = W_bb - W_bi W_ii^{-1} W_ib
            Wii = Wrr[:ni, :ni]
            Wib = Wrr[:ni, ni:]
            Wbb = Wrr[ni:, ni:]
            if ni:
                Sbb = Wbb - Wib.T @ sla.cho_solve(sla.cho_factor(Wii, lower=True), Wib)
            else:
                Sbb = Wbb
            self.Wbb_S.append(Sbb)
        self.Sc = Sc
        self.Sc_f = sla.cho_factor(Sc, lower=True) if n_c else None
        self.BD = dec.scaled_B(W_diag, precond)
        self.U = None
        if deflation or U is not None:
            self.U = dec.pair_space() if U is None else sp.csr_matrix(U)
            Ud = self.U.toarray()
            self.FU = np.column_stack([self.apply_F(Ud[:, j]) for j in range(Ud.shape[1])])
            self.E_f = sla.cho_factor(self.U.T @ self.FU, lower=True)

    # B_s^T acting from lambda-space to the r-space (zeros on interior DOFs)
    def _BT(self, s, v):
        out = np.zeros(self.nr[s])
        out[self.ni[s]:] = self.dec.B[s].T @ v
        return out

    def _B(self, s, x):
        return self.dec.B[s] @ x[self.ni[s]:]

    def _coarse_solve(self, c):
        return sla.cho_solve(self.Sc_f, c) if self.dec.n_coarse else c

    def apply_F(self, v):
        dec = self.dec
        xs = []
        c = np.zeros(dec.n_coarse)
        for s in range(dec.n_patches):
            x = sla.cho_solve(self.Wrr_f[s], self._BT(s, v))
            xs.append(x)
            np.add.at(c, dec.A[s], self.Wrp[s].T @ x)
        q = self._coarse_solve(c)
        out = np.zeros(dec.m)
        for s in range(dec.n_patches):
            y = xs[s] + self.Phi[s] @ q[dec.A[s]]
            out += self._B(s, y)
        return out

    def _dirichlet(self, r):
        if self.precond == PRECOND_NONE:
            return r.copy()
        out = np.zeros(self.dec.m)
        for s in range(self.dec.n_patches):
            out += self.BD[s] @ (self.Wbb_S[s] @ (self.BD[s].T @ r))
        return out

    def apply_precond(self, r):
        if self.U is None:
            return self._dirichlet(r)
        # M_bal r = (I - P) M (I - P)^T r + U E^{-1} U^T r, with (I - P)^T = I - F U E^{-1} U^T
        ur = self.U.T @ r
        w = self._dirichlet(r - self.FU @ sla.cho_solve(self.E_f, ur))
        return w + self.U @ sla.cho_solve(self.E_f, ur - self.FU.T @ w)

    def rhs(self, f_loc):
        """d and g_c for local right-hand sides f_s (patch-local numbering)."""
        dec = self.dec
        xs, fr = [], []
        g = np.zeros(dec.n_coarse)
        for s in range(dec.n_patches):
            r = np.concatenate([dec.i_loc[s], dec.b_loc[s]])
            x = sla.cho_solve(self.Wrr_f[s], f_loc[s][r])
            xs.append(x)
            np.add.at(g, dec.A[s], f_loc[s][dec.p_loc[s]] - self.Wrp[s].T @ x)
        q0 = self._coarse_solve(g)
        d = np.zeros(dec.m)
        for s in range(dec.n_patches):
            d += self._B(s, xs[s] - self.Phi[s] @ q0[dec.A[s]])
        return d, g

    def recover(self, f_loc, lam, g):
        dec = self.dec
        c = g.copy()
        us = []
        for s in range(dec.n_patches):
            u = self._BT(s, lam)
            us.append(u)
            np.add.at(c, dec.A[s], self.Wrp[s].T @ sla.cho_solve(self.Wrr_f[s], u))
        p = self._coarse_solve(c)
        a_loc = []
        for s in range(dec.n_patches):
            r = np.concatenate([dec.i_loc[s], dec.b_loc[s]])
            rhs = f_loc[s][r] - self.Wrp[s] @ p[dec.A[s]] - us[s]
            a = np.zeros(len(f_loc[s]))
            a[r] = sla.cho_solve(self.Wrr_f[s], rhs)
            a[dec.p_loc[s]] = p[dec.A[s]]
            a_loc.append(a)
        return a_loc, p

    def pcg(self, d, tol, max_it=5000):
        lam = np.zeros_like(d)
        r = d.copy()
        nd = np.linalg.norm(d)
        if nd == 0.0:
            return lam, 0, 0.0
        z = self.apply_precond(r)
        p = z.copy()
        rz = r @ z
        it = 0
        res = 1.0
        while it < max_it:
            q = self.apply_F(p)
            alpha = rz / (p @ q)
            lam += alpha * p
            r -= alpha * q
            it += 1
            res = np.linalg.norm(r) / nd
            if res <= tol:
                break
            z = self.apply_precond(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        return lam, it, res

    def solve(self, f_loc, tol):
        d, g = self.rhs(f_loc)
        lam, it, res = self.pcg(d, tol)
        a_loc, _ = self.recover(f_loc, lam, g)
        return a_loc, lam, it, res

    def dense_F_and_M(self):
        """Explicit F and M^{-1} (small problems only; used by the pins)."""
        m = self.dec.m
        F = np.column_stack([self.apply_F(e) for e in np.eye(m)])
        Mi = np.column_stack([self.apply_precond(e) for e in np.eye(m)])
        return F, Mi


def gather_global(dec, a_loc):
    """Global coefficient vector: r / p values from the lowest patch holding them, e = 0."""
    L = dec.asm.lat
    a = np.zeros(L.n_edges)
    done = np.zeros(L.n_edges, dtype=bool)
    for s in range(dec.n_patches):
        g = dec.asm.l2g[s]
        keep = dec.gauge.cls[g] != CLS_E
        sel = keep & ~done[g]
        a[g[sel]] = a_loc[s][sel]
        done[g[sel]] = True
    return a


def local_rhs(dec, a_global, j_global):
    """f_s = M_s a_s + dt * w_s * j_s with the 1/k load split (e entries unused)."""
    dt = dec.prob.dt
    out = []
    for s in range(dec.n_patches):
        g = dec.asm.l2g[s]
        out.append(dec.asm.M[s] @ a_global[g] + dt * dec.load_w[s] * j_global[g])
    return out
