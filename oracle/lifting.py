"""Inhomogeneous tangential boundary data and the lifted implicit-Euler run of Sec. 4.

Test infrastructure (the oracle); the library never calls it.

Sec. 4 prescribes A = e^{-t} A13 with A13 = (sin x cos y cos z, -2 cos x sin y cos z,
cos x cos y sin z) on the unit cube and derives boundary, source and initial terms
from it.  The boundary values enter by lifting: the Dirichlet DOFs (edges tangential
to and lying on the boundary) carry a_D, the L2 projection on the boundary of the
tangential trace of A onto the tangential traces of those edge functions,

    minimise  sum over boundary faces  int |n x (A_h - A)|^2 dS,

and the free DOFs solve the gauged system of Eq. (11) with the lifting moved to the
right-hand side:

    W_ff a_0^{l+1} = M_ff a_0^l + M_fD a_D^l - W_fD a_D^{l+1} + dt j^{l+1}_f,

a^l = a_0^l + a_D^l.  The initial state is the sigma-weighted L2 projection of
A(0) (only M a^0 enters the first step).  Implemented for axis-aligned
(identity-mapped) patches, the geometry of Sec. 4: a face's tangential traces are
then tensor products of 1-D B-splines and the face integrals factor.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assembly import quad_points
from .bspline import element_quadrature, h1_and_edge
from .gauge import CLS_E


def A13(x):
    """The field of Eq. (13) at t = 0."""
    sx, sy, sz = np.sin(x[..., 0]), np.sin(x[..., 1]), np.sin(x[..., 2])
    cx, cy, cz = np.cos(x[..., 0]), np.cos(x[..., 1]), np.cos(x[..., 2])
    return np.stack([sx * cy * cz, -2.0 * cx * sy * cz, cx * cy * sz], axis=-1)


def curl_A13(x):
    """curl A13 = (-3 cos x sin y sin z, 0, 3 sin x sin y cos z)."""
    sx, sy, sz = np.sin(x[..., 0]), np.sin(x[..., 1]), np.sin(x[..., 2])
    cx, cy, cz = np.cos(x[..., 0]), np.cos(x[..., 1]), np.cos(x[..., 2])
    # A = (sx cy cz, -2 cx sy cz, cx cy sz)
    # curl_x = dAz/dy - dAy/dz = -cx sy sz - 2 cx sy sz = -3 cx sy sz
    # curl_y = dAx/dz - dAz/dx = -sx cy sz + sx cy sz = 0
    # curl_z = dAy/dx - dAx/dy = 2 sx sy cz + sx sy cz = 3 sx sy cz
    return np.stack([-3.0 * cx * sy * sz, 0.0 * sx, 3.0 * sx * sy * cz], axis=-1)


def _box(prob, s):
    """Corner and edge lengths of an axis-aligned patch (asserts the identity map)."""
    net = prob.patch_ctrl(s)                       # (n2, n1, n0, 3)
    lo, hi = net[0, 0, 0], net[-1, -1, -1]
    L = hi - lo
    ne, p = prob.patch_n_el(s), prob.patch_degree(s)
    a = prob.patch_index(s)
    for d in range(3):
        t = prob.knot_vector(d, a[d])
        g = np.array([t[i + 1:i + p[d] + 1].mean() for i in range(ne[d] + p[d])])
        coord = np.moveaxis(net[..., d], [2, 1, 0], [0, 1, 2])   # (n0, n1, n2)
        want = lo[d] + L[d] * g
        shape = [1, 1, 1]
        shape[d] = -1
        assert np.allclose(coord, want.reshape(shape)), "boundary lifting needs axis-aligned patches"
    return lo, L


def _local_id(comp, idx, n):
    """Patch-local DOF id of edge function (comp, i, j, k) (component-major, i fastest)."""
    dims = [n[d] - (1 if d == comp else 0) for d in range(3)]
    off = [0, (n[0] - 1) * n[1] * n[2], (n[0] - 1) * n[1] * n[2] + n[0] * (n[1] - 1) * n[2]][comp]
    i, j, k = idx
    return off + i + dims[0] * (j + dims[1] * k)


def boundary_projection(prob, asm, A_fn):
    """Global vector with a_D on the Dirichlet DOFs (zero elsewhere): the boundary L2
    projection of the tangential trace of A_fn described in the module docstring."""
    lat = asm.lat
    rows, cols, vals = [], [], []
    rhs = np.zeros(lat.n_edges)
    for s in range(prob.n_patches):
        a = prob.patch_index(s)
        lo, L = _box(prob, s)
        ne, p = prob.patch_n_el(s), prob.patch_degree(s)
        n = [ne[d] + p[d] for d in range(3)]
        l2g = lat.patch_local_to_global(s)
        # 1-D data per direction at Gauss points: N (n, X), D (n-1, X), weights (X,)
        one = []
        for d in range(3):
            t = prob.knot_vector(d, a[d])
            x, w = element_quadrature(t, p[d], quad_points(p[d]))
            N, _, D = h1_and_edge(t, p[d], x.ravel())
            one.append(dict(x=x.ravel(), w=w.ravel(), N=N, D=D))
        for d in range(3):                          # face normal direction
            for side in (0, 1):
                if not ((side == 0 and a[d] == 0) or (side == 1 and a[d] == prob.P[d] - 1)):
                    continue
                fixed = 0 if side == 0 else n[d] - 1   # the only N in direction d non-zero there
                xd = lo[d] + side * L[d]
                e, f = [c for c in range(3) if c != d]
                for comp, other in ((e, f), (f, e)):  # tangential component, the other direction
                    B1 = one[comp]["D"]             # edge functions along comp
                    B2 = one[other]["N"]
                    w1, w2 = one[comp]["w"], one[other]["w"]
                    # physical points of the face grid
                    X = np.zeros((len(w1), len(w2), 3))
                    X[..., d] = xd
                    X[..., comp] = (lo[comp] + L[comp] * one[comp]["x"])[:, None]
                    X[..., other] = (lo[other] + L[other] * one[other]["x"])[None, :]
                    Ac = A_fn(X)[..., comp]
                    # covariant Piola on a box: tangential value D N / L_comp; dS = L_e L_f du dv
                    M1 = (B1 * w1) @ B1.T / L[comp] ** 2
                    M2 = (B2 * w2) @ B2.T
                    Mf = np.kron(M1, M2) * L[comp] * L[other]          # index (i1, i2), i2 fastest
                    bf = ((B1 * w1) @ Ac @ (B2 * w2).T / L[comp] * L[comp] * L[other]).ravel()
                    ids = np.empty((B1.shape[0], B2.shape[0]), dtype=np.int64)
                    for i1 in range(B1.shape[0]):
                        for i2 in range(B2.shape[0]):
                            idx = [0, 0, 0]
                            idx[d], idx[comp], idx[other] = fixed, i1, i2
                            ids[i1, i2] = l2g[_local_id(comp, idx, n)]
                    g = ids.ravel()
                    rr, cc = np.meshgrid(g, g, indexing="ij")
                    rows.append(rr.ravel())
                    cols.append(cc.ravel())
                    vals.append(Mf.ravel())
                    np.add.at(rhs, g, bf)
    Mb = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(lat.n_edges, lat.n_edges)).tocsr()
    bnd = np.unique(np.concatenate(rows))
    sol = spla.spsolve(Mb[bnd][:, bnd].tocsc(), rhs[bnd])
    out = np.zeros(lat.n_edges)
    out[bnd] = sol
    return out, bnd


def global_matrices(prob, asm):
    """W = sum_s R_s^T (M_s + dt K_s) R_s and M over all lattice edges (CSR)."""
    n = asm.lat.n_edges
    W = sp.csr_matrix((n, n))
    M = sp.csr_matrix((n, n))
    for s in range(prob.n_patches):
        g = asm.l2g[s]
        R = sp.csr_matrix((np.ones(len(g)), (g, np.arange(len(g)))), shape=(n, len(g)))
        W = W + R @ (asm.M[s] + prob.dt * asm.K[s]) @ R.T
        M = M + R @ asm.M[s] @ R.T
    return W.tocsr(), M.tocsr()


class LiftedRun:
    """Right-hand sides, initial state and the monolithic reference of the lifted
    implicit-Euler run for A(x, t) = g(t) A_fn(x) with g(t) = exp(-t)."""

    def __init__(self, op, A_fn, J_fn, sigma_fn):
        prob, asm = op.prob, op.asm
        self.op = op
        self.dt = prob.dt
        self.W, self.M = global_matrices(prob, asm)
        self.aD_star, self.bnd = boundary_projection(prob, asm, A_fn)
        cls = op.gauge.cls
        self.free = np.nonzero(cls != CLS_E)[0]
        assert not np.any(np.isin(self.bnd, self.free)), "boundary DOFs must be eliminated"
        from .manufactured import FieldEval
        self.fe = FieldEval(prob, asm)
        self.jJ = self.fe.load(J_fn)                       # <J(., t) / g(t), w>
        b0 = self.fe.load(lambda x: sigma_fn(x)[..., None] * A_fn(x))
        # sigma-weighted projection of A(0): M a^0 = b0 on the rows the mass reaches
        f = self.free
        Mff = self.M[f][:, f]
        C = np.nonzero(Mff.diagonal() > 0)[0]
        rhs = b0[f] - self.M[f] @ self.aD_star             # the lifting's share of M a^0
        a0 = np.zeros(len(f))
        a0[C] = spla.spsolve(Mff[C][:, C].tocsc(), rhs[C])
        self.a0 = np.zeros(asm.lat.n_edges)
        self.a0[f] = a0                                    # homogeneous part of a^0

    def g(self, t):
        return np.exp(-t)

    def j_step(self, l):
        """Load vector for step l (a^{l-1} -> a^l) of the homogeneous part: the source
        plus the lifting terms (M a_D^{l-1} - W a_D^l) / dt on the free rows."""
        t1, t0 = l * self.dt, (l - 1) * self.dt
        lift = (self.M @ (self.g(t0) * self.aD_star) - self.W @ (self.g(t1) * self.aD_star)) / self.dt
        j = self.g(t1) * self.jJ + lift
        j[np.setdiff1d(np.arange(len(j)), self.free)] = 0.0
        return j

    def total(self, a0_part, t):
        return a0_part + self.g(t) * self.aD_star

    def run_monolithic(self, n_t):
        """Homogeneous parts a_0^l, l = 1..n_t, by the oracle's sparse direct solve."""
        return self.op.run_monolithic(n_t, j_of_step=self.j_step, a0=self.a0)
