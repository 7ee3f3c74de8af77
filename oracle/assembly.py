"""Patch matrices of Sec. 2.2:  (K_i)_jk = <nu curl w_k, curl w_j>,
(M_C)_jk = <sigma w_k, w_j>,  (j_i)_j = <J, w_j>, on curved spline patches.

Spaces: edge functions of component d are D_i (direction d) times N_j, N_k (the
other two directions), see ``bspline``.  Physical functions come from the
covariant Piola map  w = DF^{-T} w_hat,  curl w = DF curl_hat(w_hat) / det DF,
with the geometry map F = sum c_ijk N_i N_j N_k (degree-p splines of the same
knots).  Quadrature: Gauss-Legendre with p_d + 2 points per direction in every
element (the paper names no rule; this is the reading both implementations use).

The source enters through a potential T with J = curl T, so that
j_k = <T, curl w_k> (the integration-by-parts form; T vanishes near the boundary).
Plain, vectorised over elements; nothing fused beyond the definition.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .bspline import element_quadrature, h1_and_edge
from .lattice import Lattice


def quad_points(p: int) -> int:
    return p + 2


def _direction_data(t, p):
    """Per-element values of N, dN (p+1 active) and D (p active) at the Gauss points."""
    q = quad_points(p)
    x, w = element_quadrature(t, p, q)
    E = x.shape[0]
    N, dN, D = h1_and_edge(t, p, x.ravel())
    N = N.reshape(N.shape[0], E, q)
    dN = dN.reshape(dN.shape[0], E, q)
    D = D.reshape(D.shape[0], E, q)
    e = np.arange(E)
    Nl = np.stack([N[e + a, e, :] for a in range(p + 1)], axis=-1)      # (E, q, p+1)
    dNl = np.stack([dN[e + a, e, :] for a in range(p + 1)], axis=-1)
    Dl = np.stack([D[e + a, e, :] for a in range(p)], axis=-1)         # (E, q, p)
    return dict(E=E, q=q, p=p, w=w, N=Nl, dN=dNl, D=Dl)


class PatchEval:
    """Geometry and basis data of one patch at all quadrature points."""

    def __init__(self, prob, s):
        self.prob = prob
        self.s = s
        a, b, c = prob.patch_index(s)
        pd = prob.patch_degree(s)
        idx = (a, b, c)
        self.dd = [_direction_data(prob.knot_vector(d, idx[d]), pd[d]) for d in range(3)]
        X, Y, Z = self.dd
        self.n = [prob.patch_n_el(s)[d] + pd[d] for d in range(3)]
        n0, n1, n2 = self.n
        Ex, Ey, Ez = X["E"], Y["E"], Z["E"]
        qx, qy, qz = X["q"], Y["q"], Z["q"]
        self.E = Ex * Ey * Ez
        self.Q = qx * qy * qz
        # ---- geometry: F and DF at all points, shape (Ez,Ey,Ex,qz,qy,qx,...)
        net = prob.patch_ctrl(s)                                      # (n2, n1, n0, 3)
        ez, ey, ex = np.arange(Ez), np.arange(Ey), np.arange(Ex)
        cz = ez[:, None] + np.arange(Z["p"] + 1)[None, :]
        cy = ey[:, None] + np.arange(Y["p"] + 1)[None, :]
        cx = ex[:, None] + np.arange(X["p"] + 1)[None, :]
        loc_net = net[cz[:, None, None, :, None, None], cy[None, :, None, None, :, None],
                      cx[None, None, :, None, None, :]]               # (Ez,Ey,Ex,pz+1,py+1,px+1,3)
        F = np.einsum("ZYXcbar,Zkc,Yjb,Xia->ZYXkjir", loc_net, Z["N"], Y["N"], X["N"])
        Fx = np.einsum("ZYXcbar,Zkc,Yjb,Xia->ZYXkjir", loc_net, Z["N"], Y["N"], X["dN"])
        Fy = np.einsum("ZYXcbar,Zkc,Yjb,Xia->ZYXkjir", loc_net, Z["N"], Y["dN"], X["N"])
        Fz = np.einsum("ZYXcbar,Zkc,Yjb,Xia->ZYXkjir", loc_net, Z["dN"], Y["N"], X["N"])
        self.F = F.reshape(self.E, self.Q, 3)
        DF = np.stack([Fx, Fy, Fz], axis=-1)                          # columns = d/dxi_k
        self.DF = DF.reshape(self.E, self.Q, 3, 3)
        self.det = np.linalg.det(self.DF)
        self.DFinv = np.linalg.inv(self.DF)
        W = (Z["w"][:, None, None, :, None, None] * Y["w"][None, :, None, None, :, None]
             * X["w"][None, None, :, None, None, :])
        self.w = W.reshape(self.E, self.Q)
        # ---- reference basis: values and curls, element-local function index
        self._basis(n0, n1, n2)

    def _basis(self, n0, n1, n2):
        X, Y, Z = self.dd
        px, py, pz = X["p"], Y["p"], Z["p"]
        Ex, Ey, Ez = X["E"], Y["E"], Z["E"]
        vals, curls, locs = [], [], []

        def outer(fz, fy, fx):
            # (Ez,qz,c),(Ey,qy,b),(Ex,qx,a) -> (E, Q, nfun) with (c,b,a) a fastest
            v = np.einsum("Zkc,Yjb,Xia->ZYXkjicba", fz, fy, fx)
            return v.reshape(self.E, self.Q, -1)

        ez, ey, ex = np.meshgrid(np.arange(Ez), np.arange(Ey), np.arange(Ex), indexing="ij")
        ez, ey, ex = ez.ravel(), ey.ravel(), ex.ravel()

        def local_ids(comp, na, nb, nc, dims):
            c, b, a = np.meshgrid(np.arange(nc), np.arange(nb), np.arange(na), indexing="ij")
            i = ex[:, None] + a.ravel()[None, :]
            j = ey[:, None] + b.ravel()[None, :]
            k = ez[:, None] + c.ravel()[None, :]
            m0, m1, _ = dims
            off = [0, (n0 - 1) * n1 * n2, (n0 - 1) * n1 * n2 + n0 * (n1 - 1) * n2][comp]
            return off + i + m0 * (j + m1 * k)

        z = lambda a: np.zeros_like(a)
        # component 0: (D_i N_j N_k, 0, 0); curl = (0, D N dN_z, -D dN_y N)
        v = outer(Z["N"], Y["N"], X["D"])
        vals.append(np.stack([v, z(v), z(v)], -1))
        curls.append(np.stack([z(v), outer(Z["dN"], Y["N"], X["D"]), -outer(Z["N"], Y["dN"], X["D"])], -1))
        locs.append(local_ids(0, px, py + 1, pz + 1, (n0 - 1, n1, n2)))
        # component 1: (0, N D N, 0); curl = (-N D dN_z, 0, dN_x D N)
        v = outer(Z["N"], Y["D"], X["N"])
        vals.append(np.stack([z(v), v, z(v)], -1))
        curls.append(np.stack([-outer(Z["dN"], Y["D"], X["N"]), z(v), outer(Z["N"], Y["D"], X["dN"])], -1))
        locs.append(local_ids(1, px + 1, py, pz + 1, (n0, n1 - 1, n2)))
        # component 2: (0, 0, N N D); curl = (N dN_y D, -dN_x N D, 0)
        v = outer(Z["D"], Y["N"], X["N"])
        vals.append(np.stack([z(v), z(v), v], -1))
        curls.append(np.stack([outer(Z["D"], Y["dN"], X["N"]), -outer(Z["D"], Y["N"], X["dN"]), z(v)], -1))
        locs.append(local_ids(2, px + 1, py + 1, pz, (n0, n1, n2 - 1)))
        self.what = np.concatenate(vals, axis=2)      # (E, Q, nloc, 3)
        self.chat = np.concatenate(curls, axis=2)
        self.loc = np.concatenate(locs, axis=1)       # (E, nloc) patch-local DOF ids
        self.n_dofs = (n0 - 1) * n1 * n2 + n0 * (n1 - 1) * n2 + n0 * n1 * (n2 - 1)

    # physical fields at the points
    def phys_values(self):
        # w = DF^{-T} w_hat  ->  w_i = sum_j DFinv[j, i] w_hat_j
        return np.einsum("eqji,eqaj->eqai", self.DFinv, self.what)

    def phys_curls(self):
        # curl w = DF chat / det
        return np.einsum("eqij,eqaj->eqai", self.DF, self.chat) / self.det[:, :, None, None]

    def _scatter(self, Ke):
        rows = np.repeat(self.loc[:, :, None], self.loc.shape[1], axis=2)
        cols = np.repeat(self.loc[:, None, :], self.loc.shape[1], axis=1)
        return sp.coo_matrix((Ke.ravel(), (rows.ravel(), cols.ravel())),
                             shape=(self.n_dofs, self.n_dofs)).tocsr()

    def stiffness(self, nu_el):
        # K_e[a,b] = sum_q nu w det (curl_a . curl_b)
        U = np.einsum("eqij,eqaj->eqai", self.DF, self.chat)            # DF chat
        scale = np.sqrt(nu_el[:, None] * self.w / self.det)
        U = U * scale[:, :, None, None]
        U = U.transpose(0, 2, 1, 3).reshape(self.E, U.shape[2], -1)
        return self._scatter(U @ U.transpose(0, 2, 1))

    def mass(self, sigma_el):
        V = self.phys_values()
        scale = np.sqrt(sigma_el[:, None] * self.w * self.det)
        V = V * scale[:, :, None, None]
        V = V.transpose(0, 2, 1, 3).reshape(self.E, V.shape[2], -1)
        return self._scatter(V @ V.transpose(0, 2, 1))

    def load_from_potential(self, T):
        """j_k = <T, curl w_k> with T(x) -> (..., 3) evaluated at physical points."""
        Tq = T(self.F)                                                    # (E, Q, 3)
        U = np.einsum("eqij,eqaj->eqai", self.DF, self.chat)
        je = np.einsum("eqi,eqai,eq->ea", Tq, U, self.w)
        out = np.zeros(self.n_dofs)
        np.add.at(out, self.loc.ravel(), je.ravel())
        return out

    def load_from_field(self, Jf):
        """j_k = <J, w_k> for a pointwise field J(x) -> (..., 3)."""
        Jq = Jf(self.F)
        V = self.phys_values()
        je = np.einsum("eqi,eqai,eq->ea", Jq, V, self.w * self.det)
        out = np.zeros(self.n_dofs)
        np.add.at(out, self.loc.ravel(), je.ravel())
        return out


def coil_potential(coil):
    """T = T_z(r) chi(|z - zc| < hz) e_z, J = curl T an azimuthal coil current."""
    J0, r_in, r_out = coil["J0"], coil["r_in"], coil["r_out"]
    xc, yc, zc, hz = coil["xc"], coil["yc"], coil["zc"], coil["hz"]

    def T(x):
        r = np.sqrt((x[..., 0] - xc) ** 2 + (x[..., 1] - yc) ** 2)
        Tz = np.where(r <= r_in, J0 * (r_out - r_in), np.where(r < r_out, J0 * (r_out - r), 0.0))
        Tz = np.where(np.abs(x[..., 2] - zc) < hz, Tz, 0.0)
        out = np.zeros(x.shape)
        out[..., 2] = Tz
        return out
    return T


class Assembled:
    """Per-patch sparse K_s, M_s, coil load j_s (patch-local numbering) and the
    global load vector j (all lattice edges, Dirichlet ones included)."""

    def __init__(self, prob, lat: Lattice | None = None, with_load=True):
        self.prob = prob
        self.lat = lat or Lattice(prob)
        self.K, self.M, self.j, self.l2g = [], [], [], []
        T = coil_potential(prob.coil) if with_load else None
        for s in range(prob.n_patches):
            pe = PatchEval(prob, s)
            nu = prob.patch_nu(s).reshape(-1)
            sig = prob.patch_sigma(s).reshape(-1)
            self.K.append(pe.stiffness(nu))
            self.M.append(pe.mass(sig))
            self.j.append(pe.load_from_potential(T) if with_load else np.zeros(pe.n_dofs))
            self.l2g.append(self.lat.patch_local_to_global(s))
        self.j_global = np.zeros(self.lat.n_edges)
        for s in range(prob.n_patches):
            np.add.at(self.j_global, self.l2g[s], self.j[s])
