"""Problem descriptions for the tree-cotree IETI-DP eddy-current solver.

A problem is the unit cube split into a structured grid of P0 x P1 x P2 hexahedral
patches.  Slab ``a`` in direction ``d`` carries ``n_el[d][a]`` elements and the
H^1 spline degree ``degree[d][a]``; every patch of that slab uses the same knot
vector in that direction, so neighbouring patches match on shared faces (the
conformity the method requires, Sec. 2.2).

Data layout (mirrored by the C ABI in ``include/ieti.h``):

* patch ``s = a + P0*(b + P1*c)``;
* ``knots[d]``: concatenation over slabs of the full open knot vectors on [0, 1]
  (length ``n_el + 2*p + 1`` each);
* ``ctrl``: concatenation over patches of the geometry control nets, each of shape
  ``(n2, n1, n0, 3)`` (index ``i`` in direction 0 fastest) with ``n_d = n_el_d + p_d``
  points per direction; the geometry map uses the degree-``p`` B-splines of the
  same knot vectors.  The unperturbed net sits at the knot averages (the identity
  map); ``perturb`` moves the strictly interior control points by
  U(-perturb, perturb) times the element size, per coordinate;
* ``sigma_el``, ``nu_el``: per element, patch-major, elements ``(e2, e1, e0)`` with
  ``e0`` fastest;
* ``coil``: parameters of the source potential ``T = T_z(r) * chi(|z - zc| < hz) e_z``
  with ``T_z = J0*(r_out - r)`` on ``r_in < r < r_out``, ``J0*(r_out - r_in)`` for
  ``r <= r_in`` and 0 beyond, ``r`` the distance to the axis ``x = xc, y = yc``.
  ``curl T`` is an azimuthal current of amplitude ``J0`` in the shell.
* ``reluctivity``: ``None`` (linear: ``nu_el`` everywhere) or the parameters
  ``nu0, k1, k2, k3`` of ``nu(|B|) = nu0 (k1 exp(k2 |B|^2) + k3)``, which then
  replaces ``nu_el`` in the conducting elements (``sigma_el > 0``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


@dataclass
class Problem:
    name: str
    P: tuple                      # patches per direction
    n_el: list                    # [d] -> int array (P_d,)
    degree: list                  # [d] -> int array (P_d,)
    knots: list                   # [d] -> float array, concatenated open knot vectors
    ctrl: np.ndarray              # float64, concatenated control nets
    sigma_el: np.ndarray          # float64 per element
    nu_el: np.ndarray             # float64 per element
    dt: float
    n_steps: int
    cg_tol: float = 1e-10
    coil: dict = field(default_factory=dict)
    seed: int = 0
    reluctivity: dict | None = None

    # ---- plain bookkeeping (sizes and offsets; no spline arithmetic) ----
    @property
    def n_patches(self) -> int:
        return int(self.P[0] * self.P[1] * self.P[2])

    def patch_index(self, s: int):
        P0, P1, _ = self.P
        return s % P0, (s // P0) % P1, s // (P0 * P1)

    def patch_n_el(self, s: int):
        a, b, c = self.patch_index(s)
        return int(self.n_el[0][a]), int(self.n_el[1][b]), int(self.n_el[2][c])

    def patch_degree(self, s: int):
        a, b, c = self.patch_index(s)
        return int(self.degree[0][a]), int(self.degree[1][b]), int(self.degree[2][c])

    def knot_vector(self, d: int, slab: int) -> np.ndarray:
        off = 0
        for t in range(slab):
            off += int(self.n_el[d][t]) + 2 * int(self.degree[d][t]) + 1
        m = int(self.n_el[d][slab]) + 2 * int(self.degree[d][slab]) + 1
        return self.knots[d][off:off + m]

    def ctrl_offsets(self) -> np.ndarray:
        offs = [0]
        for s in range(self.n_patches):
            ne, p = self.patch_n_el(s), self.patch_degree(s)
            offs.append(offs[-1] + 3 * (ne[0] + p[0]) * (ne[1] + p[1]) * (ne[2] + p[2]))
        return np.asarray(offs, dtype=np.int64)

    def patch_ctrl(self, s: int) -> np.ndarray:
        offs = self.ctrl_offsets()
        ne, p = self.patch_n_el(s), self.patch_degree(s)
        n = [ne[d] + p[d] for d in range(3)]
        return self.ctrl[offs[s]:offs[s + 1]].reshape(n[2], n[1], n[0], 3)

    def el_offsets(self) -> np.ndarray:
        offs = [0]
        for s in range(self.n_patches):
            ne = self.patch_n_el(s)
            offs.append(offs[-1] + ne[0] * ne[1] * ne[2])
        return np.asarray(offs, dtype=np.int64)

    def patch_sigma(self, s: int) -> np.ndarray:
        o = self.el_offsets()
        ne = self.patch_n_el(s)
        return self.sigma_el[o[s]:o[s + 1]].reshape(ne[2], ne[1], ne[0])

    def patch_nu(self, s: int) -> np.ndarray:
        o = self.el_offsets()
        ne = self.patch_n_el(s)
        return self.nu_el[o[s]:o[s + 1]].reshape(ne[2], ne[1], ne[0])


def _uniform_open_knots(n_el: int, p: int) -> np.ndarray:
    inner = np.arange(1, n_el, dtype=np.float64) / n_el
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def _greville(t: np.ndarray, p: int) -> np.ndarray:
    """Knot averages (t_{i+1} + ... + t_{i+p}) / p: the control net of the identity map."""
    n = len(t) - p - 1
    return np.array([t[i + 1:i + p + 1].mean() for i in range(n)])


def _slab_bounds(P: int) -> np.ndarray:
    return np.arange(P + 1, dtype=np.float64) / P


def default_coil(J0: float = 1.0) -> dict:
    return dict(J0=float(J0), r_in=0.3, r_out=0.45, xc=0.5, yc=0.5, zc=0.5, hz=0.2)


def build_problem(name, P, n_el, degree, *, sigma_fn, nu_fn, dt, n_steps, cg_tol=1e-10,
                  perturb=0.0, coil=None, seed=0, reluctivity=None) -> Problem:
    """Lay out a problem.

    ``sigma_fn(s, centers)`` / ``nu_fn(s, centers)`` give per-element values from the
    element centres of the undeformed lattice (array ``(e2, e1, e0, 3)``).
    ``perturb``: interior control points are displaced by U(-perturb, perturb) times
    the element size, per coordinate (patch faces stay planar and matching).
    """
    rng = np.random.default_rng(seed)
    P = tuple(int(x) for x in P)
    n_el = [np.asarray(n_el[d], dtype=np.int32) for d in range(3)]
    degree = [np.asarray(degree[d], dtype=np.int32) for d in range(3)]
    knots = [np.concatenate([_uniform_open_knots(int(n_el[d][a]), int(degree[d][a]))
                             for a in range(P[d])]) for d in range(3)]
    bounds = [_slab_bounds(P[d]) for d in range(3)]
    ctrl, sig, nu = [], [], []
    for c in range(P[2]):
        for b in range(P[1]):
            for a in range(P[0]):
                s = a + P[0] * (b + P[1] * c)
                idx = (a, b, c)
                ne = [int(n_el[d][idx[d]]) for d in range(3)]
                pp = [int(degree[d][idx[d]]) for d in range(3)]
                lo = [bounds[d][idx[d]] for d in range(3)]
                hi = [bounds[d][idx[d] + 1] for d in range(3)]
                n = [ne[d] + pp[d] for d in range(3)]
                kv = [_uniform_open_knots(ne[d], pp[d]) for d in range(3)]
                axes = [lo[d] + (hi[d] - lo[d]) * _greville(kv[d], pp[d]) for d in range(3)]
                Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
                net = np.stack([X, Y, Z], axis=-1)
                if perturb > 0.0:
                    spacing = np.array([(hi[d] - lo[d]) / ne[d] for d in range(3)])
                    inner = (slice(1, n[2] - 1), slice(1, n[1] - 1), slice(1, n[0] - 1))
                    shape = net[inner].shape
                    net[inner] += rng.uniform(-perturb, perturb, size=shape) * spacing
                ctrl.append(net.reshape(-1))
                ec = [lo[d] + (np.arange(ne[d]) + 0.5) * (hi[d] - lo[d]) / ne[d] for d in range(3)]
                EZ, EY, EX = np.meshgrid(ec[2], ec[1], ec[0], indexing="ij")
                centers = np.stack([EX, EY, EZ], axis=-1)
                sig.append(np.broadcast_to(np.asarray(sigma_fn(s, centers), dtype=np.float64),
                                           centers.shape[:3]).reshape(-1))
                nu.append(np.broadcast_to(np.asarray(nu_fn(s, centers), dtype=np.float64),
                                          centers.shape[:3]).reshape(-1))
    return Problem(name=name, P=P, n_el=n_el, degree=degree, knots=knots,
                   ctrl=np.concatenate(ctrl), sigma_el=np.concatenate(sig),
                   nu_el=np.concatenate(nu), dt=float(dt), n_steps=int(n_steps),
                   cg_tol=float(cg_tol), coil=coil or default_coil(), seed=seed,
                   reluctivity=reluctivity)


def _inside_box(centers, lo, hi):
    return np.all((centers > lo) & (centers < hi), axis=-1)


def _patch_center_inside(P, s, lo, hi):
    a, b, c = s % P[0], (s // P[0]) % P[1], s // (P[0] * P[1])
    ctr = np.array([(a + 0.5) / P[0], (b + 0.5) / P[1], (c + 0.5) / P[2]])
    return bool(np.all((ctr > lo) & (ctr < hi))), ctr


def config1(seed=0) -> Problem:
    """8 identity-mapped p=1 patches of 4^3 elements, conductor [0.25,0.75]^3 (sigma=1)."""
    P = (2, 2, 2)
    return build_problem(
        "c1_8x4^3_p1", P, [[4] * 2] * 3, [[1] * 2] * 3,
        sigma_fn=lambda s, C: np.where(_inside_box(C, 0.25, 0.75), 1.0, 0.0),
        nu_fn=lambda s, C: 1.0, dt=0.01, n_steps=10, perturb=0.0,
        coil=default_coil(1.0), seed=seed)


def config2(seed=0, n_steps=50) -> Problem:
    """64 curved p=2 patches of 8^3 elements; inner cube conducts with sigma=1e2, J0=1e2."""
    P = (4, 4, 4)

    def sig(s, C):
        inside, _ = _patch_center_inside(P, s, 0.25, 0.75)
        return 1e2 if inside else 0.0
    return build_problem(
        "c2_64x8^3_p2", P, [[8] * 4] * 3, [[2] * 4] * 3, sigma_fn=sig, nu_fn=lambda s, C: 1.0,
        dt=1e-3, n_steps=n_steps, perturb=0.05, coil=default_coil(1e2), seed=seed)


def config3(seed=0, n_steps=100, patches_per_dir=8, n_el=6) -> Problem:
    """512 p=2 patches of 6^3 elements; log-uniform sigma in a ball of radius 0.35.
    (patches_per_dir, n_el) give smaller members of the same family."""
    k = int(patches_per_dir)
    P = (k, k, k)
    rng = np.random.default_rng(seed + 1000)
    n = P[0] * P[1] * P[2]
    logs = rng.uniform(0.0, 4.0, size=n)
    nus = rng.uniform(0.5, 2.0, size=n)

    def sig(s, C):
        _, ctr = _patch_center_inside(P, s, 0.0, 1.0)
        return 10.0 ** logs[s] if np.linalg.norm(ctr - 0.5) < 0.35 else 0.0
    return build_problem(
        f"c3_{n}x{n_el}^3_p2", P, [[n_el] * k] * 3, [[2] * k] * 3, sigma_fn=sig,
        nu_fn=lambda s, C: nus[s], dt=1e-3, n_steps=n_steps, perturb=0.05,
        coil=default_coil(1.0), seed=seed)


def config4(seed=0, n_steps=100, patches_per_dir=7, el_range=(4, 12)) -> Problem:
    """343 patches, per-slab elements in {4..12} and per-slab degrees in {2,3}.
    (patches_per_dir, el_range) give smaller members of the same family."""
    k = int(patches_per_dir)
    P = (k, k, k)
    rng = np.random.default_rng(seed + 2000)
    n_el = [rng.integers(el_range[0], el_range[1] + 1, size=k) for _ in range(3)]
    deg = [rng.integers(2, 4, size=k) for _ in range(3)]
    cond = rng.uniform(size=k ** 3) < 0.5
    return build_problem(
        f"c4_{k ** 3}_uneven", P, n_el, deg, sigma_fn=lambda s, C: 1e3 if cond[s] else 0.0,
        nu_fn=lambda s, C: 1.0, dt=1e-3, n_steps=n_steps, perturb=0.05,
        coil=default_coil(1.0), seed=seed)


# nonlinear law of the scalability sweep: nu(|B|) = nu0 (k1 exp(k2 |B|^2) + k3)
C5_RELUCTIVITY = dict(nu0=1.0, k1=0.5, k2=2.0, k3=0.5)
# Coil amplitude of the nonlinear sweep.  With the config-2 amplitude (1e2) the field
# in the conductor approaches |B| ~ 15, where exp(2 |B|^2) overflows; an amplitude of
# 5 keeps |B| = O(1), the range in which the law above is a reluctivity curve.
C5_J0 = 5.0


def config5(patches_per_dir=4, seed=0, n_steps=200, nonlinear=True) -> Problem:
    """k^3 p=3 patches of 8^3 elements, config-2 material layout, nonlinear
    reluctivity in the conductor."""
    k = int(patches_per_dir)
    P = (k, k, k)

    def sig(s, C):
        inside, _ = _patch_center_inside(P, s, 0.25, 0.75)
        return 1e2 if inside else 0.0
    return build_problem(
        f"c5_{k}^3x8^3_p3", P, [[8] * k] * 3, [[3] * k] * 3, sigma_fn=sig,
        nu_fn=lambda s, C: 1.0, dt=5e-4, n_steps=n_steps, perturb=0.05,
        coil=default_coil(C5_J0), seed=seed, reluctivity=dict(C5_RELUCTIVITY) if nonlinear else None)


def small_problem(P=(2, 2, 1), n_el=((2, 3), (3, 2), (2,)), degree=((1, 2), (2, 1), (2,)),
                  conductor=((0.0, 0.5), (0.0, 1.0), (0.0, 1.0)), sigma=1.0, nu=1.0,
                  dt=0.05, n_steps=3, perturb=0.05, J0=1.0, seed=0, elementwise=False,
                  name="small", reluctivity=None) -> Problem:
    """Tiny uneven problems for brute-force pins and ragged-tile parity cases.

    ``conductor`` is an axis-aligned box; patches whose centre lies inside conduct
    (or elements, with ``elementwise=True``).
    """
    lo = np.array([c[0] for c in conductor])
    hi = np.array([c[1] for c in conductor])

    def sig(s, C):
        if elementwise:
            return np.where(_inside_box(C, lo, hi), sigma, 0.0)
        inside, _ = _patch_center_inside(P, s, lo, hi)
        return sigma if inside else 0.0
    return build_problem(name, P, [list(x) for x in n_el], [list(x) for x in degree],
                         sigma_fn=sig, nu_fn=lambda s, C: nu, dt=dt, n_steps=n_steps,
                         perturb=perturb, coil=default_coil(J0), seed=seed, reluctivity=reluctivity)


def sub_problem(prob: Problem, lo, hi, name=None) -> Problem:
    """The patches [lo_d, hi_d) of a problem's patch grid as a problem of its own (same
    slabs, knot vectors, control nets, materials, coil and time step; its outer faces
    become the Dirichlet boundary).  Bookkeeping only: used to take a bounded sample
    of a workload's per-patch work."""
    lo = [int(x) for x in lo]
    hi = [int(x) for x in hi]
    P = tuple(hi[d] - lo[d] for d in range(3))
    n_el = [np.asarray(prob.n_el[d][lo[d]:hi[d]], dtype=np.int32) for d in range(3)]
    degree = [np.asarray(prob.degree[d][lo[d]:hi[d]], dtype=np.int32) for d in range(3)]
    knots = [np.concatenate([prob.knot_vector(d, a) for a in range(lo[d], hi[d])]) for d in range(3)]
    c_off, e_off = prob.ctrl_offsets(), prob.el_offsets()
    ctrl, sig, nu = [], [], []
    for c in range(lo[2], hi[2]):
        for b in range(lo[1], hi[1]):
            for a in range(lo[0], hi[0]):
                s = a + prob.P[0] * (b + prob.P[1] * c)
                ctrl.append(prob.ctrl[c_off[s]:c_off[s + 1]])
                sig.append(prob.sigma_el[e_off[s]:e_off[s + 1]])
                nu.append(prob.nu_el[e_off[s]:e_off[s + 1]])
    return Problem(name=name or f"{prob.name}_sub", P=P, n_el=n_el, degree=degree, knots=knots,
                   ctrl=np.concatenate(ctrl), sigma_el=np.concatenate(sig), nu_el=np.concatenate(nu),
                   dt=prob.dt, n_steps=prob.n_steps, cg_tol=prob.cg_tol, coil=dict(prob.coil), seed=prob.seed,
                   reluctivity=prob.reluctivity)


CONFIGS = {
    "c1": config1,
    "c2": config2,
    "c3": config3,
    "c4": config4,
    "c5": config5,
}


def make_problem(name: str, **kw) -> Problem:
    return CONFIGS[name](**kw)
