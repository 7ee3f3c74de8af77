"""Pins of the oracle's coil source (Sec. 2.2 load vector (j_i)_k = <J, w_k>).

The source enters through a potential T with J = curl T, and the oracle assembles
j_k = <T, curl w_k>.  The identity that pins the gauge (j . G phi = 0) holds for any
T, so these tests pin T and the load form themselves:

* the profile: central differences of the potential give the azimuthal current
  J0 e_phi in the shell r_in < r < r_out, |z - zc| < hz, and zero elsewhere, and T
  is continuous across both radii (no current sheet);
* integration by parts on a curved patch: for a smooth T that vanishes on the
  patch boundary, <T, curl w_k> equals <curl T, w_k> (curl T by finite differences)
  up to quadrature error;
* the coil itself: for the rotation field v = (-(y - yc), x - xc, 0), which lies in
  the discrete space of identity-mapped patches, sum_k v_k <T, curl w_k> and
  sum_k v_k <J_coil, w_k> (J_coil sampled pointwise) both converge under
  h-refinement to the closed form J0 * 2 pi * 2 hz * (r_out^3 - r_in^3) / 3.

Each pin is also run against a planted mistake in a copy of the oracle's
arithmetic (a wrong inner value of T_z, a spurious det DF factor) to show that it
catches it.
"""
import numpy as np
import pytest

from workloads.configs import build_problem, default_coil
from oracle.assembly import PatchEval, coil_potential


def _curl_fd(T, x, eps=1e-6):
    """curl T at points x (n, 3) by second-order central differences."""
    d = np.zeros((len(x), 3, 3))            # d[:, i, j] = dT_i / dx_j
    for j in range(3):
        e = np.zeros(3)
        e[j] = eps
        d[:, :, j] = (T(x + e) - T(x - e)) / (2 * eps)
    return np.stack([d[:, 2, 1] - d[:, 1, 2], d[:, 0, 2] - d[:, 2, 0], d[:, 1, 0] - d[:, 0, 1]], axis=1)


def _sample(coil, n, rng, region):
    """Points in cylindrical coordinates about the coil axis, kept 1e-3 away from the
    radii and planes where T has kinks or jumps."""
    r_in, r_out, hz = coil["r_in"], coil["r_out"], coil["hz"]
    lo, hi = {"shell": (r_in, r_out), "inside": (0.0, r_in), "outside": (r_out, 0.49)}[region]
    r = rng.uniform(lo + 1e-3, hi - 1e-3, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    z = coil["zc"] + rng.uniform(-hz + 1e-3, hz - 1e-3, n)
    return np.stack([coil["xc"] + r * np.cos(phi), coil["yc"] + r * np.sin(phi), z], axis=1), r, phi


def _profile_ok(T, coil):
    rng = np.random.default_rng(5)
    J0 = coil["J0"]
    x, r, phi = _sample(coil, 200, rng, "shell")
    e_phi = np.stack([-np.sin(phi), np.cos(phi), 0 * phi], axis=1)
    ok = np.abs(_curl_fd(T, x) - J0 * e_phi).max() < 1e-6 * J0
    for region in ("inside", "outside"):
        x, _, _ = _sample(coil, 100, rng, region)
        ok &= np.abs(_curl_fd(T, x)).max() < 1e-6 * J0
    # outside the coil's height: no current
    x, _, _ = _sample(coil, 100, rng, "shell")
    x[:, 2] = coil["zc"] + np.where(rng.uniform(size=100) < 0.5, -1, 1) * rng.uniform(coil["hz"] + 1e-3, 0.45, 100)
    ok &= np.abs(_curl_fd(T, x)).max() < 1e-6 * J0
    # continuity across r_in and r_out (a jump would be a current sheet there)
    for rad in (coil["r_in"], coil["r_out"]):
        for ang in np.linspace(0, 2 * np.pi, 7):
            u = np.array([np.cos(ang), np.sin(ang), 0.0])
            c = np.array([coil["xc"], coil["yc"], coil["zc"] + 0.05])
            a, b = T((c + (rad - 1e-7) * u)[None]), T((c + (rad + 1e-7) * u)[None])
            ok &= np.abs(a - b).max() < 1e-5 * J0
    return bool(ok)


def _planted_potential(coil):
    """Copy of the coil potential with a plausible mistake: J0 r_out inside r_in."""
    J0, r_in, r_out = coil["J0"], coil["r_in"], coil["r_out"]

    def T(x):
        r = np.sqrt((x[..., 0] - coil["xc"]) ** 2 + (x[..., 1] - coil["yc"]) ** 2)
        Tz = np.where(r <= r_in, J0 * r_out, np.where(r < r_out, J0 * (r_out - r), 0.0))
        Tz = np.where(np.abs(x[..., 2] - coil["zc"]) < coil["hz"], Tz, 0.0)
        out = np.zeros(x.shape)
        out[..., 2] = Tz
        return out
    return T


def test_coil_profile_is_the_azimuthal_current():
    coil = default_coil(3.0)
    assert _profile_ok(coil_potential(coil), coil)
    assert not _profile_ok(_planted_potential(coil), coil)


class _DetPlanted(PatchEval):
    """Copy of the oracle's potential load with a spurious det DF weight."""

    def load_from_potential(self, T):
        Tq = T(self.F)
        U = np.einsum("eqij,eqaj->eqai", self.DF, self.chat)
        je = np.einsum("eqi,eqai,eq->ea", Tq, U, self.w * self.det)
        out = np.zeros(self.n_dofs)
        np.add.at(out, self.loc.ravel(), je.ravel())
        return out


def _bubble_potential(lo, hi):
    """Smooth T vanishing on the box [lo, hi]: a cubic bubble times a fixed vector field."""
    def T(x):
        t = (x - lo) * (hi - x) / ((hi - lo) / 2) ** 2
        b = np.prod(t, axis=-1)
        return np.stack([b * (1 + x[..., 1]), -b * x[..., 2], b * (0.5 + x[..., 0] * x[..., 1])], axis=-1)
    return T


def _by_parts_gap(cls, prob, s):
    pe = cls(prob, s)
    P = np.asarray(prob.P, dtype=float)
    idx = np.asarray(prob.patch_index(s), dtype=float)
    lo, hi = idx / P, (idx + 1) / P
    T = _bubble_potential(lo, hi)
    jT = pe.load_from_potential(T)
    jC = pe.load_from_field(lambda x: _curl_fd(T, x.reshape(-1, 3), 1e-5).reshape(x.shape))
    return np.abs(jT - jC).max() / np.abs(jC).max()


@pytest.mark.parametrize("perturb,tol", [(0.0, 1e-9), (0.05, 2e-4)])
def test_potential_load_integrates_by_parts(perturb, tol):
    """<T, curl w_k> = <curl T, w_k> for T = 0 on the patch boundary (identity map:
    the integrands are polynomials the Gauss rule integrates exactly, up to the finite
    differences; curved map: up to quadrature error), on a patch with det DF != 1."""
    prob = build_problem("bp", (2, 2, 1), [[3, 3], [3, 3], [4]], [[2, 2], [2, 2], [2]],
                         sigma_fn=lambda s, C: 0.0, nu_fn=lambda s, C: 1.0, dt=1.0, n_steps=1,
                         perturb=perturb, seed=3)
    assert _by_parts_gap(PatchEval, prob, 3) < tol
    assert _by_parts_gap(_DetPlanted, prob, 3) > 0.5


def _coil_moments(cls, n_el, p, coil, T):
    """sum_s c_s . j_s for the rotation field v about the coil axis: c_s from the patch
    L2 projection of v (exact: v lies in each identity-mapped patch's space), j_s from
    the potential and from the pointwise current."""
    prob = build_problem("coil", (2, 2, 1), [[n_el] * 2, [n_el] * 2, [2 * n_el]], [[p] * 2, [p] * 2, [p]],
                         sigma_fn=lambda s, C: 1.0, nu_fn=lambda s, C: 1.0, dt=1.0, n_steps=1, perturb=0.0)
    from scipy.sparse.linalg import cg
    xc, yc = coil["xc"], coil["yc"]
    v = lambda x: np.stack([-(x[..., 1] - yc), x[..., 0] - xc, 0 * x[..., 0]], axis=-1)

    def J(x):
        r = np.sqrt((x[..., 0] - xc) ** 2 + (x[..., 1] - yc) ** 2)
        on = (r > coil["r_in"]) & (r < coil["r_out"]) & (np.abs(x[..., 2] - coil["zc"]) < coil["hz"])
        f = np.where(on, coil["J0"] / np.maximum(r, 1e-300), 0.0)
        return np.stack([-(x[..., 1] - yc) * f, (x[..., 0] - xc) * f, 0 * f], axis=-1)
    IT = IJ = 0.0
    for s in range(prob.n_patches):
        pe = cls(prob, s)
        M = pe.mass(np.ones(pe.E))
        b = pe.load_from_field(v)
        c, info = cg(M, b, rtol=1e-13, maxiter=2000, M=None)    # the edge mass matrix is well conditioned
        assert info == 0
        IT += c @ pe.load_from_potential(T)
        IJ += c @ pe.load_from_field(J)
    return IT, IJ


def test_coil_load_converges_to_the_closed_form():
    # the coil's planes z = zc +- hz on element faces (h = 1/8 .. 1/32): only the
    # cylinders r = r_in, r_out cut elements
    coil = dict(default_coil(2.0), hz=0.25)
    exact = coil["J0"] * 2 * np.pi * 2 * coil["hz"] * (coil["r_out"] ** 3 - coil["r_in"] ** 3) / 3
    errT, errJ = [], []
    for n in (4, 8, 16):
        IT, IJ = _coil_moments(PatchEval, n, 1, coil, coil_potential(coil))
        errT.append(abs(IT - exact) / exact)
        errJ.append(abs(IJ - exact) / exact)
    # both quadratures of the non-smooth integrands converge to the closed form (and
    # so to each other): measured 1.5e-3, 1.8e-4, 7.9e-5 (potential) and 4.0e-2,
    # 1.5e-2, 3.3e-3 (pointwise current)
    assert errT[-1] < 2e-4 and errJ[-1] < 1e-2, (errT, errJ)
    assert errT[2] < errT[0] / 8 and errJ[2] < errJ[0] / 4, (errT, errJ)
    # planted mistakes: a spurious det DF factor (det = 1/4 here), a wrong inner T_z
    IT, _ = _coil_moments(_DetPlanted, 4, 1, coil, coil_potential(coil))
    assert abs(IT - exact) / exact > 0.5
    IT, _ = _coil_moments(PatchEval, 4, 1, coil, _planted_potential(coil))
    assert abs(IT - exact) / exact > 0.5
