"""Pins of the oracle's Newton step for the nonlinear reluctivity (the extension the
paper names after Eq. (3), Sec. 2; law nu(|B|) = nu0 (k1 exp(k2 |B|^2) + k3)).

Each pin fixes the oracle against something other than itself: the energy whose
gradient the residual must be (finite differences of E), finite differences of the
residual for the tangent, the linear law (k1 = 0) against the linear monolithic
step, quadratic convergence, and the closed forms of the law."""
import numpy as np
import pytest

from oracle.nonlinear import NewtonProblem, Reluctivity
from oracle.stepping import OracleProblem
from workloads import make_problem, small_problem

LAW = dict(nu0=1.0, k1=0.5, k2=2.0, k3=0.5)


def _c1(J0=15.0, law=LAW):
    prob = make_problem("c1")
    prob.coil = dict(prob.coil, J0=J0)
    prob.reluctivity = dict(law)
    return prob


@pytest.fixture(scope="module")
def c1():
    return NewtonProblem(_c1())


def _state(npb, rng, scale=0.02):
    """A free-DOF state with |B| = O(1) in the conductor: the converged first step
    plus a random perturbation of comparable size per entry."""
    a, _ = npb.step(np.zeros(npb.asm.lat.n_edges), npb.asm.j_global)
    af = a[npb.free]
    return af + scale * np.abs(af).max() * rng.standard_normal(npb.n)


def test_law_closed_forms():
    m = Reluctivity(**LAW)
    assert m.nu(0.0) == pytest.approx(LAW["nu0"] * (LAW["k1"] + LAW["k3"]))
    s = np.linspace(0.0, 1.5, 7)
    h = 1e-6
    # nu' and Phi' = nu by central differences
    assert np.allclose((m.nu(s + h) - m.nu(s - h)) / (2 * h), m.dnu(s), rtol=1e-7)
    assert np.allclose((m.Phi(s + h) - m.Phi(s - h)) / (2 * h), m.nu(s), rtol=1e-7)
    assert m.Phi(0.0) == 0.0


def test_residual_is_energy_gradient(c1):
    rng = np.random.default_rng(0)
    a_prev = _state(c1, rng)
    a = _state(c1, rng)
    jf = c1.asm.j_global[c1.free]
    v = np.abs(a).max() * rng.standard_normal(c1.n)     # a direction on the state's scale
    g = c1.residual(a, a_prev, jf) @ v
    err = []
    for eps in (1e-4, 1e-5):   # central differences: the error falls like eps^2
        fd = (c1.energy(a + eps * v, a_prev, jf) - c1.energy(a - eps * v, a_prev, jf)) / (2 * eps)
        err.append(abs(fd - g) / abs(g))
    assert err[1] <= 1e-6 and err[1] <= 0.05 * err[0], err


def test_tangent_matches_residual_differences(c1):
    rng = np.random.default_rng(1)
    a = _state(c1, rng)
    a_prev = np.zeros(c1.n)
    jf = c1.asm.j_global[c1.free]
    v = np.abs(a).max() * rng.standard_normal(c1.n)
    Jv = c1.jacobian(a) @ v
    err = []
    for eps in (1e-4, 1e-5):
        fd = (c1.residual(a + eps * v, a_prev, jf) - c1.residual(a - eps * v, a_prev, jf)) / (2 * eps)
        err.append(np.linalg.norm(fd - Jv) / np.linalg.norm(Jv))
    assert err[1] <= 1e-6 and err[1] <= 0.05 * err[0], err
    J = c1.jacobian(a)
    assert abs(J - J.T).max() <= 1e-12 * abs(J).max()          # symmetric tangent


def test_linear_law_reduces_to_linear_step():
    """k1 = 0: nu = nu0 k3 in the conductor; Newton stops after one correction and
    equals the linear monolithic step with that per-element nu."""
    law = dict(nu0=1.0, k1=0.0, k2=2.0, k3=0.7)
    prob = _c1(law=law)
    npb = NewtonProblem(prob)
    a, hist = npb.step(np.zeros(npb.asm.lat.n_edges), npb.asm.j_global)
    assert len(hist) <= 2 and hist[-1] <= 1e-12
    lin = _c1()
    lin.reluctivity = None
    lin.nu_el = np.where(lin.sigma_el > 0, 0.7, lin.nu_el)
    ref = OracleProblem(lin).run_monolithic(1)[0]
    assert np.linalg.norm(a - ref) <= 1e-12 * np.linalg.norm(ref)


def test_newton_converges_quadratically(c1):
    a0 = np.zeros(c1.asm.lat.n_edges)
    a, hist = c1.step(a0, c1.asm.j_global, tol=1e-13)
    assert hist[-1] <= 1e-13
    h = np.array(hist)
    # once in the basin: e_{k+1} <= C e_k^2 with a modest C
    k = np.nonzero(h < 1e-2)[0]
    assert len(k) >= 2
    for i in k[:-1]:
        if h[i + 1] > 1e-14:
            assert h[i + 1] <= 50.0 * h[i] ** 2, hist
    # the converged state solves the nonlinear system
    R = c1.residual(a[c1.free], a0[c1.free], c1.asm.j_global[c1.free])
    f = c1.prob.dt * c1.asm.j_global[c1.free]
    assert np.linalg.norm(R) <= 1e-11 * np.linalg.norm(f)


def test_nonlinearity_is_active(c1):
    """The pinned case is really nonlinear: nu varies by more than 10% in the
    conductor at the converged first step."""
    a, _ = c1.step(np.zeros(c1.asm.lat.n_edges), c1.asm.j_global)
    s2 = np.concatenate([np.einsum("eqi,eqi->eq", B, B).ravel()
                         for B in (c1._B(a[c1.free], it) for it in c1.nl)])
    nu = c1.model.nu(s2)
    assert nu.max() / nu.min() > 1.1


def test_small_uneven_patches_newton():
    """Mixed degrees and a conductor crossing patches: same convergence."""
    prob = small_problem(P=(3, 2, 2), n_el=((2, 3, 2), (2, 3), (3, 2)), degree=((1, 2, 1), (2, 1), (1, 2)),
                         conductor=((0.3, 0.7), (0.2, 0.8), (0.2, 0.8)), elementwise=True, J0=10.0,
                         reluctivity=LAW)
    npb = NewtonProblem(prob)
    a, hist = npb.step(np.zeros(npb.asm.lat.n_edges), npb.asm.j_global)
    assert hist[-1] <= 1e-10 and len(hist) <= 8
