"""The paper's convergence experiment (Sec. 4) on the GPU path, at reduced size.

Setup of Sec. 4: unit cube split at x = 0.5 into two subdomains (patches), the left
one conducting (sigma = 1), nu = 1, spline degree p per direction, n^3 elements per
subdomain, n_t implicit-Euler steps on t in (0, 1], the unscaled Dirichlet
preconditioner and PCG tolerance 1e-6 (caption of Fig. 2).  The manufactured field is
A = (1 - e^{-t}) A*, A* = (sin pi y sin pi z, sin pi z sin pi x, sin pi x sin pi y):
zero tangential trace and zero initial state, so no lifting is needed (the field of
Eq. (13) has inhomogeneous data); J = nu curl curl A + sigma dA/dt
= 2 pi^2 (1 - e^{-t}) A* + sigma e^{-t} A*, sampled at the library's quadrature points
(ieti_quad_points / ieti_load_vector_points).  Errors as in Sec. 4: eps_B of
B = curl A on the domain and eps_E of E = -dA/dt on the conductor (relative L2, at
t = 1), measured by the oracle's quadrature on the GPU states.
"""
import numpy as np
import pytest

from oracle.manufactured import A_star, curl_A_star, FieldEval, PI
from oracle.ietidp import PRECOND_DIRICHLET
from oracle.stepping import OracleProblem
from workloads import small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ieti():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti as mod
    return mod


def two_subdomains(n, p, n_t):
    return small_problem(P=(2, 1, 1), n_el=((n, n), (n,), (n,)), degree=((p, p), (p,), (p,)),
                         conductor=((0.0, 0.5), (0.0, 1.0), (0.0, 1.0)), sigma=1.0, nu=1.0,
                         dt=1.0 / n_t, n_steps=n_t, perturb=0.0, J0=0.0, name="paper_two_subdomains")


def source(S, n_t):
    """j(t_l) = 2 pi^2 (1 - e^{-t_l}) <A*, w> + e^{-t_l} <sigma A*, w> (library quadrature)."""
    xyz = S.quad_points()
    Aq = A_star(xyz)
    jA = S.load_vector_points(Aq)
    jS = S.load_vector_points(Aq * (xyz[:, :1] < 0.5))
    dt = 1.0 / n_t
    return lambda l: 2 * PI ** 2 * (1 - np.exp(-l * dt)) * jA + np.exp(-l * dt) * jS


def gpu_run(ieti, prob, n_t, **kw):
    S = ieti.Solver.from_problem(prob, device=0, precond="dirichlet", **kw)
    j = source(S, n_t)
    out, its = [], []
    for l in range(1, n_t + 1):
        st = S.step(j(l))
        its.append(st["cg_its"])
        out.append(S.solution().copy())
    S.close()
    return out, its


def errors(prob, op, a_end, a_prev, n_t):
    fe = FieldEval(prob, op.asm)
    f = 1 - np.exp(-1.0)
    _, eB = fe.errors(a_end, lambda x: f * A_star(x), lambda x: f * curl_A_star(x))
    eE, _ = fe.errors(-(a_end - a_prev) * n_t, lambda x: -np.exp(-1.0) * A_star(x), lambda x: 0 * x)
    return eB, eE


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_paper_case_steps_match_oracle(ieti, mode):
    """Every step of the two-subdomain run equals the oracle's monolithic solve."""
    n, p, n_t = 2, 3, 8
    prob = two_subdomains(n, p, n_t)
    op = OracleProblem(prob)
    fe = FieldEval(prob, op.asm)
    jA = fe.load(A_star)
    jS = fe.load(lambda x: A_star(x) * (x[..., :1] < 0.5))
    ref = op.run_monolithic(n_t, j_of_step=lambda l: 2 * PI ** 2 * (1 - np.exp(-l / n_t)) * jA + np.exp(-l / n_t) * jS)
    kw = (dict(precision="fp64", cg_tol=1e-12, max_sweeps=1) if mode == "fp64" else
          dict(precision="mixed", cg_tol=1e-6, outer_tol=1e-12, max_sweeps=20))
    got, _ = gpu_run(ieti, prob, n_t, **kw)
    tol = 1e-10 if mode == "fp64" else 1e-8
    for l, (a, b) in enumerate(zip(ref, got)):
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(a), (mode, l)


def test_paper_case_rates_and_iterations(ieti):
    """With the paper's solver settings (unscaled Dirichlet, PCG tol 1e-6): eps_B falls
    faster than h^2 from 2^3 to 4^3 elements per subdomain (p = 3, pre-asymptotic
    order ~2.4 here, the oracle's own value), eps_E falls like 1/n_t, the errors are
    the oracle's to the PCG tolerance, and the mean PCG iterations per step grow as h
    decreases (Sec. 4: linear growth in 1/h for this preconditioner)."""
    p = 3
    res = {}
    for n, n_t in ((2, 64), (4, 64), (4, 16)):
        prob = two_subdomains(n, p, n_t)
        op = OracleProblem(prob)
        got, its = gpu_run(ieti, prob, n_t, precision="fp64", cg_tol=1e-6, max_sweeps=1)
        eB, eE = errors(prob, op, got[-1], got[-2], n_t)
        res[(n, n_t)] = (eB, eE, float(np.mean(its)))
        if n_t == 64 and n == 4:
            fe = FieldEval(prob, op.asm)
            jA = fe.load(A_star)
            jS = fe.load(lambda x: A_star(x) * (x[..., :1] < 0.5))
            ref = op.run_monolithic(n_t, j_of_step=lambda l: 2 * PI ** 2 * (1 - np.exp(-l / n_t)) * jA
                                    + np.exp(-l / n_t) * jS)
            rB, rE = errors(prob, op, ref[-1], ref[-2], n_t)
            assert abs(eB - rB) <= 1e-3 * rB and abs(eE - rE) <= 1e-3 * rE, (eB, rB, eE, rE)
    assert res[(2, 64)][0] / res[(4, 64)][0] > 4.0, res            # B: better than h^2
    assert res[(4, 16)][1] / res[(4, 64)][1] > 3.0, res            # E: first order in time
    assert res[(4, 64)][2] > res[(2, 64)][2], res                  # iterations grow with 1/h


# ----------------------------------------------------------------------------- Eq. (13)
def _eq13(n, p, n_t):
    """The paper's own field A = e^{-t} A13 with its inhomogeneous tangential boundary
    data lifted by the oracle (boundary L2 projection), its source
    J = (3 nu - sigma) A (curl curl A13 = 3 A13) and its initial state; the library
    solves for the homogeneous part with the lifting's terms in the load vector."""
    from oracle.lifting import A13, LiftedRun
    prob = two_subdomains(n, p, n_t)
    op = OracleProblem(prob, with_load=False)
    sig = lambda x: (x[..., 0] < 0.5).astype(float)
    run = LiftedRun(op, A13, lambda x: (3.0 - sig(x))[..., None] * A13(x), sig)
    return prob, op, run


def _gpu_eq13(ieti, prob, run, n_t, **kw):
    S = ieti.Solver.from_problem(prob, device=0, precond="dirichlet", **kw)
    S.set_state(run.a0)
    out, its = [], []
    for l in range(1, n_t + 1):
        st = S.step(run.j_step(l))
        its.append(st["cg_its"])
        out.append(S.solution().copy())
    S.close()
    return out, its


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_eq13_lifted_run_matches_oracle(ieti, mode):
    """Every step of the Eq. (13) run (inhomogeneous data, non-zero initial state)
    equals the oracle's monolithic solve of the same lifted system."""
    n, p, n_t = 2, 3, 8
    prob, op, run = _eq13(n, p, n_t)
    ref = run.run_monolithic(n_t)
    kw = (dict(precision="fp64", cg_tol=1e-12, max_sweeps=1) if mode == "fp64" else
          dict(precision="mixed", cg_tol=1e-6, outer_tol=1e-12, max_sweeps=20))
    got, _ = _gpu_eq13(ieti, prob, run, n_t, **kw)
    tol = 1e-10 if mode == "fp64" else 1e-8
    for l, (a, b) in enumerate(zip(ref, got)):
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(a), (mode, l)


def test_eq13_rates_on_the_gpu_path(ieti):
    """Sec. 4 with its own field: eps_B = O(h^p) (p = 2, 2^3 -> 4^3 elements per
    subdomain, order ~2), eps_E = O(1/n_t), from GPU states with the paper's solver
    settings (unscaled Dirichlet, PCG tol 1e-6), equal to the oracle's errors."""
    from oracle.lifting import A13, curl_A13
    p = 2
    res = {}
    for n, n_t in ((2, 64), (4, 64), (4, 16)):
        prob, op, run = _eq13(n, p, n_t)
        got, its = _gpu_eq13(ieti, prob, run, n_t, precision="fp64", cg_tol=1e-6, max_sweeps=1)
        fe = FieldEval(prob, op.asm)
        A1, A0 = run.total(got[-1], 1.0), run.total(got[-2], 1.0 - 1.0 / n_t)
        _, eB = fe.errors(A1, lambda x: np.exp(-1.0) * A13(x), lambda x: np.exp(-1.0) * curl_A13(x))
        eE, _ = fe.errors(-(A1 - A0) * n_t, lambda x: np.exp(-1.0) * A13(x), lambda x: 0 * x)
        res[(n, n_t)] = (eB, eE, float(np.mean(its)))
        if (n, n_t) == (4, 64):
            ref = run.run_monolithic(n_t)
            R1, R0 = run.total(ref[-1], 1.0), run.total(ref[-2], 1.0 - 1.0 / n_t)
            _, rB = fe.errors(R1, lambda x: np.exp(-1.0) * A13(x), lambda x: np.exp(-1.0) * curl_A13(x))
            rE, _ = fe.errors(-(R1 - R0) * n_t, lambda x: np.exp(-1.0) * A13(x), lambda x: 0 * x)
            assert abs(eB - rB) <= 1e-3 * rB and abs(eE - rE) <= 1e-3 * rE, (eB, rB, eE, rE)
    print(res)
    assert res[(2, 64)][0] / res[(4, 64)][0] > 3.0, res            # B: order ~p = 2 in h
    assert 3.0 < res[(4, 16)][1] / res[(4, 64)][1] < 5.5, res      # E: first order in time
