"""Pins of the oracle's dual-primal solve (Sec. 3) and time loop (Eq. (11))."""
import numpy as np
import pytest

from workloads import make_problem, small_problem
from oracle.ietidp import PRECOND_DIRICHLET, PRECOND_MULT, PRECOND_STIFF, PRECOND_NONE
from oracle.manufactured import A_star, curl_A_star, FieldEval, PI
from oracle.stepping import OracleProblem


def _cases():
    return [make_problem("c1"),
            small_problem(P=(3, 2, 2), n_el=((2, 3, 2), (2, 3), (3, 2)),
                          degree=((1, 2, 1), (2, 1), (1, 2)),
                          conductor=((0.3, 0.7), (0, 1), (0, 1)), name="uneven"),
            small_problem(P=(3, 3, 3), n_el=((2, 2, 2), (2, 2, 2), (2, 2, 2)),
                          degree=((1, 1, 1), (1, 1, 1), (1, 1, 1)),
                          conductor=((0.4, 0.6), (0.4, 0.6), (0.4, 0.6)), name="buried")]


@pytest.mark.parametrize("prob", _cases(), ids=lambda p: p.name)
@pytest.mark.parametrize("pc", [PRECOND_DIRICHLET, PRECOND_STIFF])
def test_dd_equals_monolithic(prob, pc):
    """The dual-primal system is an exact rewrite of Eq. (11): both give the same a."""
    op = OracleProblem(prob)
    ref = op.run_monolithic(3)
    got, its = op.run_ietidp(3, tol=1e-12, precond=pc)
    for a, b in zip(ref, got):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)
    assert max(its) < 200


def test_brute_force_dense_c1():
    """Config-1 gauged system: dense numpy solve equals the sparse direct solve."""
    op = OracleProblem(make_problem("c1"))
    W = op.mono.W.toarray()
    a = np.zeros(op.asm.lat.n_edges)
    for _ in range(3):
        f = op.mono.rhs(a, op.asm.j_global)
        x = np.linalg.solve(W, f)
        a_next = op.mono.step(a, op.asm.j_global)
        assert np.linalg.norm(a_next[op.mono.free] - x) <= 1e-12 * np.linalg.norm(x)
        a = a_next


@pytest.mark.parametrize("prob", _cases()[:2], ids=lambda p: p.name)
def test_preconditioner_algebra(prob):
    """Scaled B_D: B B_D^T B = B and P_D = B_D^T B is a projection, hence
    lambda_min(M^{-1} F) >= 1 on range(F) (FETI-DP theory, Farhat et al. 2001 and
    its analysis); unscaled Dirichlet (the paper's Sec. 4 variant) has no such bound
    but is still SPD on range(F)."""
    op = OracleProblem(prob)
    for pc in (PRECOND_MULT, PRECOND_STIFF):
        I = op.ietidp(pc)
        B = np.hstack([x.toarray() for x in op.dec.B])
        BD = np.hstack([x.toarray() for x in I.BD])
        assert np.abs(B @ BD.T @ B - B).max() < 1e-13
        PD = BD.T @ B
        assert np.abs(PD @ PD - PD).max() < 1e-13
        F, Mi = I.dense_F_and_M()
        ev = np.sort(np.linalg.eigvals(Mi @ F).real)
        ev = ev[ev > 1e-8 * ev.max()]
        assert ev[0] > 1 - 1e-8
    F, Mi = op.ietidp(PRECOND_DIRICHLET).dense_F_and_M()
    assert np.abs(F - F.T).max() < 1e-10 * np.abs(F).max()
    ev = np.linalg.eigvalsh(F)
    assert ev[0] > -1e-10 * ev[-1]


def test_time_rate_in_nt():
    """Sec. 4: eps_E = O(h^p + 1/n_t) for E_C = -dA/dt; on a fine enough mesh the
    1/n_t part dominates, so halving dt halves eps_E."""
    sigma = 50.0
    prob0 = small_problem(P=(2, 1, 1), n_el=((3, 3), (6,), (6,)), degree=((2, 2), (2,), (2,)),
                          conductor=((0, 0.5), (0, 1), (0, 1)), sigma=sigma, dt=1.0, perturb=0.0)
    sig = lambda x: np.where(x[..., 0] < 0.5, sigma, 0.0)[..., None]
    errs = []
    for nt in (4, 8, 16):
        prob0.dt = 1.0 / nt
        op = OracleProblem(prob0, with_load=False)
        fe = FieldEval(prob0, op.asm)
        jstar = fe.load(lambda x: (2 * PI ** 2 - sig(x)) * A_star(x))
        # a^0: discrete field of A(0) = A*, from (M + K) a = <sigma A* + curl curl A*, w>
        j0 = fe.load(lambda x: (2 * PI ** 2 + sig(x)) * A_star(x))
        prob0.dt = 1.0
        op0 = OracleProblem(prob0, with_load=False)
        a = op0.mono.step(np.zeros(op0.asm.lat.n_edges), j0)
        prob0.dt = 1.0 / nt
        eE = []
        for l in range(nt):
            t = (l + 1) / nt
            a_next = op.mono.step(a, np.exp(-t) * jstar)
            E_h = (a - a_next) / prob0.dt
            ee, _ = fe.errors(E_h, lambda x: np.exp(-t) * A_star(x), curl_A_star)
            eE.append(ee)
            a = a_next
        errs.append(max(eE))
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(0.75 < r < 1.25 for r in rates), (errs, rates)


def test_unscaled_iterations_grow_with_h():
    """Sec. 4 observes iteration counts growing as h decreases for the unscaled
    Dirichlet preconditioner.  The values of Fig. 2e are not in the text: logged,
    only monotone growth is checked."""
    its = []
    for ne in (2, 4):
        prob = small_problem(P=(2, 1, 1), n_el=((ne, ne), (ne,), (ne,)), degree=((1, 1), (1,), (1,)),
                             conductor=((0, 0.5), (0, 1), (0, 1)), sigma=1.0, dt=0.05, perturb=0.0)
        op = OracleProblem(prob)
        _, it = op.run_ietidp(2, tol=1e-6, precond=PRECOND_DIRICHLET)
        its.append(np.mean(it))
    print("mean PCG iterations (unscaled Dirichlet, tol 1e-6):", its)
    assert its[1] >= its[0]


def test_long_time_limit_is_the_magnetostatic_solve():
    """With a constant load the implicit-Euler iterates approach the gauged
    magnetostatic solution: the fixed point of W a^{l+1} = M a^l + dt j is K a = j on
    the free DOFs (Eq. (11) with a^{l+1} = a^l).  Every step contracts the defect
    K a^l - j by a fixed factor, so its norm falls geometrically; a wrong sign or a
    misplaced dt in the step breaks that."""
    prob = make_problem("c1")
    prob.dt = 5.0                                  # long steps: few of them reach the limit
    op = OracleProblem(prob)
    mono = op.mono
    K = (mono.W - mono.M) / prob.dt                # gauged stiffness on the free DOFs
    jf = op.asm.j_global[mono.free]
    defect = []
    for a in op.run_monolithic(12):
        defect.append(np.linalg.norm(K @ a[mono.free] - jf) / np.linalg.norm(jf))
    assert defect[-1] < 1e-8, defect
    # geometric decay down to the rounding floor of the sparse direct solves
    d = np.array(defect)
    above = d[:-1] > 1e-9
    ratios = d[1:][above] / d[:-1][above]
    assert above.sum() >= 3 and np.all(ratios < 0.5), (defect, ratios)
    # the limit field is gradient-free against the load: (K a, a) = (j, a) at the end
    a = op.run_monolithic(12)[-1][mono.free]
    assert abs(a @ (K @ a) - jf @ a) <= 1e-8 * abs(jf @ a)
