"""GPU parity of the C-ABI solver against the CPU oracle (same seeded inputs).

Tolerances (relative l2 of the global coefficient vector a, every step):
  FP64 path  <= 1e-10   (PCG tolerance 1e-12 on ||r||/||d||, one sweep)
  mixed path <= 1e-8    (FP32 local operators, PCG tolerance 1e-6 per sweep, FP64
                         defect correction of the assembled system to 1e-12)
The reference is the oracle's monolithic sparse direct solve of Eq. (11); the
dual-primal rewrite of Sec. 3 reaches the same a exactly up to rounding.
"""
import numpy as np
import pytest

from workloads import make_problem, small_problem
from oracle.stepping import OracleProblem

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-8}
OPTS = {"fp64": dict(precision="fp64", cg_tol=1e-12, max_sweeps=1),
        "mixed": dict(precision="mixed", cg_tol=1e-6, outer_tol=1e-12, max_sweeps=20)}


@pytest.fixture(scope="module")
def ieti():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti as mod
    return mod


CASES = {
    "c1": lambda: make_problem("c1"),
    "uneven_p123": lambda: small_problem(P=(3, 2, 2), n_el=((2, 3, 2), (2, 3), (3, 2)),
                                         degree=((1, 2, 1), (2, 1), (1, 2)),
                                         conductor=((0.3, 0.7), (0, 1), (0, 1))),
    "buried": lambda: small_problem(P=(3, 3, 3), n_el=((2, 2, 2),) * 3, degree=((1, 1, 1),) * 3,
                                    conductor=((0.4, 0.6),) * 3),
    "ragged_p23": lambda: small_problem(P=(4, 3, 2), n_el=((3, 2, 5, 2), (2, 4, 2), (3, 2)),
                                        degree=((2, 3, 2, 2), (3, 2, 2), (2, 3)),
                                        conductor=((0.2, 0.8), (0.3, 0.7), (0.0, 1.0)), sigma=50.0,
                                        dt=0.01),
    "all_insulating_but_one": lambda: small_problem(P=(3, 3, 2), n_el=((2, 3, 2), (3, 2, 2), (2, 2)),
                                                    degree=((2, 1, 2), (1, 2, 2), (2, 1)),
                                                    conductor=((0.34, 0.66), (0.34, 0.66), (0.0, 0.5))),
    # smaller members of the 512-patch family (per-patch log-uniform sigma up to 1e4 in a
    # ball, nu in [0.5, 2]) and of the 343-patch family (uneven slabs, p in {2, 3} per
    # slab, random conductors with sigma = 1e3), from the same generators
    # degenerate material layouts: no insulator (no tree, no primal unknowns: the dual
    # problem has no coarse space) and no conductor (W = dt K, the whole domain gauged,
    # the coarse space only the wirebasket cotree edges)
    "all_conducting": lambda: small_problem(P=(2, 2, 2), n_el=((2, 3), (3, 2), (2, 2)),
                                            degree=((1, 2), (2, 1), (2, 2)), conductor=((0.0, 1.0),) * 3,
                                            sigma=5.0, dt=0.05),
    "all_insulating": lambda: small_problem(P=(2, 2, 2), n_el=((2, 3), (3, 2), (2, 2)),
                                            degree=((1, 2), (2, 1), (2, 2)), conductor=((2.0, 3.0),) * 3,
                                            sigma=5.0, dt=0.05),
    "c3_family": lambda: make_problem("c3", patches_per_dir=3, n_el=2),
    "c4_family": lambda: make_problem("c4", patches_per_dir=3, el_range=(2, 3)),
}

_ORACLE = {}


def oracle_run(name, steps):
    key = (name, steps)
    if key not in _ORACLE:
        prob = CASES[name]()
        op = OracleProblem(prob)
        _ORACLE[key] = (prob, op, op.run_monolithic(steps))
    return _ORACLE[key]


def gpu_run(ieti, prob, steps, j=None, **kw):
    S = ieti.Solver.from_problem(prob, device=0, **kw)
    if j is None:
        j = S.load_vector(prob.coil)
    out, stats = [], []
    for _ in range(steps):
        stats.append(S.step(j))
        out.append(S.solution().copy())
    S.close()
    return out, stats


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_steps_match_oracle(ieti, name, mode):
    steps = 4
    prob, op, ref = oracle_run(name, steps)
    got, stats = gpu_run(ieti, prob, steps, precond="dirichlet_stiff", **OPTS[mode])
    for l, (a, b) in enumerate(zip(ref, got)):
        err = np.linalg.norm(a - b) / np.linalg.norm(a)
        assert err <= TOL[mode], (name, mode, l, err, stats[l])
        assert np.all(b[op.gauge.cls == 0] == 0.0)     # eliminated DOFs are exactly zero


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("factor", ["fp32", "tf32x3", "bf16x3"])
def test_mixed_reduced_factors_match_oracle(ieti, name, factor):
    """Mixed path with the patch blocks factored in FP32 (SIMT, or tensor-core
    trailing updates as three TF32 products): the FP64 defect correction brings
    every step to the mixed tolerance against the oracle."""
    steps = 3
    prob, op, ref = oracle_run(name, steps)
    got, stats = gpu_run(ieti, prob, steps, precond="dirichlet_stiff", factor=factor, **OPTS["mixed"])
    for l, (a, b) in enumerate(zip(ref, got)):
        err = np.linalg.norm(a - b) / np.linalg.norm(a)
        assert err <= TOL["mixed"], (name, factor, l, err, stats[l])
        assert np.all(b[op.gauge.cls == 0] == 0.0)


@pytest.mark.parametrize("factor", ["tf32", "bf16"])
def test_single_product_ablation_factor_reaches_tolerance_or_reports(ieti, factor):
    """One-product tensor-core factors (TF32: 11-bit operands, BF16: 8-bit): the
    refinement either still reaches the mixed tolerance (in more sweeps) or reports
    non-convergence; it never returns a wrong state as converged."""
    prob, op, ref = oracle_run("c1", 2)
    S = ieti.Solver.from_problem(prob, device=0, precond="dirichlet_stiff", factor=factor, **OPTS["mixed"])
    j = S.load_vector(prob.coil)
    for l in range(2):
        st = S.step(j, raise_on_error=False)
        if st["rc"] == -4:
            break
        assert st["rc"] == 0
        a = S.solution()
        assert np.linalg.norm(a - ref[l]) <= TOL["mixed"] * np.linalg.norm(ref[l]), st
    S.close()


def test_factor_option_validation(ieti):
    prob = CASES["c1"]()
    with pytest.raises(ieti.IetiError) as e:
        ieti.Solver.from_problem(prob, device=0, precision="fp64", factor="tf32x3")
    assert e.value.code == -1


@pytest.mark.parametrize("precond", ["none", "dirichlet", "dirichlet_mult", "dirichlet_stiff"])
def test_preconditioners_same_solution(ieti, precond):
    prob, op, ref = oracle_run("uneven_p123", 2)
    got, stats = gpu_run(ieti, prob, 2, precond=precond, **OPTS["fp64"])
    for a, b in zip(ref, got):
        assert np.linalg.norm(a - b) <= TOL["fp64"] * np.linalg.norm(a)


def test_iteration_counts_match_oracle_pcg(ieti):
    """Same algorithm, same operators: the GPU PCG takes the oracle's iteration count
    (within one iteration, rounding) for the unscaled and scaled Dirichlet variants."""
    from oracle.ietidp import PRECOND_DIRICHLET, PRECOND_STIFF
    prob, op, ref = oracle_run("c1", 1)
    for name, pc in (("dirichlet", PRECOND_DIRICHLET), ("dirichlet_stiff", PRECOND_STIFF)):
        _, its = op.run_ietidp(1, tol=1e-8, precond=pc)
        _, stats = gpu_run(ieti, prob, 1, precond=name, precision="fp64", cg_tol=1e-8, max_sweeps=1)
        assert abs(stats[0]["cg_its"] - its[0]) <= 1, (name, stats[0]["cg_its"], its[0])


def test_device_and_host_inputs_agree(ieti):
    import torch
    prob = CASES["c1"]()
    S = ieti.Solver.from_problem(prob, device=0, **OPTS["fp64"])
    j = S.load_vector(prob.coil)
    S.step(j)
    a_host = S.solution().copy()
    S.close()
    S = ieti.Solver.from_problem(prob, device=0, **OPTS["fp64"])
    S.step(torch.from_numpy(j).cuda())
    out = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    S.solution(out)
    assert np.array_equal(out.cpu().numpy(), a_host)          # same kernels, same order
    S.close()


def test_checkpoint_resume(ieti):
    prob = CASES["ragged_p23"]()
    S = ieti.Solver.from_problem(prob, device=0, **OPTS["fp64"])
    j = S.load_vector(prob.coil)
    for _ in range(2):
        S.step(j)
    mid = S.solution().copy()
    S.step(j)
    end = S.solution().copy()
    S.close()
    R = ieti.Solver.from_problem(prob, device=0, **OPTS["fp64"])
    R.set_state(mid)
    R.step(j)
    assert np.array_equal(R.solution(), end)
    R.close()


def test_cg_not_converged_is_reported(ieti):
    prob = CASES["c1"]()
    S = ieti.Solver.from_problem(prob, device=0, precision="fp64", cg_tol=1e-12, cg_max_it=2, max_sweeps=1)
    j = S.load_vector(prob.coil)
    st = S.step(j, raise_on_error=False)
    assert st["rc"] == -4 and st["cg_its"] == 2
    S.close()


def test_zero_load_gives_zero_state(ieti):
    prob = CASES["c1"]()
    S = ieti.Solver.from_problem(prob, device=0, **OPTS["fp64"])
    st = S.step(np.zeros(S.n))
    assert st["cg_its"] == 0 and not np.any(S.solution())
    S.close()


@pytest.fixture(scope="module")
def c2_oracle():
    prob = make_problem("c2")
    op = OracleProblem(prob)
    return prob, op


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_tf32x3"])
def test_c2_full_size_residual(ieti, c2_oracle, mode):
    """Bench configuration (64 curved p=2 patches of 8^3 elements), launched as the
    bench launches it: each GPU step solves the oracle's assembled gauged system
    W_g a = M_g a^l + dt j to a small FP64 residual (a property that holds at any
    size), and the FP64 and mixed paths agree to the mixed tolerance."""
    prob, op = c2_oracle
    opts = dict(precision=mode.split("_")[0], cg_tol=1e-10 if mode == "fp64" else 1e-6, outer_tol=1e-11,
                max_sweeps=20)
    if mode == "mixed_tf32x3":
        opts["factor"] = "tf32x3"
    got, stats = gpu_run(ieti, prob, 2, precond="dirichlet_stiff", **opts)
    prev = np.zeros(op.asm.lat.n_edges)
    for l, a in enumerate(got):
        res = op.mono.residual(a, prev, op.asm.j_global)
        assert res <= 2e-11, (mode, l, res, stats[l])
        prev = a
    if mode != "fp64":
        ref, _ = gpu_run(ieti, prob, 2, precond="dirichlet_stiff", precision="fp64", cg_tol=1e-12,
                         outer_tol=1e-13, max_sweeps=5)
        for a, b in zip(ref, got):
            assert np.linalg.norm(a - b) <= TOL["mixed"] * np.linalg.norm(a)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_pcg_modes_agree(ieti, mode):
    """The persistent cooperative PCG kernel and the launch-per-phase loop run the
    same algorithm: same iteration count, same solution within the mode tolerance."""
    prob, op, ref = oracle_run("ragged_p23", 2)
    a, sa = gpu_run(ieti, prob, 2, precond="dirichlet_stiff", pcg_mode=0, **OPTS[mode])
    b, sb = gpu_run(ieti, prob, 2, precond="dirichlet_stiff", pcg_mode=1, **OPTS[mode])
    for x, y, s1, s2 in zip(a, b, sa, sb):
        assert abs(s1["cg_its"] - s2["cg_its"]) <= 1
        assert np.linalg.norm(x - y) <= TOL[mode] * np.linalg.norm(x)


@pytest.mark.parametrize("name", ["c1", "ragged_p23"])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("predictor", [1, 2])
def test_predictor_steps_match_oracle(ieti, name, mode, predictor):
    """Sweeps started from the iterate extrapolated in time (linear or quadratic): same
    right-hand side and stopping test, so every step still matches the oracle's solve."""
    steps = 4
    prob, op, ref = oracle_run(name, steps)
    got, stats = gpu_run(ieti, prob, steps, precond="dirichlet_stiff", predictor=predictor, **OPTS[mode])
    for l, (a, b) in enumerate(zip(ref, got)):
        err = np.linalg.norm(a - b) / np.linalg.norm(a)
        assert err <= TOL[mode], (name, mode, l, err, stats[l])
        assert np.all(b[op.gauge.cls == 0] == 0.0)


def test_predictor_history_reset_by_set_state(ieti):
    """A resumed context has no a^{l-1}: its first step starts from a^l and still
    reaches the state of the uninterrupted run within the tolerance."""
    prob = CASES["ragged_p23"]()
    S = ieti.Solver.from_problem(prob, device=0, predictor=2, **OPTS["fp64"])
    j = S.load_vector(prob.coil)
    for _ in range(3):
        S.step(j)
    mid = S.solution().copy()
    S.step(j)
    end = S.solution().copy()
    S.close()
    R = ieti.Solver.from_problem(prob, device=0, predictor=2, **OPTS["fp64"])
    R.set_state(mid)
    R.step(j)
    assert np.linalg.norm(R.solution() - end) <= TOL["fp64"] * np.linalg.norm(end)
    R.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_c2_bench_options_match_oracle_monolithic(ieti, c2_oracle, mode):
    """The 64-patch workload with the bench's exact options (stiffness-scaled Dirichlet,
    quadratic time predictor, autotuned schedule, L2 hints, sweep loop as a CUDA graph,
    TF32x3 tensor-core factors in the mixed path, assembled residual to 1e-12), element
    by element against the oracle's monolithic sparse direct solve of Eq. (11) over three
    steps from a^0 = 0.  (With the residual stopped at 1e-11 the mixed state was 3.7e-8
    from the oracle's: the step system amplifies the residual about 4000-fold.)"""
    prob, op = c2_oracle
    steps = 3
    ref = op.run_monolithic(steps)
    opts = {"fp64": dict(precision="fp64", cg_tol=1e-11),
            "mixed": dict(precision="mixed", cg_tol=1e-6, factor="tf32x3")}[mode]
    got, stats = gpu_run(ieti, prob, steps, precond="dirichlet_stiff", outer_tol=1e-12, max_sweeps=30, predictor=2,
                         autotune=1, l2_persist=2, graph=1, **opts)
    for l, (a, b) in enumerate(zip(ref, got)):
        err = np.linalg.norm(a - b) / np.linalg.norm(a)
        assert err <= TOL[mode], (mode, l, err, stats[l])


@pytest.mark.parametrize("name", ["c3_family", "c4_family"])
def test_autotuned_schedule_matches_oracle(ieti, name):
    """The autotuned schedule of the persistent kernel (CTAs, ring stages and stage
    bytes timed at setup) against the oracle, not only against the rule's schedule."""
    prob, op, ref = oracle_run(name, 3)
    for mode in ("fp64", "mixed"):
        got, stats = gpu_run(ieti, prob, 3, precond="dirichlet_stiff", autotune=1, **OPTS[mode])
        for l, (a, b) in enumerate(zip(ref, got)):
            assert np.linalg.norm(a - b) <= TOL[mode] * np.linalg.norm(a), (name, mode, l, stats[l])
