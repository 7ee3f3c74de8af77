"""The sweep loop of a step as one CUDA graph (while node; the stop decisions taken by
a device kernel from the assembled residual norm and the PCG status) against the
host loop, through the C ABI.  Both run the same kernels in the same order on the
same data, so states, PCG iterations and sweep counts must be identical."""
import numpy as np
import pytest

from workloads import make_problem, small_problem

pytestmark = pytest.mark.gpu

OPTS = {"fp64": dict(precision="fp64", cg_tol=1e-12, max_sweeps=1),
        "mixed": dict(precision="mixed", cg_tol=1e-6, outer_tol=1e-12, max_sweeps=20, factor="tf32x3")}


@pytest.fixture(scope="module")
def ieti():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti as mod
    return mod


def _ragged():
    return small_problem(P=(4, 3, 2), n_el=((3, 2, 5, 2), (2, 4, 2), (3, 2)),
                         degree=((2, 3, 2, 2), (3, 2, 2), (2, 3)), perturb=0.05, name="ragged_p23")


def _run(ieti, prob, steps, **kw):
    S = ieti.Solver.from_problem(prob, device=0, precond="dirichlet_stiff", **kw)
    j = S.load_vector(prob.coil)
    out, stats = [], []
    for _ in range(steps):
        stats.append(S.step(j, raise_on_error=False))
        out.append(S.solution().copy())
    info = S.info()
    S.close()
    return out, stats, info


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["c1", "ragged"])
@pytest.mark.parametrize("predictor", [0, 2])
def test_graph_loop_equals_host_loop(ieti, mode, case, predictor):
    prob = make_problem("c1") if case == "c1" else _ragged()
    a, sa, ia = _run(ieti, prob, 4, graph=0, predictor=predictor, **OPTS[mode])
    b, sb, ib = _run(ieti, prob, 4, graph=1, predictor=predictor, **OPTS[mode])
    assert ia["step_graph"] == 0 and ib["step_graph"] == 1
    for x, y, s1, s2 in zip(a, b, sa, sb):
        assert s1["rc"] == 0 and s2["rc"] == 0
        assert (s1["cg_its"], s1["sweeps"]) == (s2["cg_its"], s2["sweeps"])
        assert s1["outer_res"] == s2["outer_res"]
        assert np.array_equal(x, y)


def test_graph_reports_like_host_loop(ieti):
    """Non-convergence reaches the caller the same way: PCG capped at 3 iterations in
    one sweep, and the refinement capped at 2 sweeps."""
    prob = make_problem("c1")
    for kw in (dict(precision="fp64", cg_tol=1e-12, cg_max_it=3, max_sweeps=1),
               dict(precision="mixed", cg_tol=1e-6, outer_tol=1e-14, max_sweeps=2)):
        a, sa, _ = _run(ieti, prob, 2, graph=0, **kw)
        b, sb, ib = _run(ieti, prob, 2, graph=1, **kw)
        assert ib["step_graph"] == 1
        for x, y, s1, s2 in zip(a, b, sa, sb):
            assert s1["rc"] == s2["rc"] == -4
            assert (s1["cg_its"], s1["sweeps"]) == (s2["cg_its"], s2["sweeps"])
            assert np.array_equal(x, y)


def test_graph_mode_selection(ieti):
    """The graph serves linear problems with the persistent kernel and no per-launch
    profiling; the other configurations run the host loop."""
    prob = make_problem("c1")
    for kw, want in ((dict(), 1), (dict(graph=0), 0), (dict(profile=1), 0), (dict(pcg_mode=1), 0),
                     (dict(l2_persist=1), 0)):
        S = ieti.Solver.from_problem(prob, device=0, **OPTS["fp64"], **kw)
        inf = S.info()
        S.close()
        if kw.get("l2_persist") == 1 and inf["l2_window_bytes"] == 0:
            want = 1      # no access-policy window on this device: nothing blocks the graph
        assert inf["step_graph"] == want, kw


def test_profiled_steps_equal_unprofiled(ieti):
    """Per-launch CUDA-event profiling (host loop) changes no result and fills the
    kernel-class statistics."""
    prob = make_problem("c1")
    a, sa, _ = _run(ieti, prob, 2, **OPTS["mixed"])
    S = ieti.Solver.from_problem(prob, device=0, precond="dirichlet_stiff", profile=1, **OPTS["mixed"])
    j = S.load_vector(prob.coil)
    for x, s1 in zip(a, sa):
        st = S.step(j)
        assert (st["cg_its"], st["sweeps"]) == (s1["cg_its"], s1["sweeps"])
        assert np.array_equal(S.solution(), x)
    ks = S.kernel_stats()
    assert ks["pcg"]["launches"] == sum(s["sweeps"] for s in sa) and ks["pcg"]["total_ms"] > 0
    assert ks["spmv"]["launches"] > 0
    S.close()
