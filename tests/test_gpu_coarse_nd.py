"""GPU parity of the nested-dissection coarse solve (Sec. 3, the coarse Schur
complement S_c, factored along a nested dissection of the patch grid and solved by a
forward sweep by height and a backward sweep by depth inside the persistent kernel).

Same tolerances and oracle as tests/test_gpu_parity.py: relative l2 of the global
coefficient vector against the oracle's monolithic solve of Eq. (11), 1e-10 (FP64
path) and 1e-8 (mixed path), every step, for every parity case and two tree shapes
(leaf boxes of 1 and 8 patches).  The coarse solve is exact up to rounding, so the
states also equal those of the dense coarse inverse to 1e-12 (FP64 path)."""
import numpy as np
import pytest

from test_gpu_parity import CASES, OPTS, TOL, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ieti():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti as mod
    return mod


@pytest.mark.parametrize("leaf", [1, 8])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_nd_steps_match_oracle(ieti, name, mode, leaf):
    steps = 3
    prob, op, ref = oracle_run(name, steps)
    S = ieti.Solver.from_problem(prob, device=0, precond="dirichlet_stiff", coarse="nd", coarse_leaf=leaf,
                                 **OPTS[mode])
    inf = S.info()
    S.close()
    if inf["n_coarse"] == 0:
        pytest.skip("no coarse unknowns")
    assert inf["coarse_mode"] == 2 and inf["coarse_nodes"] > 0
    got, stats = gpu_run(ieti, prob, steps, precond="dirichlet_stiff", coarse="nd", coarse_leaf=leaf, **OPTS[mode])
    for l, (a, b) in enumerate(zip(ref, got)):
        err = np.linalg.norm(a - b) / np.linalg.norm(a)
        assert err <= TOL[mode], (name, mode, leaf, l, err, stats[l])
        assert np.all(b[op.gauge.cls == 0] == 0.0)


@pytest.mark.parametrize("name", ["c4_family", "ragged_p23", "c3_family"])
@pytest.mark.parametrize("graph", [0, 1])
def test_nd_equals_dense_coarse(ieti, name, graph):
    """Same PCG on the same operators: the two coarse solves agree to rounding, the
    iteration counts within one, in the host sweep loop and in the step graph."""
    prob, op, ref = oracle_run(name, 3)
    kw = dict(precond="dirichlet_stiff", graph=graph, **OPTS["fp64"])
    a_d, st_d = gpu_run(ieti, prob, 3, coarse="dense", **kw)
    a_n, st_n = gpu_run(ieti, prob, 3, coarse="nd", **kw)
    for x, y, s, t in zip(a_d, a_n, st_d, st_n):
        assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(x)
        assert abs(s["cg_its"] - t["cg_its"]) <= 1


@pytest.mark.parametrize("name", ["c4_family", "ragged_p23"])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_nd_top_merged_tree_matches_oracle(ieti, name, mode):
    """coarse_top = 2: the first bisection level's separators merged into one dense
    root block (fewer levels, a wider root): the same states within the path's
    tolerance."""
    prob, op, ref = oracle_run(name, 2)
    kw = dict(precond="dirichlet_stiff", coarse="nd", coarse_leaf=1, **OPTS[mode])
    S = ieti.Solver.from_problem(prob, device=0, coarse_top=2, **kw)
    merged = S.info()["coarse_nodes"]
    S.close()
    S = ieti.Solver.from_problem(prob, device=0, **kw)
    plain = S.info()["coarse_nodes"]
    S.close()
    assert merged < plain
    got, stats = gpu_run(ieti, prob, 2, coarse_top=2, **kw)
    for l, (a, b) in enumerate(zip(ref, got)):
        assert np.linalg.norm(a - b) <= TOL[mode] * np.linalg.norm(a), (name, mode, l, stats[l])


def test_nd_with_autotuned_schedule(ieti):
    """The autotuner re-cuts the level partitions for every schedule it times."""
    prob, op, ref = oracle_run("c4_family", 2)
    got, stats = gpu_run(ieti, prob, 2, precond="dirichlet_stiff", coarse="nd", autotune=1, **OPTS["mixed"])
    for a, b in zip(ref, got):
        assert np.linalg.norm(a - b) <= TOL["mixed"] * np.linalg.norm(a)


def test_nd_option_validation(ieti):
    prob = CASES["c1"]()
    with pytest.raises(ieti.IetiError) as e:
        ieti.Solver.from_problem(prob, device=0, coarse="nd", pcg_mode=1, **OPTS["fp64"])
    assert e.value.code == -1


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["ragged_p23", "c4_family"])
def test_batched_factorization_equals_one_batch(ieti, name, mode):
    """The patch blocks factored in batches that reuse one arena (a 1 MiB budget: a few
    patches per batch) give the operators of the one-batch factorization: same states
    (same arithmetic per patch, coarse contributions added in the same patch order)."""
    prob, op, ref = oracle_run(name, 2)
    S = ieti.Solver.from_problem(prob, device=0, precond="dirichlet_stiff", factor_arena_mb=1, **OPTS[mode])
    nb = S.info()["factor_batches"]
    S.close()
    assert nb > 1
    kw = dict(precond="dirichlet_stiff", **OPTS[mode])
    a1, _ = gpu_run(ieti, prob, 2, **kw)
    ab, _ = gpu_run(ieti, prob, 2, factor_arena_mb=1, **kw)
    for x, y, r in zip(a1, ab, ref):
        assert np.array_equal(x, y)
        assert np.linalg.norm(y - r) <= TOL[mode] * np.linalg.norm(r)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["c4_family", "ragged_p23", "c3_family"])
def test_nd_levels_on_node_counters(ieti, name, mode, tmp_path):
    """The coarse levels waiting on per-node completion counters (a node's children
    done; its parent final) instead of grid barriers, forced through the schedule cache:
    the same states as with the barriers (same arithmetic and order), within the parity
    tolerance of the oracle, in the host loop and in the step graph."""
    prob, op, ref = oracle_run(name, 3)
    cache = tmp_path / "tune.txt"
    kw = dict(precond="dirichlet_stiff", coarse="nd", coarse_leaf=1, **OPTS[mode])
    S = ieti.Solver.from_problem(prob, device=0, autotune=1, tune_cache=str(cache), **kw)
    S.close()
    line = [l for l in cache.read_text().splitlines() if l.startswith("ieti_tune3 ")][0].split()
    for graph in (0, 1):
        states = {}
        for flow in (0, 1):
            cache.write_text(" ".join(line[:7] + [str(flow)]) + "\n")
            S = ieti.Solver.from_problem(prob, device=0, autotune=1, tune_cache=str(cache), graph=graph, **kw)
            inf = S.info()
            assert inf["pcg_sched_source"] == 3 and inf["coarse_flow"] == flow
            j = S.load_vector(prob.coil)
            out = []
            for _ in range(3):
                S.step(j)
                out.append(S.solution().copy())
            S.close()
            states[flow] = out
        for a, b, r in zip(states[0], states[1], ref):
            assert np.array_equal(a, b)
            assert np.linalg.norm(b - r) <= TOL[mode] * np.linalg.norm(r)
