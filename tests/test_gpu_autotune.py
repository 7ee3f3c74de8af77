"""The schedule autotuner of the persistent dual-primal kernel (CTAs per SM, TMA ring
stages, bytes per stage) and its cache file, through the C ABI.  A schedule changes
only the rounding order of the cross-CTA reductions, so every schedule must give
the rule's state within the parity bounds (the bounds against the oracle are
checked in the parity tests)."""
import numpy as np
import pytest

from workloads import make_problem, small_problem

pytestmark = pytest.mark.gpu

OPTS = {"fp64": dict(precision="fp64", cg_tol=1e-12, max_sweeps=1),
        "mixed": dict(precision="mixed", cg_tol=1e-6, outer_tol=1e-12, max_sweeps=20, factor="tf32x3")}
# two runs that each meet the parity bound against the oracle (1e-10 FP64, 1e-8 mixed)
# agree to twice that bound
TOL = {"fp64": 2e-10, "mixed": 2e-8}


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
    out = []
    for _ in range(steps):
        S.step(j)
        out.append(S.solution().copy())
    info = S.info()
    S.close()
    return out, info


def _n_sm():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["c1", "ragged"])
def test_autotuned_schedule_gives_the_rule_state(ieti, mode, case):
    prob = make_problem("c1") if case == "c1" else _ragged()
    ref, inf0 = _run(ieti, prob, 3, **OPTS[mode])
    got, inf1 = _run(ieti, prob, 3, autotune=1, **OPTS[mode])
    assert inf0["pcg_sched_source"] == 0 and inf1["pcg_sched_source"] == 1
    assert inf1["tune_candidates"] >= 2
    assert inf1["pcg_grid"] % _n_sm() == 0 and inf1["pcg_grid"] // _n_sm() in (1, 2)
    assert inf1["pcg_stages"] in (2, 3, 4, 6) and inf1["pcg_stage_bytes"] % 128 == 0
    # the choice is the rule unless it measured faster than the rule
    assert inf1["tune_us_per_it"][1] <= inf1["tune_us_per_it"][0]
    for a, b in zip(ref, got):
        assert np.linalg.norm(a - b) <= TOL[mode] * np.linalg.norm(a)


def test_tune_cache_round_trip_and_forced_schedules(ieti, tmp_path):
    """A tuned choice is written to the cache and read back without timing; cache
    entries edited to other schedules (two stages of 16 KB; three of 32 KB with the Psi
    rows on their own partition; two CTAs per SM, infeasible with this kernel's
    registers) are used as given where feasible and reach the same state; malformed
    lines are ignored."""
    prob = _ragged()
    cache = tmp_path / "tune.txt"
    cache.write_text("garbage line\nieti_tune2 other-key 1 3 65536 0\nieti_tune2 short-line 1 3\n")
    ref, inf1 = _run(ieti, prob, 2, autotune=1, tune_cache=str(cache), **OPTS["mixed"])
    assert inf1["pcg_sched_source"] == 2
    lines = cache.read_text().splitlines()
    ours = [l for l in lines if l.startswith("ieti_tune3 ") and "other-key" not in l and "short-line" not in l]
    assert len(ours) == 1 and "garbage line" in lines and any("other-key" in l for l in lines)
    key = ours[0].split()[1]
    _, inf2 = _run(ieti, prob, 1, autotune=1, tune_cache=str(cache), **OPTS["mixed"])
    assert inf2["pcg_sched_source"] == 3 and inf2["tune_candidates"] == 0
    assert (inf2["pcg_grid"], inf2["pcg_stages"], inf2["pcg_stage_bytes"]) == \
        (inf1["pcg_grid"], inf1["pcg_stages"], inf1["pcg_stage_bytes"])
    for cps, ns, stage, psi in [(1, 2, 16384, 0), (1, 3, 32768, 64), (2, 2, 16384, 0)]:
        cache.write_text(f"ieti_tune2 {key} {cps} {ns} {stage} {psi}\n")
        got, inf = _run(ieti, prob, 2, autotune=1, tune_cache=str(cache), **OPTS["mixed"])
        if inf["pcg_sched_source"] != 3:        # not feasible on this device: tuned afresh instead
            assert cps == 2 and inf["pcg_sched_source"] == 2
            continue
        assert (inf["pcg_grid"], inf["pcg_stages"], inf["pcg_stage_bytes"], inf["pcg_psi_partition"]) == \
            (cps * _n_sm(), ns, stage, psi)
        for a, b in zip(ref, got):
            assert np.linalg.norm(a - b) <= TOL["mixed"] * np.linalg.norm(a)
