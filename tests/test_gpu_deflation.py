"""GPU parity of the balanced (deflated) preconditioner (Sec. 5 outlook, read as
M_bal = (I - P) M (I - P)^T + U E^{-1} U^T over the patch-pair space U) against the
oracle: the oracle's monolithic solve for the state (FP64 path <= 1e-10, mixed path
<= 1e-8) and the oracle's balanced PCG for the iteration count (FP64, within one).
The pair space's dimension is the oracle's number of patch pairs."""
import numpy as np
import pytest

from workloads import make_problem, small_problem
from oracle.ietidp import PRECOND_STIFF, PRECOND_DIRICHLET
from oracle.stepping import OracleProblem

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-8}
OPTS = {"fp64": dict(precision="fp64", cg_tol=1e-12, max_sweeps=1),
        "mixed": dict(precision="mixed", cg_tol=1e-6, outer_tol=1e-12, max_sweeps=20)}
CASES = {
    "c1": lambda: make_problem("c1"),
    "uneven": lambda: small_problem(P=(3, 2, 2), n_el=((2, 3, 2), (2, 3), (3, 2)),
                                    degree=((1, 2, 1), (2, 1), (1, 2)),
                                    conductor=((0.3, 0.7), (0, 1), (0, 1))),
    "c3_family": lambda: make_problem("c3", patches_per_dir=3, n_el=2),
}
_REF = {}


@pytest.fixture(scope="module")
def ieti():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti as mod
    return mod


def oracle(name, steps):
    if (name, steps) not in _REF:
        prob = CASES[name]()
        op = OracleProblem(prob)
        _REF[(name, steps)] = (prob, op, op.run_monolithic(steps))
    return _REF[(name, steps)]


def gpu_run(ieti, prob, steps, **kw):
    S = ieti.Solver.from_problem(prob, device=0, **kw)
    j = S.load_vector(prob.coil)
    out, stats = [], []
    for _ in range(steps):
        stats.append(S.step(j))
        out.append(S.solution().copy())
    info = S.info()
    S.close()
    return out, stats, info


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("precond", ["dirichlet_stiff", "dirichlet"])
def test_balanced_steps_match_oracle(ieti, name, mode, precond):
    prob, op, ref = oracle(name, 2)
    got, stats, info = gpu_run(ieti, prob, 2, precond=precond, deflation=1, **OPTS[mode])
    assert info["deflation_dim"] == op.dec.pair_space().shape[1] > 0
    for l, (a, b) in enumerate(zip(ref, got)):
        assert np.linalg.norm(a - b) <= TOL[mode] * np.linalg.norm(a), (name, mode, precond, l, stats[l])


@pytest.mark.parametrize("name", ["c1", "c3_family"])
def test_balanced_iteration_counts_match_oracle(ieti, name):
    prob, op, _ = oracle(name, 1)
    for gpu_pc, pc in (("dirichlet_stiff", PRECOND_STIFF), ("dirichlet", PRECOND_DIRICHLET)):
        _, its = op.run_ietidp(1, tol=1e-8, precond=pc, deflation=True)
        _, stats, _ = gpu_run(ieti, prob, 1, precond=gpu_pc, deflation=1, precision="fp64", cg_tol=1e-8,
                              max_sweeps=1)
        assert abs(stats[0]["cg_its"] - its[0]) <= 1, (name, gpu_pc, stats[0]["cg_its"], its[0])


def test_none_preconditioner_balanced(ieti):
    """The balancing form also wraps the identity (deflated plain CG)."""
    prob, op, ref = oracle("uneven", 2)
    got, stats, _ = gpu_run(ieti, prob, 2, precond="none", deflation=1, **OPTS["fp64"])
    for a, b in zip(ref, got):
        assert np.linalg.norm(a - b) <= TOL["fp64"] * np.linalg.norm(a)
