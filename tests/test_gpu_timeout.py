"""Failure detection on the device without a GPU fault: every grid-barrier wait of the
persistent dual-primal kernel is bounded.  With the bound set to a couple of polls
(ieti_options.wait_limit) the first barrier runs out before the other CTAs arrive;
the kernel must then set its error flag, let every CTA wait for its own copies in
flight and return, so that the step reports IETI_ERR_TIMEOUT (host loop and graph
mode) and the process, the device and the context stay usable."""
import numpy as np
import pytest

from workloads import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ieti():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti as mod
    return mod


@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_barrier_wait_runs_out_and_reports(ieti, graph, precision):
    import torch
    prob = make_problem("c1")
    kw = dict(precision=precision, precond="dirichlet_stiff", cg_tol=1e-10, autotune=0, graph=graph)
    if precision == "mixed":
        kw.update(factor="tf32x3", cg_tol=1e-6)
    S = ieti.Solver.from_problem(prob, device=0, wait_limit=1, **kw)
    jd = torch.from_numpy(S.load_vector(prob.coil)).cuda()
    st = S.step(jd, raise_on_error=False)
    assert st["rc"] == -9, st
    assert b"timed out" in ieti.lib.ieti_last_error(S.ctx)
    # the context still answers, and the device runs the next context's steps
    assert np.all(np.isfinite(S.solution()))
    S.close()
    torch.cuda.synchronize()
    R = ieti.Solver.from_problem(prob, device=0, **kw)
    st = R.step(jd)
    assert st["rc"] == 0 and st["cg_its"] > 0
    R.close()
