"""CPU checks of the library's host side: it loads, exports every symbol of
include/ieti.h, and its host setup (assembly, gauge, classes, load vector)
reproduces the oracle's on the same seeded inputs (no GPU compute)."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from workloads import make_problem, small_problem
from oracle.stepping import OracleProblem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ieti():
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti as mod
    return mod


def test_exports_every_declared_symbol(ieti):
    hdr = open(os.path.join(ROOT, "include", "ieti.h")).read()
    declared = set(re.findall(r"\b(ieti_[a-z0-9_]+)\s*\(", hdr))
    lib = ctypes.CDLL(ieti.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(ieti.EXPORTED)


CASES = {
    "c1": lambda: make_problem("c1"),
    "uneven": lambda: small_problem(P=(3, 2, 2), n_el=((2, 3, 2), (2, 3), (3, 2)),
                                    degree=((1, 2, 1), (2, 1), (1, 2)),
                                    conductor=((0.3, 0.7), (0, 1), (0, 1))),
    "buried": lambda: small_problem(P=(3, 3, 3), n_el=((2, 2, 2),) * 3, degree=((1, 1, 1),) * 3,
                                    conductor=((0.4, 0.6),) * 3),
    "c3_slice": lambda: small_problem(P=(4, 3, 2), n_el=((3, 2, 3, 2), (2, 3, 2), (3, 2)),
                                      degree=((2, 3, 2, 2), (3, 2, 2), (2, 3)),
                                      conductor=((0.2, 0.8), (0.3, 0.7), (0.0, 1.0))),
}


@pytest.mark.parametrize("name", list(CASES))
def test_host_setup_matches_oracle(ieti, name):
    prob = CASES[name]()
    S = ieti.Solver.from_problem(prob, device=-1)
    op = OracleProblem(prob)
    cls, tree = S.dof_classes()
    assert np.array_equal(cls, op.gauge.cls)            # integer work: bit-exact
    assert np.array_equal(tree.astype(bool), op.gauge.tree)
    j = S.load_vector(prob.coil)
    assert np.linalg.norm(j - op.asm.j_global) <= 1e-13 * np.linalg.norm(op.asm.j_global)
    for s in range(prob.n_patches):
        for which, ref in ((0, op.asm.K[s]), (1, op.asm.M[s])):
            ptr, col, val = S.patch_csr(s, which)
            A = sp.csr_matrix((val, col, ptr), shape=ref.shape)
            scale = max(abs(ref).max(), 1e-300)
            assert abs(A - ref).max() <= 1e-13 * scale
    info = S.info()
    assert info["n_coarse"] == op.dec.n_coarse
    assert info["n_lambda"] == op.dec.m
    S.close()


def test_c2_classes_match(ieti):
    prob = make_problem("c2")
    S = ieti.Solver.from_problem(prob, device=-1)
    from oracle.gauge import Gauge
    G = Gauge(prob)
    cls, tree = S.dof_classes()
    assert np.array_equal(cls, G.cls) and np.array_equal(tree.astype(bool), G.tree)
    S.close()


def test_host_only_context_refuses_compute(ieti):
    prob = make_problem("c1")
    S = ieti.Solver.from_problem(prob, device=-1)
    with pytest.raises(ieti.IetiError) as e:
        S.step(np.zeros(S.n))
    assert e.value.code == -7
    S.close()


@pytest.mark.parametrize("mutate,code", [
    (lambda p: setattr(p, "dt", -1.0), -1),
    (lambda p: p.sigma_el.__setitem__(0, np.nan), -1),
    (lambda p: p.knots[0].__setitem__(1, 0.3), -1),
])
def test_invalid_inputs_return_codes(ieti, mutate, code):
    prob = make_problem("c1")
    mutate(prob)
    with pytest.raises(ieti.IetiError) as e:
        ieti.Solver.from_problem(prob, device=-1)
    assert e.value.code == code


@pytest.mark.parametrize("kw", [
    dict(precision="fp64", factor="tf32x3"),   # the FP64 mode factors in FP64
    dict(precision="mixed", factor=7),
    dict(precision="mixed", pcg_mode=3),
    dict(precision="fp64", predictor=3),
    dict(precision="mixed", factor="bf16", autotune=2),
    dict(precision="fp64", graph=2),
    dict(precision="fp64", l2_persist=3),
    dict(precision="fp64", wait_limit=-1),
    dict(precision="fp64", coarse_leaf=-1),
    dict(precision="fp64", coarse_top=-1),
    dict(precision="fp64", deflation=2),
    dict(precision="fp64", coarse_ranks=32),
    dict(precision="fp64", coarse_ranks=-1),
])
def test_invalid_options_return_codes(ieti, kw):
    prob = make_problem("c1")
    with pytest.raises(ieti.IetiError) as e:
        ieti.Solver.from_problem(prob, device=-1, **kw)
    assert e.value.code == -1


def test_potrf_f32_rejects_bad_arguments_without_a_device(ieti):
    """Argument checks of ieti_potrf_batched_f32 run before any device work."""
    import ctypes as C
    z = np.zeros(1, dtype=np.int64)
    n = np.array([30], dtype=np.int32)
    ld = np.array([30], dtype=np.int32)      # not a multiple of 4: refused for the tensor-core modes
    st = np.zeros(1, dtype=np.int32)
    rc = ieti.lib.ieti_potrf_batched_f32(1, C.c_void_p(16), z.ctypes.data, n.ctypes.data, ld.ctypes.data,
                                         n.ctypes.data, 2, st.ctypes.data, None)
    assert rc == -1
    rc = ieti.lib.ieti_potrf_batched_f32(1, C.c_void_p(16), z.ctypes.data, n.ctypes.data, ld.ctypes.data,
                                         n.ctypes.data, 9, st.ctypes.data, None)
    assert rc == -1
    for factor in (4, 5):                    # BF16 tensor-core modes: same 16-byte rule
        rc = ieti.lib.ieti_potrf_batched_f32(1, C.c_void_p(16), z.ctypes.data, n.ctypes.data, ld.ctypes.data,
                                             n.ctypes.data, factor, st.ctypes.data, None)
        assert rc == -1


@pytest.mark.parametrize("name", ["uneven", "c3_slice"])
def test_load_vector_from_points_matches_oracle(ieti, name):
    """<J, w_k> from J sampled at the library's quadrature points equals the oracle's
    quadrature of the same analytic field (curved patches, uneven degrees)."""
    from oracle.manufactured import A_star, FieldEval
    prob = CASES[name]()
    op = OracleProblem(prob)
    S = ieti.Solver.from_problem(prob, device=-1)
    xyz = S.quad_points()
    assert xyz.shape[0] == sum(int(np.prod(prob.patch_n_el(s))) * int(np.prod(np.asarray(prob.patch_degree(s)) + 2))
                               for s in range(prob.n_patches))
    field = lambda x: A_star(x) * (1.0 + x[..., :1])      # smooth, direction-dependent
    got = S.load_vector_points(field(xyz))
    ref = FieldEval(prob, op.asm).load(field)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    # the points lie in the unit cube and sample every element
    assert xyz.min() > 0.0 and xyz.max() < 1.0
    S.close()
