"""ieti_potrf_batched_noalloc: the batched partial Cholesky for callers that cannot
allocate device memory (its scratch is a static device array).  Called through the
C ABI twice in a row on different batches, it must reproduce ieti_potrf_batched
(same kernels) within the kernel tests' tolerance, and reject oversized batches.
This file is collected last, and passes alone in a fresh process as well."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ieti():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti as mod
    return mod


def _batch(seed, sizes):
    rng = np.random.default_rng(seed)
    mats = []
    for n in sizes:
        A = rng.standard_normal((n, n))
        mats.append(A @ A.T + n * np.eye(n))
    offs = np.cumsum([0] + [n * n for n in sizes[:-1]]).astype(np.int64)
    return offs, np.concatenate([m.ravel() for m in mats])


def _call(ieti, fn, flat, offs, sizes, piv):
    import torch
    base = torch.from_numpy(flat.copy()).cuda()
    nn = np.asarray(sizes, dtype=np.int32)
    kp = np.asarray(piv, dtype=np.int32)
    st = np.full(len(sizes), -1, dtype=np.int32)
    rc = fn(len(sizes), ctypes.c_void_p(base.data_ptr()), offs.ctypes.data, nn.ctypes.data, kp.ctypes.data,
            st.ctypes.data, ctypes.c_void_p(0))
    assert rc == 0, ieti.lib.ieti_setup_error().decode()
    return base.cpu().numpy(), st


@pytest.mark.parametrize("seed,sizes,piv", [
    (11, [3, 40, 65, 129, 17], [3, 40, 50, 100, 0]),
    (12, [200, 33, 1, 96], [200, 20, 1, 96]),
])
def test_noalloc_matches_allocating_entry_point(ieti, seed, sizes, piv):
    offs, flat = _batch(seed, sizes)
    ref, st_ref = _call(ieti, ieti.lib.ieti_potrf_batched, flat, offs, sizes, piv)
    for _ in range(2):                                   # two calls in a row share the scratch
        got, st = _call(ieti, ieti.lib.ieti_potrf_batched_noalloc, flat, offs, sizes, piv)
        assert np.array_equal(st, st_ref) and np.all(st == 0)
        for o, n in zip(offs, sizes):
            a = np.tril(ref[o:o + n * n].reshape(n, n))
            b = np.tril(got[o:o + n * n].reshape(n, n))
            assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


def test_noalloc_rejects_oversized_batch(ieti):
    import torch
    n_max = 4096
    base = torch.zeros(n_max + 1, dtype=torch.float64, device="cuda")
    offs = np.arange(n_max + 1, dtype=np.int64)
    nn = np.ones(n_max + 1, dtype=np.int32)
    st = np.zeros(n_max + 1, dtype=np.int32)
    rc = ieti.lib.ieti_potrf_batched_noalloc(n_max + 1, ctypes.c_void_p(base.data_ptr()), offs.ctypes.data,
                                             nn.ctypes.data, nn.ctypes.data, st.ctypes.data, ctypes.c_void_p(0))
    assert rc == -8
    assert b"IETI_NOALLOC_MAX_BATCH" in ieti.lib.ieti_setup_error()
