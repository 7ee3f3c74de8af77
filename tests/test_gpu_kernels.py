"""Kernel-level GPU parity: the batched partial Cholesky (both Schur complements of
Sec. 3 are computed with it) against NumPy/LAPACK on random SPD batches of uneven
sizes, through the C ABI."""
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


def _spd(rng, n):
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


def _batch(rng, sizes):
    mats = [_spd(rng, n) for n in sizes]
    offs = np.cumsum([0] + [n * n for n in sizes[:-1]]).astype(np.int64)
    flat = np.concatenate([m.ravel() for m in mats])
    return mats, offs, flat


@pytest.mark.parametrize("sizes,piv", [
    ([1, 5, 31, 32, 33, 64, 65, 130], "full"),
    ([7, 100, 257, 3, 96], "partial"),
    ([300], "full"),
])
def test_partial_cholesky_matches_lapack(ieti, sizes, piv):
    import torch
    rng = np.random.default_rng(1)
    mats, offs, flat = _batch(rng, sizes)
    k = [n if piv == "full" else max(0, n - (n // 3) - 1) for n in sizes]
    base = torch.from_numpy(flat.copy()).cuda()
    st = ieti.potrf_batched(base, offs, sizes, k)
    assert np.all(st == 0)
    out = base.cpu().numpy()
    for A, o, n, kk in zip(mats, offs, sizes, k):
        R = out[o:o + n * n].reshape(n, n)
        L = np.tril(R[:, :kk])
        L11 = np.linalg.cholesky(A[:kk, :kk]) if kk else np.zeros((0, 0))
        assert np.abs(np.tril(L[:kk]) - L11).max() <= 1e-12 * max(1.0, np.abs(L11).max(initial=1.0))
        if kk < n:
            L21 = np.linalg.solve(L11, A[:kk, kk:]).T if kk else np.zeros((n - kk, 0))
            assert np.abs(L[kk:] - L21).max() <= 1e-11 * max(1.0, np.abs(L21).max(initial=1.0))
            S = A[kk:, kk:] - L21 @ L21.T
            assert np.abs(np.tril(R[kk:, kk:]) - np.tril(S)).max() <= 1e-11 * np.abs(S).max()


def test_partial_cholesky_flags_indefinite(ieti):
    import torch
    rng = np.random.default_rng(2)
    mats, offs, flat = _batch(rng, [20, 40])
    M = mats[1].copy()
    M[10, 10] = -5.0 * abs(M).max()
    flat = np.concatenate([mats[0].ravel(), M.ravel()])
    base = torch.from_numpy(flat).cuda()
    st = ieti.potrf_batched(base, offs, [20, 40], [20, 40])
    assert st[0] == 0 and st[1] == 1 + 10


def test_partial_cholesky_rejects_bad_args(ieti):
    import torch
    base = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(ieti.IetiError) as e:
        ieti.potrf_batched(base, [0], [4], [5])
    assert e.value.code == -1
