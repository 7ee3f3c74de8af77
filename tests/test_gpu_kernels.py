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


# ----------------------------------------------------------------------------- FP32 / tensor cores
def _batch_f32(rng, sizes, pad=4):
    """SPD matrices rounded to FP32, row-major with a padded leading dimension
    (a multiple of 4) at 16-byte aligned offsets."""
    mats, lds, offs, o = [], [], [], 0
    for n in sizes:
        A = _spd(rng, n) / n
        mats.append(A.astype(np.float32).astype(np.float64))
        ld = (n + 3) // 4 * 4 + pad
        lds.append(ld)
        offs.append(o)
        o += n * ld
    flat = np.full(o, np.nan, dtype=np.float32)   # padding columns stay NaN: never read into results
    for A, n, ld, off in zip(mats, sizes, lds, offs):
        blk = np.full((n, ld), -7.0, dtype=np.float32)
        blk[:, :n] = A
        flat[off:off + n * ld] = blk.ravel()
    return mats, np.array(offs, np.int64), np.array(lds, np.int32), flat


def _f32_errors(mats, offs, lds, sizes, piv, out, inp):
    errs = []
    for A, o, ld, n, kk in zip(mats, offs, lds, sizes, piv):
        R = out[o:o + n * ld].reshape(n, ld)[:, :n].astype(np.float64)
        R0 = inp[o:o + n * ld].reshape(n, ld)
        # the strict upper triangle and the padding columns are left bit-identical
        iu = np.triu_indices(n, 1)
        assert np.array_equal(out[o:o + n * ld].reshape(n, ld)[iu], R0[iu])
        assert np.array_equal(out[o:o + n * ld].reshape(n, ld)[:, n:], R0[:, n:])
        L11 = np.linalg.cholesky(A[:kk, :kk])
        e = np.abs(np.tril(R[:kk, :kk]) - L11).max() / np.abs(L11).max()
        if kk < n:
            L21 = np.linalg.solve(L11, A[:kk, kk:]).T
            S = A[kk:, kk:] - L21 @ L21.T
            e = max(e, np.abs(R[kk:, :kk] - L21).max() / np.abs(L21).max(),
                    np.abs(np.tril(R[kk:, kk:]) - np.tril(S)).max() / np.abs(S).max())
        errs.append(e)
    return np.array(errs)


@pytest.mark.parametrize("sizes,frac", [
    ([300, 520, 1030, 64, 7, 257], 1.0),       # full factorizations, several 256-column panels, ragged
    ([700, 900, 33, 1200], 0.55),               # partial: trailing Schur complements
])
def test_partial_cholesky_f32_modes(ieti, sizes, frac):
    import torch
    rng = np.random.default_rng(7)
    mats, offs, lds, flat = _batch_f32(rng, sizes)
    piv = [max(1, int(round(frac * n))) for n in sizes]
    err = {}
    for mode in ("fp32", "tf32x3", "tf32", "bf16x3", "bf16"):
        base = torch.from_numpy(flat.copy()).cuda()
        st = ieti.potrf_batched_f32(base, offs, sizes, lds, piv, factor=mode)
        assert np.all(st == 0), (mode, st)
        err[mode] = _f32_errors(mats, offs, lds, sizes, piv, base.cpu().numpy(), flat)
    print({k: v.max() for k, v in err.items()})
    # FP32 arithmetic (SIMT or three TF32 products) vs the exact factor of the FP32 input
    assert err["fp32"].max() <= 2e-5, err
    assert err["tf32x3"].max() <= 2e-5, err
    # one TF32 product carries an 11-bit operand: clearly worse, still a factorization
    assert err["tf32"].max() <= 1e-2, err
    big = [i for i, n in enumerate(sizes) if piv[i] < n or n > 256]   # the tensor-core update ran
    assert err["tf32"][big].min() > 10 * err["tf32x3"][big].max(), err
    # BF16 ablation: hi + lo planes carry ~16 significant bits (three products), one
    # product 8 bits, i.e. 8x the TF32 operand rounding
    assert err["bf16x3"].max() <= 2e-4, err
    assert err["bf16"].max() <= 5e-2, err
    assert err["bf16"][big].min() > 10 * err["bf16x3"][big].max(), err
    assert err["bf16"][big].mean() > 2 * err["tf32"][big].mean(), err


def test_partial_cholesky_f32_flags_indefinite(ieti):
    import torch
    rng = np.random.default_rng(3)
    mats, offs, lds, flat = _batch_f32(rng, [600, 300])
    n, ld, o = 600, int(lds[0]), int(offs[0])
    flat[o + 400 * ld + 400] = -1e3
    for mode in ("fp32", "tf32x3"):
        base = torch.from_numpy(flat.copy()).cuda()
        st = ieti.potrf_batched_f32(base, offs, [600, 300], lds, [600, 300], factor=mode)
        assert st[0] == 1 + 400 and st[1] == 0, (mode, st)


def test_partial_cholesky_f32_rejects_misaligned(ieti):
    import torch
    base = torch.zeros(4096, dtype=torch.float32, device="cuda")
    with pytest.raises(ieti.IetiError) as e:
        ieti.potrf_batched_f32(base, [2], [30], [32], [30], factor="tf32x3")   # offset not a multiple of 4
    assert e.value.code == -1
    with pytest.raises(ieti.IetiError) as e:
        ieti.potrf_batched_f32(base, [0], [30], [30], [30], factor="tf32x3")   # ld not a multiple of 4
    assert e.value.code == -1
