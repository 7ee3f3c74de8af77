// Tensor-core trailing update of the batched partial Cholesky (FP32 data).
//
// The right-looking blocked factorization of every augmented patch block (the
// two Schur complements of Sec. 3) spends its flops in the trailing update
// A22 -= L21 L21^T.  Here that update runs on the tcgen05 tensor cores in TF32
// (or, as an ablation, BF16) with FP32 accumulation in tensor memory, once per
// outer panel of TC_KP = 256 columns (the inner 32-column steps stay on the SIMT
// kernels):
//
//   1. k_panel_split writes the finished panel rows L21 of every patch into a
//      stacked panel buffer (rows ro[s] + r, TC_KP columns, zero padded) as two
//      planes, hi = round(L21) and lo = round(L21 - hi), rounded to TF32 (kept in
//      FP32 words) or to BF16 (16-bit words).
//   2. k_syrk_tc: one persistent CTA per SM walks a host-built list of
//      128 x 128 output tiles (patch-major, lower triangle only).  Warp 0 feeds
//      the 128-byte-swizzled K-major operand tiles (one K chunk of 128 bytes per
//      row and stage: 32 TF32 or 64 BF16 values) by TMA through a shared-memory
//      ring; warp 1 issues, per chunk,
//      the MMAs hi*hi into one TMEM accumulator and (three-term split, FP32
//      accuracy) hi*lo + lo*hi into a second, alternating between two chunk
//      buffers; 16 epilogue warps add every chunk's accumulators to FP32 register
//      sums (one row and 32 of the tile's columns per thread) and finally subtract the sums from A22 in global
//      memory (lower triangle, the patch's active rows, the AugLimits
//      restrictions).  The tensor cores truncate when they accumulate; a fresh
//      accumulator per chunk and round-to-nearest sums across chunks keep that
//      error at the level of the SIMT FP32 update instead of growing with K.
//
// Every wait is bounded; a timeout sets *err_flag, stops the work loops, drains
// the copies and MMAs in flight and frees the tensor memory before returning.
#pragma once
#include <cuda.h>  // CUtensorMap
#include <cuda_bf16.h>

#include <climits>
#include <cstdint>
#include <type_traits>

#include "tc.cuh"

namespace ieti {

// Per-patch restrictions of a partial-Cholesky phase: rows in [sk_lo, sk_hi) hold
// zeros in the pivot columns (no work); rows >= rlim only need columns < clim.
struct AugLimits {
  const int32_t *sk_lo, *sk_hi, *rlim, *clim;
};

constexpr int TC_KP = 256;  // outer panel width = K of one trailing update
constexpr int TC_BM = 128;  // tile rows (MMA M)
constexpr int TC_BN = 128;  // tile columns (MMA N)
constexpr int TC_EPI_WARPS = 16;                          // 4 per TMEM lane quarter
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);        // producer, MMA issuer, epilogue
constexpr int TC_EPI_COLS = TC_BN / (TC_EPI_WARPS / 4);    // columns per epilogue thread

struct TcItem {
  int32_t s, R0, C0, t0, nk, pad;  // patch, tile origin, first trailing column, K chunks
};

// Operand element of the trailing update: BF = 0 TF32 (FP32 words, kind::tf32, 8 K per
// MMA), BF = 1 BF16 (kind::f16, 16 K per MMA).  Either way a K chunk fills one
// 128-byte swizzle row and one MMA consumes 32 bytes of it.
template <int BF>
struct TcElem {
  using T = typename std::conditional<BF != 0, __nv_bfloat16, float>::type;
  static constexpr int KCH = 128 / (int)sizeof(T);  // K values per chunk
  static constexpr uint32_t FMT = BF ? 1u : 2u;      // operand format in the instruction descriptor
};

__device__ __forceinline__ void split_store(float v, float *hi, float *lo, int k, bool x3) {
  float h = 0.f;
  {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    h = __uint_as_float(r);
  }
  hi[k] = h;
  if (x3) lo[k] = v - h;
}
__device__ __forceinline__ void split_store(float v, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int k, bool x3) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[k] = h;
  if (x3) lo[k] = __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Panel P of every patch: rows [t0, nact) x columns [J, J + jb) -> planes hi (and lo)
// of the stacked panel buffer PB (plane stride R_total * TC_KP elements), zero padded
// to TC_KP columns.  One warp per row.
template <int X3, int BF>
__global__ void k_panel_split(const float *base, const int64_t *off, const int32_t *ldv, const int32_t *kbeg,
                              const int32_t *kend, const int32_t *nact, int P, const int64_t *ro, int64_t R_total,
                              typename TcElem<BF>::T *PB) {
  int s = blockIdx.y;
  int J = kbeg[s] + P * TC_KP;
  int ke = kend[s];
  if (J >= ke) return;
  int jb = min(TC_KP, ke - J);
  int t0 = J + jb;
  int m = nact[s] - t0;
  int lane = threadIdx.x & 31;
  int wpb = blockDim.x >> 5;
  int64_t ld = ldv[s];
  const float *A = base + off[s];
  for (int rr = blockIdx.x * wpb + (threadIdx.x >> 5); rr < m; rr += gridDim.x * wpb) {
    int r = t0 + rr;
    const float *src = A + (int64_t)r * ld + J;
    auto *hi = PB + (ro[s] + r) * (int64_t)TC_KP;
    auto *lo = hi + R_total * (int64_t)TC_KP;
    for (int k = lane; k < TC_KP; k += 32) split_store(k < jb ? src[k] : 0.f, hi, lo, k, X3 != 0);
  }
}

template <int X3>
struct TcCfg {
  static constexpr int NPLANE = X3 ? 2 : 1;
  static constexpr int NS = X3 ? 3 : 6;  // ring stages (one K chunk each)
  static constexpr uint32_t A_BYTES = TC_BM * 128;  // one plane, 128 bytes of K per row
  static constexpr uint32_t B_BYTES = TC_BN * 128;
  static constexpr uint32_t STAGE = NPLANE * (A_BYTES + B_BYTES);
  static constexpr uint32_t SMEM = NS * STAGE + 1024 /* alignment */ + 256 /* barriers */;
};

// TMEM: two chunk buffers of 2 * TC_BN columns: [hi*hi | hi*lo + lo*hi]
constexpr uint32_t TC_TMEM_COLS = 4 * TC_BN;

template <int X3, int BF>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_syrk_tc(const __grid_constant__ CUtensorMap tmap, const TcItem *items, int n_items, float *base,
              const int64_t *off, const int32_t *ldv, const int64_t *ro, const int32_t *nact, AugLimits lim,
              int32_t *err_flag) {
  using C = TcCfg<X3>;
  using E = TcElem<BF>;
  constexpr uint32_t IDESC = tc_idesc(E::FMT, TC_BM, TC_BN);
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(sm + C::NS * C::STAGE);
  uint64_t *empty = full + C::NS;
  uint64_t *cfull = empty + C::NS;  // [2] chunk accumulators ready
  uint64_t *cempty = cfull + 2;     // [2] chunk accumulators drained by the epilogue
  uint64_t *drain = cempty + 2;
  uint32_t *tbase = (uint32_t *)(drain + 1);
  volatile int *abort_ = (volatile int *)(tbase + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NS; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(cfull + i, 1);
      mbar_init(cempty + i, TC_EPI_WARPS);
    }
    mbar_init(drain, 1);
    *abort_ = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    tmem_alloc(tbase, TC_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;
  auto give_up = [&](int code) {
    *abort_ = 1;
    atomicCAS(err_flag, 0, code);
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmap);
      int it = 0;
      for (int w = blockIdx.x; w < n_items && !*abort_; w += gridDim.x) {
        const TcItem t = items[w];
        const int ya = (int)(ro[t.s] + t.R0), yb = (int)(ro[t.s] + t.C0);
        for (int kc = 0; kc < t.nk; ++kc, ++it) {
          const int st = it % C::NS;
          const unsigned ph = (unsigned)(it / C::NS) & 1u;
          if (!mbar_wait(empty + st, ph ^ 1u)) {
            give_up(1);
            break;
          }
          unsigned char *sb = sm + st * C::STAGE;
          mbar_arrive_expect_tx(full + st, C::STAGE);
#pragma unroll
          for (int pl = 0; pl < C::NPLANE; ++pl) {
            tma_load_3d(sb + pl * C::A_BYTES, &tmap, kc * E::KCH, ya, pl, full + st);
            tma_load_3d(sb + C::NPLANE * C::A_BYTES + pl * C::B_BYTES, &tmap, kc * E::KCH, yb, pl, full + st);
          }
        }
      }
      // the last fill of every stage has landed before the CTA may exit
      for (int i = (it > C::NS ? it - C::NS : 0); i < it; ++i)
        if (!mbar_wait(full + i % C::NS, (unsigned)(i / C::NS) & 1u)) give_up(2);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int it = 0;  // chunk counter (ring stage and chunk buffer)
      for (int w = blockIdx.x; w < n_items && !*abort_; w += gridDim.x) {
        const TcItem t = items[w];
        bool ok = true;
        for (int kc = 0; kc < t.nk; ++kc, ++it) {
          const int cb = it & 1;
          const unsigned cph = (unsigned)(it >> 1) & 1u;
          if (!mbar_wait(cempty + cb, cph ^ 1u)) {
            give_up(3);
            ok = false;
            break;
          }
          const int st = it % C::NS;
          const unsigned ph = (unsigned)(it / C::NS) & 1u;
          if (!mbar_wait(full + st, ph)) {
            give_up(4);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dh = tmem + (uint32_t)(cb * 2 * TC_BN), dc = dh + TC_BN;
          const uint32_t sa = smem_u32(sm + st * C::STAGE);
          const uint32_t sb = sa + C::NPLANE * C::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 4 MMAs of 32 bytes of K inside the 128-byte row
            const uint64_t ah = tc_desc_sw128(sa + kk * 32), bh = tc_desc_sw128(sb + kk * 32);
            tc_mma<BF>(dh, ah, bh, IDESC, kk != 0);
            if constexpr (X3) {
              const uint64_t al = tc_desc_sw128(sa + C::A_BYTES + kk * 32);
              const uint64_t bl = tc_desc_sw128(sb + C::B_BYTES + kk * 32);
              tc_mma<BF>(dc, ah, bl, IDESC, kk != 0);
              tc_mma<BF>(dc, al, bh, IDESC, 1u);
            }
          }
          tc_commit(empty + st);  // the stage is free once these MMAs have read it
          tc_commit(cfull + cb);  // the chunk accumulators are complete
        }
        if (!ok) break;
      }
      tc_commit(drain);
      if (!mbar_wait(drain, 0)) give_up(5);
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2-17)
    // Every K chunk is accumulated afresh in TMEM and added here to FP32
    // register sums with round-to-nearest: the tensor-core accumulation then spans
    // 4 MMAs of one chunk instead of a whole panel.  Each thread owns one row and
    // TC_EPI_COLS columns of the tile; its part of A22 is loaded when the tile
    // starts, so the read is in flight while the tile's chunks are multiplied.
    const int q = warp & 3;                                      // TMEM lane quarter of this warp
    const int c_off = ((warp - 2) >> 2) * TC_EPI_COLS;           // its columns of the tile
    const uint32_t lane_off = ((uint32_t)(q * 32) << 16) + (uint32_t)c_off;
    int it = 0;
    bool dead = false;
    for (int w = blockIdx.x; w < n_items && !dead; w += gridDim.x) {
      const TcItem t = items[w];
      const int s = t.s;
      const int na = nact[s], sk_lo = lim.sk_lo[s], sk_hi = lim.sk_hi[s], rlim = lim.rlim[s], clim = lim.clim[s];
      const int r = t.R0 + q * 32 + lane;
      const bool row_ok = r < na && !(r >= sk_lo && r < sk_hi);
      const int cmax = row_ok ? min(r, (r >= rlim) ? clim - 1 : INT_MAX) : -1;  // last column this row updates
      const int cb0 = t.C0 + c_off;
      float4 *Arow = reinterpret_cast<float4 *>(base + off[s] + (int64_t)(row_ok ? r : 0) * ldv[s] + cb0);
      float4 x[TC_EPI_COLS / 4];
#pragma unroll
      for (int g = 0; g < TC_EPI_COLS / 4; ++g) {
        const int c = cb0 + 4 * g;
        if (!(c + 3 < t.t0 || c > cmax)) x[g] = Arow[g];  // groups holding an updated column
      }
      float acc[TC_EPI_COLS];
#pragma unroll
      for (int j = 0; j < TC_EPI_COLS; ++j) acc[j] = 0.f;
      for (int kc = 0; kc < t.nk; ++kc, ++it) {
        const int cb = it & 1;
        const unsigned cph = (unsigned)(it >> 1) & 1u;
        const bool ok = mbar_wait(cfull + cb, cph);
        if (__any_sync(0xffffffffu, !ok || *abort_)) {
          if (lane == 0) give_up(6);
          dead = true;
          break;
        }
        tc_fence_after();
        const uint32_t dh = tmem + lane_off + (uint32_t)(cb * 2 * TC_BN);
#pragma unroll
        for (int g = 0; g < TC_EPI_COLS / 8; ++g) {
          float h[8];
          tmem_ld8(dh + g * 8, h);
          if constexpr (X3) {
            float c[8];
            tmem_ld8(dh + TC_BN + g * 8, c);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[g * 8 + i] += h[i] + c[i];
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[g * 8 + i] += h[i];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(cempty + cb);
      }
      if (dead) break;
#pragma unroll
      for (int g = 0; g < TC_EPI_COLS / 4; ++g) {
        const int c = cb0 + 4 * g;
        if (c + 3 < t.t0 || c > cmax) continue;  // no updated column in this group
        float4 v = x[g];
        if (c + 0 >= t.t0 && c + 0 <= cmax) v.x -= acc[4 * g + 0];
        if (c + 1 >= t.t0 && c + 1 <= cmax) v.y -= acc[4 * g + 1];
        if (c + 2 >= t.t0 && c + 2 <= cmax) v.z -= acc[4 * g + 2];
        if (c + 3 >= t.t0 && c + 3 <= cmax) v.w -= acc[4 * g + 3];
        Arow[g] = v;
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TC_TMEM_COLS);
  }
}

}  // namespace ieti
