// Persistent cooperative PCG on the dual interface problem F lambda = d (Sec. 3-4:
// Dirichlet-preconditioned CG, lambda_0 = 0, stop on ||r|| <= tol ||d||).
//
// One launch runs every iteration.  Per iteration six phases separated by grid
// barriers (monotonic arrival counter; a wait that does not complete within ~2 s
// sets an error flag and every CTA returns):
//   P1  beta from the (r,z) partials; p_new = z + beta p_old (owners store it, the
//       gathers recompute it); u = B^T p_new per patch (kept in ub);
//       [F_s; Psi_s^T] u_s  -> zb, tpi
//   P2  coarse right-hand side c = -sum_s A_s^T tpi  (chunk per CTA)
//   P3  q = S_c^{-1} c (c staged whole in shared memory, rows per CTA)
//   P4  zf = zb - Psi_s q per interface row; partials of (p, F p) = (u, zf)
//   P5  alpha; owners: F p = B zf, lambda += alpha p, r_new = r - alpha F p;
//       Dirichlet preconditioner S_bb (B_D^T r_new) per patch -> zp (r_new
//       recomputed in the gather)
//   P6  convergence test on ||r_new||; z = B_D zp; partials of (r_new, z)
// Every vector written by another CTA inside the launch is read with ld.global.cg.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "tma.cuh"

namespace ieti {

constexpr int PCG_THREADS = 256;
constexpr int BT_W = 3;   // multipliers per interface copy (a DOF shared by at most 4 patches)
constexpr int CP_W = 4;   // copies per coarse DOF

template <class T>
struct PcgArgs {
  int64_t m;
  int nc, ldc;
  int precond_none, scaled;
  int max_it;
  double tol2;
  // multipliers: ELL gather lists per interface copy, pairs per multiplier
  const int32_t *bt_lam;            // [NBt][BT_W], -1 = none
  const double *bt_sgn, *bt_wd;     // [NBt][BT_W]
  const int32_t *lam_qp, *lam_qm;
  const double *lam_wp, *lam_wm;
  // per patch
  const int64_t *bofs, *pofs, *hoff, *qoff, *poff;
  const int32_t *nb, *np, *ldb, *ldp;
  const int32_t *pc;
  const int32_t *cp_pos;            // [nc][CP_W], -1 = none
  const T *H, *Q, *P;
  const double *Sinv;
  // work partitions (per CTA)
  const int32_t *hseg_ptr, *hseg_s, *hseg_r0, *hseg_r1;   // H rows
  const int32_t *bseg_ptr, *bseg_s, *bseg_r0, *bseg_r1;   // interface rows (Psi and P)
  // vectors
  const double *d;
  double *lam, *p0, *p1, *r0, *r1, *z, *ub, *zb, *zf, *tpi, *cc, *q, *zp;
  double *part;        // [4][G]
  unsigned *bar;       // arrival counter, error flag
  int *out_its;
  double *out_rr, *out_dd;
  unsigned long long *trace;  // optional: CTA 0 phase timestamps, [TRACE_IT][2 * 8]
  // TMA streaming: stage size and per-operator switch (rows longer than a stage are
  // read directly from global memory)
  unsigned stage_bytes, xs_bytes;
};

constexpr int TRACE_IT = 16;
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// grid barrier: every CTA adds 1 to a counter that only grows; barrier k completes
// when it reaches k * G.  Bounded wait; returns false when any CTA gave up.
__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned G, unsigned &target,
                                          unsigned long long *tr = nullptr) {
  __syncthreads();
  __shared__ int ok;
  target += G;
  if (threadIdx.x == 0) {
    if (tr) tr[0] = gtimer();
    __threadfence();
    atomicAdd(bar, 1u);
    int good = 1;
    long long spins = 0;
    while (ld_acquire(bar) < target) {
      if (++spins > 64) __nanosleep(32);
      if (spins > (1ll << 25)) {  // ~1-3 s
        atomicExch(bar + 1, 1u);
        good = 0;
        break;
      }
      if ((spins & 1023) == 0 && *(volatile unsigned *)(bar + 1)) {
        good = 0;
        break;
      }
    }
    if (*(volatile unsigned *)(bar + 1)) good = 0;
    ok = good;
    if (tr) tr[1] = gtimer();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double warp_red(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of v, result broadcast to every thread
__device__ __forceinline__ double block_sum(double v, double *sh) {
  v = warp_red(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0;
  int nw = blockDim.x >> 5;
  for (int k = 0; k < nw; ++k) t += sh[k];
  return t;
}

// deterministic sum of the G partials of one slot (same order in every CTA)
__device__ __forceinline__ double reduce_slot(const double *part, int G, double *sh) {
  double v = 0;
  for (int c = threadIdx.x; c < G; c += blockDim.x) v += ldcg(part + c);
  return block_sum(v, sh);
}

template <class T> struct V16;
template <> struct V16<float> { using t = float4; static constexpr int n = 4; };
template <> struct V16<double> { using t = double2; static constexpr int n = 2; };

__device__ __forceinline__ float dot16(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ double dot16(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }

template <class T>
__device__ __forceinline__ T warp_red_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// R padded (16-byte aligned, zero-padded) rows against the staged x, by one warp.
// Every lane issues its loads of a 32*U-vector chunk of all R rows before using
// them (R*U independent 16-byte loads in flight per lane).  Partial sums and the
// warp reduction stay in the operator precision T (the FP64 pipe of this GPU is
// ~1/64 of its FP32 rate).  On return every lane holds all R row sums.
template <class T, int R, bool GLOBAL = true>
__device__ __forceinline__ void rows_dot(const T *A, int64_t ld, int r, int nvalid, const T *xs, T (&out)[R]) {
  using V = typename V16<T>::t;
  constexpr int U = R >= 4 ? 2 : 8;
  const V *x = reinterpret_cast<const V *>(xs);
  int nv = (int)(ld / V16<T>::n);
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < R; ++i) out[i] = 0;
  for (int base = 0; base < nv; base += 32 * U) {
    V va[R][U];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const V *row = reinterpret_cast<const V *>(A + (int64_t)(r + (i < nvalid ? i : 0)) * ld);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int k = base + lane + 32 * u;
        if (k < nv && i < nvalid) va[i][u] = GLOBAL ? __ldg(row + k) : row[k];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int k = base + lane + 32 * u;
      if (k < nv) {
        V xv = x[k];
#pragma unroll
        for (int i = 0; i < R; ++i)
          if (i < nvalid) out[i] += dot16(va[i][u], xv);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) out[i] = warp_red_t(out[i]);
}

// rows [r0, r1) of a patch operator against xs, RW rows per warp; out(r, value) is
// called by lane i of the warp for its i-th row (epilogues run in parallel)
template <int RW, bool GLOBAL = true, class T, class Out>
__device__ __forceinline__ void rows_gemv(const T *A, int ld, int r0, int r1, const T *xs, Out out) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = r0 + RW * warp; r < r1; r += RW * nw) {
    int nvalid = min(RW, r1 - r);
    T v[RW];
    rows_dot<T, RW, GLOBAL>(A, ld, r, nvalid, xs, v);
    T mine = 0;
#pragma unroll
    for (int i = 0; i < RW; ++i)
      if (lane == i) mine = v[i];
    if (lane < nvalid) out(r + lane, (double)mine);
  }
}

// ---------------------------------------------------------------------------
// TMA ring: rows of a contiguous row-major block streamed HBM -> shared memory in
// chunks of whole rows (NS stages in flight), dot products computed from shared.
constexpr int NS = 3;
struct Ring {
  unsigned char *stage;   // NS * bytes
  uint64_t *bar;          // NS mbarriers
  unsigned bytes;
  unsigned long long issued, consumed;
};

// returns false (after setting the error flag and draining its copies) when a
// wait timed out
template <int RW, class T, class Out>
__device__ bool stream_rows(Ring &ring, const T *A, int ld, int r0, int r1, const T *xs, unsigned *errflag,
                            Out out) {
  int nrows = r1 - r0;
  if (nrows <= 0) return true;
  if (ld == 0) {
    for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) out(r, 0.0);
    return true;
  }
  unsigned row_bytes = (unsigned)ld * sizeof(T);
  int rpc = max(1, (int)(ring.bytes / row_bytes));
  int nchunks = (nrows + rpc - 1) / rpc;
  auto issue = [&](int c) {
    int st = (int)(ring.issued % NS);
    if (threadIdx.x == 0) {
      int c0 = c * rpc;
      unsigned bytes = (unsigned)min(rpc, nrows - c0) * row_bytes;
      fence_proxy_async();
      mbar_arrive_expect_tx(ring.bar + st, bytes);
      tma_load_1d(ring.stage + (size_t)st * ring.bytes, A + (int64_t)(r0 + c0) * ld, bytes, ring.bar + st);
    }
    ring.issued++;
  };
  int pre = min(NS, nchunks);
  for (int c = 0; c < pre; ++c) issue(c);
  for (int c = 0; c < nchunks; ++c) {
    int st = (int)(ring.consumed % NS);
    unsigned parity = (unsigned)((ring.consumed / NS) & 1ull);
    bool ok = mbar_wait(ring.bar + st, parity);
    if (__syncthreads_or(!ok)) {  // the same decision in every thread of the CTA
      atomicExch(errflag, 1u);
      // drain the copies still in flight before leaving (bounded)
      for (unsigned long long g = ring.consumed + 1; g < ring.issued; ++g)
        mbar_wait(ring.bar + (g % NS), (unsigned)((g / NS) & 1ull));
      return false;
    }
    ring.consumed++;
    const T *buf = reinterpret_cast<const T *>(ring.stage + (size_t)st * ring.bytes);
    int c0 = c * rpc, cn = min(rpc, nrows - c0);
    rows_gemv<RW, false>(buf, ld, 0, cn, xs, [&](int r, double v) { out(r0 + c0 + r, v); });
    __syncthreads();  // every warp is done with this stage
    if (c + NS < nchunks) issue(c + NS);
  }
  return true;
}

// operator rows of one phase: TMA-streamed (patch operators) or direct (S_c^{-1},
// whose FP64 rows are bound by the FP64 pipe, not by the memory system)
template <int RW, bool TMA, class T, class Out>
__device__ __forceinline__ bool phase_rows(Ring &ring, const T *A, int ld, int r0, int r1, const T *xs,
                                           unsigned *errflag, Out out) {
  if constexpr (TMA) {
    return stream_rows<RW>(ring, A, ld, r0, r1, xs, errflag, out);
  } else {
    rows_gemv<RW, true>(A, ld, r0, r1, xs, out);
    return true;
  }
}

template <class T>
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg(const __grid_constant__ PcgArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ __align__(8) uint64_t ring_bar[NS];
  T *xs = reinterpret_cast<T *>(smem_raw);
  double *ccs = reinterpret_cast<double *>(smem_raw);
  Ring ring{smem_raw + a.xs_bytes, ring_bar, a.stage_bytes, 0ull, 0ull};
  if (threadIdx.x == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(ring_bar + k, 1);
    mbar_fence_init();
  }
  __syncthreads();
  unsigned *errflag = a.bar + 1;
  const int G = gridDim.x, cta = blockIdx.x;
  const int nthr = blockDim.x;
  unsigned target = 0;
  const int64_t lb = a.m * cta / G, le = a.m * (cta + 1) / G;
  const int64_t cb = (int64_t)a.nc * cta / G, ce = (int64_t)a.nc * (cta + 1) / G;
  const double *wd = a.scaled ? a.bt_wd : a.bt_sgn;
  double *part_dd = a.part, *part_rz = a.part + G, *part_pq = a.part + 2 * G, *part_rr = a.part + 3 * G;

  // stage B^T-type gathers of patch s into xs (and into ub for this CTA's rows)
  auto gather = [&](int s, const double *w, int r0, int r1, bool store_ub, auto val) {
    int nbs = a.nb[s], ld = a.ldb[s];
    int64_t b0 = a.bofs[s];
    for (int k = threadIdx.x; k < ld; k += nthr) {
      double acc = 0;
      if (k < nbs) {
        const int32_t *L = a.bt_lam + (b0 + k) * BT_W;
        const double *W = w + (b0 + k) * BT_W;
#pragma unroll
        for (int t = 0; t < BT_W; ++t) {
          int l = L[t];
          if (l >= 0) acc += W[t] * val(l);
        }
        if (store_ub && k >= r0 && k < r1) a.ub[b0 + k] = acc;
      }
      xs[k] = (T)acc;
    }
  };
  auto jumpD = [&](const double *v, int64_t l) {
    double wp = a.lam_wp ? a.lam_wp[l] : 1.0, wm = a.lam_wm ? a.lam_wm[l] : 1.0;
    return wp * ldcg(v + a.lam_qp[l]) - wm * ldcg(v + a.lam_qm[l]);
  };
  auto precond_rows = [&](auto val) -> bool {
    for (int sg = a.bseg_ptr[cta]; sg < a.bseg_ptr[cta + 1]; ++sg) {
      int s = a.bseg_s[sg];
      __syncthreads();
      gather(s, wd, 0, 0, false, val);
      __syncthreads();
      int64_t bo = a.bofs[s];
      if (!phase_rows<4, true>(ring, a.P + a.poff[s], a.ldb[s], a.bseg_r0[sg], a.bseg_r1[sg], xs, errflag,
                         [&](int r, double v) { a.zp[bo + r] = v; }))
        return false;
    }
    return true;
  };

  // ---------------- initial residual r = d, z = M^{-1} d
  double acc = 0;
  for (int64_t l = lb + threadIdx.x; l < le; l += nthr) {
    double dv = a.d[l];
    a.lam[l] = 0.0;
    a.r0[l] = dv;
    acc += dv * dv;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part_dd[cta] = acc;
  if (!a.precond_none && !precond_rows([&](int l) { return ldcg(a.d + l); })) return;
  if (!grid_sync(a.bar, G, target)) return;
  const double dd = reduce_slot(part_dd, G, sh);
  if (cta == 0 && threadIdx.x == 0) *a.out_dd = dd;
  if (!(dd > 0.0)) {
    if (cta == 0 && threadIdx.x == 0) { *a.out_its = 0; *a.out_rr = 0.0; }
    return;
  }
  acc = 0;
  for (int64_t l = lb + threadIdx.x; l < le; l += nthr) {
    double zv = a.precond_none ? a.d[l] : jumpD(a.zp, l);
    a.z[l] = zv;
    acc += a.d[l] * zv;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part_rz[cta] = acc;
  if (!grid_sync(a.bar, G, target)) return;
  double rz_old = reduce_slot(part_rz, G, sh);
  double rr = dd;
  double *rcur = a.r0, *rnxt = a.r1, *pcur = a.p0, *pnxt = a.p1;
  int it = 0;
  for (it = 1; it <= a.max_it; ++it) {
    unsigned long long *tr =
        (a.trace && cta == 0 && it <= TRACE_IT) ? a.trace + (size_t)(it - 1) * 16 : nullptr;
    if (tr && threadIdx.x == 0) tr[14] = gtimer();
    // ---------------- P1: p_new, u = B^T p_new, [F; Psi^T] u
    double beta = 0.0;
    if (it > 1) {
      double rz_new = reduce_slot(part_rz, G, sh);
      beta = rz_new / rz_old;
      rz_old = rz_new;
    }
    for (int64_t l = lb + threadIdx.x; l < le; l += nthr) pnxt[l] = ldcg(a.z + l) + beta * ldcg(pcur + l);
    for (int sg = a.hseg_ptr[cta]; sg < a.hseg_ptr[cta + 1]; ++sg) {
      int s = a.hseg_s[sg], r0 = a.hseg_r0[sg], r1 = a.hseg_r1[sg];
      __syncthreads();
      gather(s, a.bt_sgn, r0, r1, true, [&](int l) { return ldcg(a.z + l) + beta * ldcg(pcur + l); });
      __syncthreads();
      int nbs = a.nb[s];
      int64_t bo = a.bofs[s], po = a.pofs[s];
      if (!phase_rows<4, true>(ring, a.H + a.hoff[s], a.ldb[s], r0, r1, xs, errflag, [&](int r, double v) {
            if (r < nbs) a.zb[bo + r] = v;
            else a.tpi[po + (r - nbs)] = v;
          }))
        return;
    }
    if (!grid_sync(a.bar, G, target, tr ? tr + 0 : nullptr)) return;
    // ---------------- P2: coarse right-hand side, chunk per CTA
    for (int64_t k = cb + threadIdx.x; k < ce; k += nthr) {
      double c = 0;
#pragma unroll
      for (int t = 0; t < CP_W; ++t) {
        int pos = a.cp_pos[k * CP_W + t];
        if (pos >= 0) c -= ldcg(a.tpi + pos);
      }
      a.cc[k] = c;
    }
    if (!grid_sync(a.bar, G, target, tr ? tr + 2 : nullptr)) return;
    // ---------------- P3: q = S_c^{-1} c
    if (ce > cb) {
      for (int k = threadIdx.x; k < a.ldc; k += nthr) ccs[k] = k < a.nc ? ldcg(a.cc + k) : 0.0;
      __syncthreads();
      if (!phase_rows<1, false>(ring, a.Sinv, a.ldc, (int)cb, (int)ce, ccs, errflag,
                         [&](int r, double v) { a.q[r] = v; }))
        return;
    }
    if (!grid_sync(a.bar, G, target, tr ? tr + 4 : nullptr)) return;
    // ---------------- P4: zf = zb - Psi q on the interface rows; (p, F p) = (u, zf)
    acc = 0;
    for (int sg = a.bseg_ptr[cta]; sg < a.bseg_ptr[cta + 1]; ++sg) {
      int s = a.bseg_s[sg];
      int nps = a.np[s], ldq = a.ldp[s];
      __syncthreads();
      const int32_t *pcs = a.pc + a.pofs[s];
      for (int k = threadIdx.x; k < ldq; k += nthr) xs[k] = (T)(k < nps ? ldcg(a.q + pcs[k]) : 0.0);
      __syncthreads();
      int64_t bo = a.bofs[s];
      if (!phase_rows<4, true>(ring, a.Q + a.qoff[s], ldq, a.bseg_r0[sg], a.bseg_r1[sg], xs, errflag,
                         [&](int r, double v) {
                           double zv = ldcg(a.zb + bo + r) - v;
                           a.zf[bo + r] = zv;
                           acc += zv * ldcg(a.ub + bo + r);
                         }))
        return;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part_pq[cta] = acc;
    if (!grid_sync(a.bar, G, target, tr ? tr + 6 : nullptr)) return;
    // ---------------- P5: alpha, owner updates, preconditioner
    double pq = reduce_slot(part_pq, G, sh);
    double alpha = rz_old / pq;
    acc = 0;
    for (int64_t l = lb + threadIdx.x; l < le; l += nthr) {
      double fp = ldcg(a.zf + a.lam_qp[l]) - ldcg(a.zf + a.lam_qm[l]);
      a.lam[l] += alpha * ldcg(pnxt + l);
      double rv = ldcg(rcur + l) - alpha * fp;
      rnxt[l] = rv;
      acc += rv * rv;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part_rr[cta] = acc;
    if (!a.precond_none && !precond_rows([&](int l) {
          return ldcg(rcur + l) - alpha * (ldcg(a.zf + a.lam_qp[l]) - ldcg(a.zf + a.lam_qm[l]));
        }))
      return;
    if (!grid_sync(a.bar, G, target, tr ? tr + 8 : nullptr)) return;
    // ---------------- P6: convergence, z = B_D zp, (r, z)
    rr = reduce_slot(part_rr, G, sh);
    if (!(rr > a.tol2 * dd) || !isfinite(rr)) break;
    acc = 0;
    for (int64_t l = lb + threadIdx.x; l < le; l += nthr) {
      double rv = ldcg(rnxt + l);
      double zv = a.precond_none ? rv : jumpD(a.zp, l);
      a.z[l] = zv;
      acc += rv * zv;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part_rz[cta] = acc;
    if (!grid_sync(a.bar, G, target, tr ? tr + 10 : nullptr)) return;
    double *t = rcur; rcur = rnxt; rnxt = t;
    t = pcur; pcur = pnxt; pnxt = t;
  }
  if (cta == 0 && threadIdx.x == 0) {
    *a.out_its = it > a.max_it ? a.max_it : it;
    *a.out_rr = rr;
  }
}

}  // namespace ieti
