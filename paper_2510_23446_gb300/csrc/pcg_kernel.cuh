// Persistent cooperative dual-primal solve of one defect-correction sweep (Sec. 3-4):
// interior condensation, right-hand side d of the dual problem, PCG on
// F lambda = d (Dirichlet preconditioner, lambda_0 = 0, stop on ||r|| <= tol ||d||)
// and recovery of the patch unknowns, all in one launch.
//
// Per-patch operators (rows padded to 16-byte multiples, streamed HBM -> shared
// memory by 1-D TMA bulk copies through an NS-stage mbarrier ring):
//   IG_s = [W_ii^{-1}; G_s]  (G_s = W_[bp]i W_ii^{-1})  condensation
//   H_s  = [F_s; Psi_s^T]                              dual operator / primal rhs
//   Q_s  = Psi_s                                       primal correction
//   P_s  = S_bb                                        Dirichlet preconditioner
//   GT_s = G_s^T                                       interior recovery
// and the dense FP64 S_c^{-1} (coarse problem).
//
// Phases are separated by grid barriers (monotonic arrival counter; a wait that does
// not complete within ~1-3 s sets an error flag and every CTA returns).  Every
// vector written by another CTA inside the launch is read with ld.global.cg.
//   C   z_i = W_ii^{-1} f_i, g_[bp] = f_[bp] - G f_i                      (kg)
//   D1-D4  d = B (F g_b - Psi S_c^{-1} sum A^T (g_p - Psi^T g_b))         (zf)
//   per iteration: P1 beta, p_new, u = B^T p_new, [F; Psi^T] u; P2 coarse rhs;
//     P3 q = S_c^{-1} c; P4 zf = zb - Psi q, (p, F p) = (u, zf); P5 alpha, owner
//     updates, S_bb (B_D^T r_new); P6 convergence, z = B_D zp, (r, z)
//   R1-R4  v_b = g_b - B^T lambda: a_b = F v_b - Psi q, a_p = q               (kx)
//   R5  a_i = z_i - G^T a_[bp]                                             (kx)
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "tma.cuh"

namespace ieti {

constexpr int PCG_THREADS = 256;
constexpr int BT_W = 3;   // multipliers per interface copy (a DOF shared by at most 4 patches)
constexpr int CP_W = 4;   // copies per coarse DOF
constexpr int NB_W = 4;   // an interface copy and the other copies of its DOF

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
  // interface-copy neighbour lists [NBt][NB_W] (self first, -1 = none) with the
  // coefficients of B_D^T B (ca) and of B^T B_D (cb), and B_D^T r kept in B-space
  const int32_t *nb_idx;
  const double *nb_ca, *nb_cb;
  double *yv0, *yv1;
  // per patch
  const int64_t *kofs, *bofs, *pofs, *hoff, *qoff, *poff, *igoff, *gtoff;
  const int32_t *ni, *nb, *np, *ldb, *ldp, *ldi, *ldg;
  const int32_t *pc;
  const int64_t *p_kept, *b_kept;   // Pi / B position -> kept-space index
  const int32_t *cp_pos;            // [nc][CP_W], -1 = none
  const T *IG, *H, *Q, *P, *GT;
  const double *Sinv;               // FP64 path: S_c^{-1}; mixed path: (hi, lo) FP32 pairs of it
  int64_t nbt;
  // work partitions (per CTA): patch segments of operator rows
  const int32_t *iseg_ptr, *iseg_s, *iseg_r0, *iseg_r1;   // IG rows
  const int32_t *hseg_ptr, *hseg_s, *hseg_r0, *hseg_r1;   // H rows
  const int32_t *bseg_ptr, *bseg_s, *bseg_r0, *bseg_r1;   // interface rows (S_bb)
  const int32_t *qseg_ptr, *qseg_s, *qseg_r0, *qseg_r1;   // interface rows (Psi; the S_bb ones or their own)
  const int32_t *tseg_ptr, *tseg_s, *tseg_r0, *tseg_r1;   // GT rows
  // vectors
  const double *rhs;                // kept space
  double *kg, *kx;                  // kept space: condensed rhs, solution
  double *lam, *p0, *p1, *r0, *r1, *z, *ub, *ub1, *uz, *zb, *zf, *tpi, *cc, *q, *zp;
  double *part;        // [4][G]
  unsigned *bar;       // arrival counter, error flag
  int *out_its;
  double *out_rr, *out_dd;
  unsigned long long *trace;  // optional: CTA 0 phase timestamps, [TRACE_IT][TRACE_SLOTS]
  unsigned stage_bytes, xs_bytes;
  int n_stages;
  float l2_keep_frac;  // > 0: L2 eviction-priority hints on the operator streams
  long long spin_max;  // polls of a grid-barrier wait before it gives up (~1-3 s by default)
  // coarse solve by nested dissection (coarse_nd = 1; else the dense S_c^{-1} rows above).
  // Node p owns the coarse unknowns [k0, k0 + nk) and couples to the ns ancestor
  // unknowns sidx[soff .. soff + ns).  Z_p = [D_p^{-1}; Lbar_p] ((nk + ns) x nk, leading
  // dimension zld) with D_p the node's pivot block after the updates of its subtree and
  // Lbar_p = F_SK D_p^{-1}; Lt_p = Lbar_p^T (nk x ns, ltld).  Forward, by height:
  // f_K = c_K + child updates, q_K = D^{-1} f_K, u_p = f_S + child updates - Lbar f_K.
  // Child updates live in slots: cw per front position of every node (node p's from
  // srcoff[p]), slot w of a position filled by the w-th child contributing there (zero
  // if none); row j of u_p goes to slot dst[uoff[p] + j] of its parent's front.
  // Backward, by depth: q_K -= Lt_p q_S.
  int coarse_nd, nd_cw, nd_H, nd_D, nd_nodes;
  const int32_t *nd_k0, *nd_nk, *nd_ns, *nd_zld, *nd_ltld, *nd_sidx, *nd_dst, *nd_nch;
  const int64_t *nd_zoff, *nd_ltoff, *nd_soff, *nd_uoff, *nd_srcoff;
  const double *nd_Z, *nd_Lt;
  double *nd_slot;
  const int32_t *ndf_ptr, *ndf_s, *ndf_r0, *ndf_r1;   // forward rows per level: ptr [H][G + 1]
  const int32_t *ndb_ptr, *ndb_s, *ndb_r0, *ndb_r1;   // backward rows per level (depth 1 ..): ptr [D][G + 1]
  // nd_flow = 1: the levels wait on per-node completion counters instead of grid barriers
  // (forward: a node's children done; backward: its parent final), nd_done [2][nodes]
  // counting finished segments (targets: solves so far x segments of the node)
  int nd_flow;
  const int32_t *nd_cptr, *nd_cidx, *nd_parent, *nd_nsegf, *nd_nsegb;
  unsigned *nd_done;
};

constexpr int TRACE_IT = 16;
// per traced iteration: [2 ph] end of the work of phase ph, [2 ph + 1] end of its
// barrier wait (ph = 0..5), [14] start of the iteration, and for the streaming phases
// (P1, P3, P4, P5 = sub 0..3) [16 + 3 sub + k]: k = 0 first segment staged, k = 1
// first operator chunk arrived, k = 2 last row done
// nested-dissection level lv of the coarse solve: [32 + 4 lv + k], k = 0 first segment
// staged, 1 first chunk arrived, 2 last row done, 3 end of the level's barrier
constexpr int TRACE_SLOTS = 128;
constexpr int TRACE_ND = 24;
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
// when it reaches k * G.  Bounded wait (spin_max polls); returns false when any CTA
// gave up.
__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned G, unsigned &target, long long spin_max,
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
      if (spins > spin_max) {
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

template <class T>
__device__ __forceinline__ T warp_red_t(T v) {
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
// s + a . b for one 16-byte unit.  FP32: the dot of the unit, then the add (the FP32
// pipe is not the limit of any row kernel).  FP64: two chained FMAs, two FP64
// instructions per unit instead of three (GB300's FP64 pipe bounds the FP64 rows).
__device__ __forceinline__ float fma16(float4 a, float4 b, float s) { return s + dot16(a, b); }
__device__ __forceinline__ double fma16(double2 a, double2 b, double s) { return fma(a.y, b.y, fma(a.x, b.x, s)); }

// R padded (16-byte aligned, zero-padded) rows against the staged x, by one warp.
// Every lane issues its loads of a 32*U-vector chunk of all R rows before using
// them.  Partial sums and the warp reduction stay in the operator precision T (the
// FP64 pipe of this GPU is ~1/64 of its FP32 rate).  Every lane gets all R sums.
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
          if (i < nvalid) out[i] = fma16(va[i][u], xv, out[i]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) out[i] = warp_red_t(out[i]);
}

struct NoPre {
  __device__ double2 operator()(int) const { return make_double2(0.0, 0.0); }
  __device__ double2 operator()(int, int) const { return make_double2(0.0, 0.0); }
};

// segment-completion hook of stream_phase (none by default)
struct NoDone {
  __device__ void operator()(int) const {}
};

// rows [r0, r1) of an operator against xs, RW rows per warp; lane i of the warp
// handles the epilogue of the group's i-th row: pre(r) is loaded before the dot
// products (so its latency overlaps them) and out(r, value, pre) runs after
template <int RW, bool GLOBAL = true, class T, class Out, class Pre = NoPre>
__device__ __forceinline__ void rows_gemv(const T *A, int ld, int r0, int r1, const T *xs, Out out,
                                          Pre pre = Pre()) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = r0 + RW * warp; r < r1; r += RW * nw) {
    int nvalid = min(RW, r1 - r);
    double2 pv = make_double2(0.0, 0.0);
    if (lane < nvalid) pv = pre(r + lane);
    T v[RW];
    rows_dot<T, RW, GLOBAL>(A, ld, r, nvalid, xs, v);
    T mine = 0;
#pragma unroll
    for (int i = 0; i < RW; ++i)
      if (lane == i) mine = v[i];
    if (lane < nvalid) out(r + lane, (double)mine, pv);
  }
}

constexpr int RPC_MAX = 512;  // operator rows per ring chunk at most (their results are staged)

// y[r] = A_r . x for the rows of a chunk in shared memory (row-major, leading
// dimension ld = an odd number of 16-byte units, zero-padded), G lanes per row:
// lane j of a row group sums the 16-byte units j, j + G, ...; the G partial sums are
// combined by log2(G) shuffles.  With the odd row pitch, the eight lanes of a
// shared-memory wavefront read distinct banks both for G = 1 (eight rows) and for
// G >= 8 (one row).
template <class T, int G>
__device__ __noinline__ void chunk_rows_g(const T *A, int ld, int cn, const T *xs, T *y) {
  using V = typename V16<T>::t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sub = lane / G, j = lane % G;
  const int nv = ld / V16<T>::n;
  const V *x = reinterpret_cast<const V *>(xs);
  for (int r0 = warp * (32 / G); r0 < cn; r0 += nw * (32 / G)) {
    const int r = r0 + sub;
    T s = 0;
    if (r < cn) {
      const V *row = reinterpret_cast<const V *>(A + (int64_t)r * ld);
      T s0 = 0, s1 = 0;
      int k = j;
      for (; k + G < nv; k += 2 * G) {
        V a = row[k], b = row[k + G], xa = x[k], xb = x[k + G];
        s0 = fma16(a, xa, s0);
        s1 = fma16(b, xb, s1);
      }
      if (k < nv) s0 = fma16(row[k], x[k], s0);
      s = s0 + s1;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (j == 0 && r < cn) y[r] = s;
  }
}

// y[r] = A_r . x for a chunk of fewer than 16 long rows (more than 32 16-byte units
// each): a warp per row (rows w, w + 8 for cn >= 8), or, for cn < 8, wpr = 8 / cn
// (rounded down to a power of two) warps per row, each on a slice of its units, with
// one exchange of the partial sums through part[] (8 entries) and one CTA barrier.
// Lanes read consecutive 16-byte units: no bank conflicts.
template <class T>
__device__ __noinline__ void chunk_rows_wide(const T *A, int ld, int cn, const T *xs, T *y, T *part) {
  using V = typename V16<T>::t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nv = ld / V16<T>::n;
  const V *x = reinterpret_cast<const V *>(xs);
  int wpr = 1;
  while (wpr * 2 * cn <= nw) wpr *= 2;
  const int rows_per_pass = nw / wpr;
  for (int rb = 0; rb < cn; rb += rows_per_pass) {
    const int r = rb + warp / wpr, j = warp % wpr;
    T s0 = 0, s1 = 0;
    if (r < cn) {
      const V *row = reinterpret_cast<const V *>(A + (int64_t)r * ld);
      const int step = 32 * wpr;
      int k = j * 32 + lane;
      for (; k + step < nv; k += 2 * step) {
        s0 = fma16(row[k], x[k], s0);
        s1 = fma16(row[k + step], x[k + step], s1);
      }
      if (k < nv) s0 = fma16(row[k], x[k], s0);
    }
    const T v = warp_red_t(s0 + s1);
    if (wpr == 1) {
      if (lane == 0 && r < cn) y[r] = v;
    } else {
      if (lane == 0) part[warp] = v;
      __syncthreads();
      if ((int)threadIdx.x < rows_per_pass && rb + (int)threadIdx.x < cn) {
        T t = 0;
        for (int q = 0; q < wpr; ++q) t += part[threadIdx.x * wpr + q];
        y[rb + threadIdx.x] = t;
      }
      __syncthreads();
    }
  }
}

// Double-FP32 rows: entries stored as (hi, lo) FP32 pairs of FP64 values, dotted with
// staged (hi, lo) pairs by exact FP32 products (TwoProd by FMA) accumulated with TwoSum;
// the cross terms hi*lo + lo*hi go into the compensation, lo*lo (2^-48) is dropped.
// About 2^-45 of sum |a x| per dot, on the FP32 pipe (GB300's FP64 pipe is ~1/64 of it).
// One 16-byte unit = two pairs.
__device__ __forceinline__ void df_acc(float &S, float &c, float4 a, float4 x) {
  const float p0 = a.x * x.x, e0 = fmaf(a.x, x.x, -p0), t0 = fmaf(a.x, x.y, a.y * x.x);
  const float p1 = a.z * x.z, e1 = fmaf(a.z, x.z, -p1), t1 = fmaf(a.z, x.w, a.w * x.z);
  float s = S + p0, bb = s - S;
  c += ((S - (s - bb)) + (p0 - bb)) + (e0 + t0);
  S = s;
  s = S + p1;
  bb = s - S;
  c += ((S - (s - bb)) + (p1 - bb)) + (e1 + t1);
  S = s;
}

// (S, c) += (S2, c2) for double-FP32 partial sums: TwoSum of the leading parts, the
// compensations and the rounding error of that sum into c (FP32 only)
__device__ __forceinline__ void df_add(float &S, float &c, float S2, float c2) {
  const float s = S + S2, bb = s - S;
  c = (c + c2) + ((S - (s - bb)) + (S2 - bb));
  S = s;
}

// y[r] = A_r . x (FP64 results) for the rows of a chunk of (hi, lo) pairs, G lanes per
// row, NACC accumulator pairs per lane; ld in pairs (even).  The lane partials are
// combined in double-FP32 (df_add, shuffles of FP32 pairs): one FP64 conversion per
// row, so the FP64 pipe (a small fraction of the FP32 rate on this part) stays idle.
template <int G, int NACC>
__device__ __forceinline__ void chunk_rows_df(const float2 *A, int ld, int cn, const float2 *xs, double *y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sub = lane / G, j = lane % G;
  const int nv = ld / 2;
  const float4 *x = reinterpret_cast<const float4 *>(xs);
  for (int r0 = warp * (32 / G); r0 < cn; r0 += nw * (32 / G)) {
    const int r = r0 + sub;
    float S[NACC], c[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) S[i] = c[i] = 0.f;
    if (r < cn) {
      const float4 *row = reinterpret_cast<const float4 *>(A + (int64_t)r * ld);
      int k = j;
      for (; k + (NACC - 1) * G < nv; k += NACC * G) {
#pragma unroll
        for (int i = 0; i < NACC; ++i) df_acc(S[i], c[i], row[k + i * G], x[k + i * G]);
      }
      for (; k < nv; k += G) df_acc(S[0], c[0], row[k], x[k]);
    }
#pragma unroll
    for (int i = 1; i < NACC; ++i) df_add(S[0], c[0], S[i], c[i]);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const float S2 = __shfl_xor_sync(0xffffffffu, S[0], o), c2 = __shfl_xor_sync(0xffffffffu, c[0], o);
      df_add(S[0], c[0], S2, c2);
    }
    if (j == 0 && r < cn) y[r] = (double)S[0] + (double)c[0];
  }
}

// the same for chunks of fewer than 8 long rows of (hi, lo) pairs: warps per row as in
// chunk_rows_wide, the warps' double-FP32 partials exchanged through part (FP32 pairs)
__device__ __forceinline__ void chunk_rows_df_wide(const float2 *A, int ld, int cn, const float2 *xs, double *y,
                                                float2 *part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nv = ld / 2;
  const float4 *x = reinterpret_cast<const float4 *>(xs);
  int wpr = 1;
  while (wpr * 2 * cn <= nw) wpr *= 2;
  const int rows_per_pass = nw / wpr;
  for (int rb = 0; rb < cn; rb += rows_per_pass) {
    const int r = rb + warp / wpr, j = warp % wpr;
    float S0 = 0.f, c0 = 0.f, S1 = 0.f, c1 = 0.f;
    if (r < cn) {
      const float4 *row = reinterpret_cast<const float4 *>(A + (int64_t)r * ld);
      const int step = 32 * wpr;
      int k = j * 32 + lane;
      for (; k + step < nv; k += 2 * step) {
        df_acc(S0, c0, row[k], x[k]);
        df_acc(S1, c1, row[k + step], x[k + step]);
      }
      if (k < nv) df_acc(S0, c0, row[k], x[k]);
    }
    df_add(S0, c0, S1, c1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float S2 = __shfl_xor_sync(0xffffffffu, S0, o), c2 = __shfl_xor_sync(0xffffffffu, c0, o);
      df_add(S0, c0, S2, c2);
    }
    if (wpr == 1) {
      if (lane == 0 && r < cn) y[r] = (double)S0 + (double)c0;
    } else {
      if (lane == 0) part[warp] = make_float2(S0, c0);
      __syncthreads();
      if ((int)threadIdx.x < rows_per_pass && rb + (int)threadIdx.x < cn) {
        float S = 0.f, c = 0.f;
        for (int q = 0; q < wpr; ++q) {
          const float2 t = part[threadIdx.x * wpr + q];
          df_add(S, c, t.x, t.y);
        }
        y[rb + threadIdx.x] = (double)S + (double)c;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// TMA ring.  The operator rows a CTA multiplies in a phase are fixed by the static
// partition, independent of the iteration's vectors, so they are streamed HBM ->
// shared memory in chunks of whole rows through an ns-stage mbarrier ring, and the
// first chunks of the NEXT phase are issued before the grid barrier that ends the
// current one (they arrive while the CTA waits).
constexpr int NS_MAX = 6;
struct Ring {
  unsigned char *stage;   // ns * bytes
  uint64_t *bar;          // ns mbarriers
  unsigned bytes;
  int ns;
  unsigned long long issued, consumed;
};

// the rows of one operator a CTA processes in one phase: segments (patch s, rows
// [r0, r1)) of row-major blocks at base + off[s] with leading dimension ld[s];
// single-segment form (s = 0, rows [r0s, r1s), off 0, ld lds) when seg_s is null
template <class E>
struct OpRows {
  const E *base;
  const int64_t *off;
  const int32_t *ld;
  const int32_t *seg_s, *seg_r0, *seg_r1;
  int sb, se;
  int r0s, r1s, lds;
  uint64_t policy;  // L2 eviction policy of the TMA loads (used when hint != 0)
  int hint;
  __device__ int nseg() const { return seg_s ? se - sb : (r1s > r0s ? 1 : 0); }
  __device__ void seg(int k, int &s, int &r0, int &r1, int &l, const E *&A) const {
    if (seg_s) {
      s = seg_s[sb + k]; r0 = seg_r0[sb + k]; r1 = seg_r1[sb + k]; l = ld[s]; A = base + off[s];
    } else {
      s = 0; r0 = r0s; r1 = r1s; l = lds; A = base;
    }
  }
};

// producer cursor over the chunks of an OpRows (uniform across the CTA)
struct Cursor {
  int seg = 0, chunk = 0, issued = 0;
};

// whole rows per chunk; from 32 rows on a multiple of 32, so that the 8 warps of a
// CTA get the same number of 4-row groups from every chunk
template <class E>
__device__ __forceinline__ int rows_per_chunk(const Ring &ring, int ld) {
  unsigned rb = (unsigned)ld * sizeof(E);
  if (rb == 0) return 1 << 30;
  int r = min((int)(ring.bytes / rb), RPC_MAX);
  return r >= 32 ? r & ~31 : max(1, r);
}

// issue the next chunk of `op` (if any) into the next ring stage; returns false at the end
template <class E>
__device__ bool issue_next(Ring &ring, const OpRows<E> &op, Cursor &cur) {
  int nseg = op.nseg();
  while (cur.seg < nseg) {
    int s, r0, r1, ld;
    const E *A;
    op.seg(cur.seg, s, r0, r1, ld, A);
    int rpc = rows_per_chunk<E>(ring, ld);
    int c0 = cur.chunk * rpc;
    if (ld == 0 || r0 + c0 >= r1) {
      cur.seg++;
      cur.chunk = 0;
      continue;
    }
    int st = (int)(ring.issued % ring.ns);
    if (threadIdx.x == 0) {
      unsigned bytes = (unsigned)min(rpc, r1 - r0 - c0) * (unsigned)ld * sizeof(E);
      fence_proxy_async();
      mbar_arrive_expect_tx(ring.bar + st, bytes);
      if (op.hint)
        tma_load_1d_hint(ring.stage + (size_t)st * ring.bytes, A + (int64_t)(r0 + c0) * ld, bytes, ring.bar + st,
                         op.policy);
      else
        tma_load_1d(ring.stage + (size_t)st * ring.bytes, A + (int64_t)(r0 + c0) * ld, bytes, ring.bar + st);
    }
    ring.issued++;
    cur.chunk++;
    cur.issued++;
    return true;
  }
  return false;
}

// issue up to ns chunks of the next phase's operator rows (the ring is empty here)
template <class E>
__device__ __forceinline__ Cursor prefetch(Ring &ring, const OpRows<E> &op) {
  Cursor cur;
  for (int k = 0; k < ring.ns; ++k)
    if (!issue_next(ring, op, cur)) break;
  return cur;
}

// stream every row of `op` through the ring (continuing cursor `cur`, whose first
// chunks may have been prefetched): before the first chunk of each segment,
// stage(s, r0, r1) runs with every thread of the CTA; out(s, r, value, pre) per row.
// Returns false (after setting the error flag and draining) when a wait timed out.
// DF: the rows hold (hi, lo) FP32 pairs (E = double only sizes them), xs holds staged
// pairs, y receives FP64 results (double-FP32 row kernels)
// done(s) runs with every thread of the CTA once all rows of the CTA's segment of s
// are written (after a CTA barrier)
template <int RW, class E, bool DF = false, class Stage, class Out, class Pre = NoPre, class Done = NoDone>
__device__ bool stream_phase(Ring &ring, const OpRows<E> &op, Cursor &cur, const E *xs, E *y, unsigned *errflag,
                             Stage stage, Out out, Pre pre = Pre(), unsigned long long *ts = nullptr,
                             Done done = Done()) {
  constexpr bool kDone = !std::is_same<Done, NoDone>::value;
  while (cur.issued - 0 < ring.ns && issue_next(ring, op, cur)) {
  }
  int nseg = op.nseg();
  int prev_s = -1;
  for (int k = 0; k < nseg; ++k) {
    int s, r0, r1, ld;
    const E *A;
    op.seg(k, s, r0, r1, ld, A);
    __syncthreads();
    if constexpr (kDone) {
      if (prev_s >= 0) done(prev_s);
      prev_s = s;
    }
    stage(s, r0, r1);
    __syncthreads();
    if (ts && k == 0 && threadIdx.x == 0) ts[0] = gtimer();
    if (ld == 0) {
      for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) out(s, r, 0.0, pre(s, r));
      continue;
    }
    int rpc = rows_per_chunk<E>(ring, ld);
    for (int c0 = 0; r0 + c0 < r1; c0 += rpc) {
      int st = (int)(ring.consumed % ring.ns);
      unsigned parity = (unsigned)((ring.consumed / ring.ns) & 1ull);
      bool ok = mbar_wait(ring.bar + st, parity);
      if (__syncthreads_or(!ok)) {  // the same decision in every thread of the CTA
        atomicExch(errflag, 1u);
        for (unsigned long long g = ring.consumed + 1; g < ring.issued; ++g)
          mbar_wait(ring.bar + (g % ring.ns), (unsigned)((g / ring.ns) & 1ull));
        ring.consumed = ring.issued;
        return false;
      }
      if (ts && k == 0 && c0 == 0 && threadIdx.x == 0) ts[1] = gtimer();
      ring.consumed++;
      const E *buf = reinterpret_cast<const E *>(ring.stage + (size_t)st * ring.bytes);
      const int cn = min(rpc, r1 - r0 - c0), base_r = r0 + c0;
      // row kernel per row length and operator precision (measured on the c2
      // workload): short rows one per lane; long FP64 rows 8 lanes per row; long
      // FP32 rows RW rows per warp; chunks of fewer than 16 long rows (wide patches:
      // a stage holds a few rows) spread over the whole CTA
      const int nv = ld / V16<E>::n;
      const int split = nv <= 32 ? 1 : (cn < 16 ? 2 : (sizeof(E) == 8 ? 8 : 0));
      // epilogue inputs of the chunk's rows (one thread per row, at most two rows per
      // thread: RPC_MAX = 2 x 256), loaded before the row kernel so that their latency
      // overlaps it
      double2 pv[RPC_MAX / PCG_THREADS];
      if (DF || split) {
#pragma unroll
        for (int i = 0; i < RPC_MAX / PCG_THREADS; ++i) {
          const int r = threadIdx.x + i * PCG_THREADS;
          if (r < cn) pv[i] = pre(s, base_r + r);
        }
      }
      if constexpr (DF) {
        static_assert(sizeof(E) == 8, "double-FP32 rows are sized as 8-byte entries");
        double *yc = reinterpret_cast<double *>(y) + (ring.consumed & 1ull) * RPC_MAX;
        const float2 *ap = reinterpret_cast<const float2 *>(buf);
        const float2 *xp = reinterpret_cast<const float2 *>(xs);
        // lanes per row by row length (about 10 to 20 16-byte units per lane; measured
        // on shared-memory chunks of 13 to 81 rows); fewer than 8 long rows: warps per row
        if (nv <= 32) chunk_rows_df<1, 2>(ap, ld, cn, xp, yc);
        else if (cn < 8 && nv > 160)
          chunk_rows_df_wide(ap, ld, cn, xp, yc, reinterpret_cast<float2 *>(yc + RPC_MAX / 2));
        else if (nv <= 80) chunk_rows_df<4, 2>(ap, ld, cn, xp, yc);
        else if (nv <= 160) chunk_rows_df<8, 4>(ap, ld, cn, xp, yc);
        else if (nv <= 320) chunk_rows_df<16, 2>(ap, ld, cn, xp, yc);
        else chunk_rows_df<32, 2>(ap, ld, cn, xp, yc);
        __syncthreads();
        issue_next(ring, op, cur);
#pragma unroll
        for (int i = 0; i < RPC_MAX / PCG_THREADS; ++i) {
          const int r = threadIdx.x + i * PCG_THREADS;
          if (r < cn) out(s, base_r + r, yc[r], pv[i]);
        }
      } else if (split) {
        // row results into y (two buffers: the epilogues of the previous chunk may
        // still read the other one), then one thread per row
        E *yc = y + (ring.consumed & 1ull) * RPC_MAX;
        if (split == 1) chunk_rows_g<E, 1>(buf, ld, cn, xs, yc);
        else if (split == 8) chunk_rows_g<E, 8>(buf, ld, cn, xs, yc);
        else chunk_rows_wide<E>(buf, ld, cn, xs, yc, yc + RPC_MAX / 2);
        __syncthreads();  // every warp is done with this stage; yc is complete
        issue_next(ring, op, cur);
#pragma unroll
        for (int i = 0; i < RPC_MAX / PCG_THREADS; ++i) {
          const int r = threadIdx.x + i * PCG_THREADS;
          if (r < cn) out(s, base_r + r, (double)yc[r], pv[i]);
        }
      } else {
        // long rows: RW rows per warp, lane i of the group runs row i's epilogue
        rows_gemv<RW, false>(buf, ld, 0, cn, xs,
                             [&](int r, double v, double2 pv) { out(s, base_r + r, v, pv); },
                             [&](int r) { return pre(s, base_r + r); });
        __syncthreads();  // every warp is done with this stage
        issue_next(ring, op, cur);
      }
    }
  }
  if (ts && threadIdx.x == 0) ts[2] = gtimer();
  if constexpr (kDone) {
    if (prev_s >= 0) {
      __syncthreads();
      done(prev_s);
    }
  }
  return true;
}

// ND: the coarse solve by nested dissection (a separate instantiation, so that the
// dense-coarse kernel carries none of its code or registers)
template <class T, bool ND>
__global__ void __launch_bounds__(PCG_THREADS, 1) k_ddsolve(const __grid_constant__ PcgArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sh[32];
  // the coarse rows (FP64, or double-FP32 pairs in the mixed path) stage FP64 results too
  using YB = typename std::conditional<ND || sizeof(T) == 4, double, T>::type;
  __shared__ __align__(16) YB ybuf_raw[2 * RPC_MAX];  // row results of the last two chunks
  T *ybuf = reinterpret_cast<T *>(ybuf_raw);
  __shared__ __align__(8) uint64_t ring_bar[NS_MAX];
  T *xs = reinterpret_cast<T *>(smem_raw);
  double *ccs = reinterpret_cast<double *>(smem_raw);
  Ring ring{smem_raw + a.xs_bytes, ring_bar, a.stage_bytes, a.n_stages, 0ull, 0ull};
  if (threadIdx.x == 0) {
    for (int k = 0; k < a.n_stages; ++k) mbar_init(ring_bar + k, 1);
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

  // the operator rows of each phase (static per CTA)
  // L2 hints (l2_keep_frac > 0): the per-iteration operators (H, Psi, S_bb, coarse) are
  // re-read every iteration, a fraction of their lines is kept in L2; the per-sweep
  // operators (IG, GT) stream through
  const int hint = a.l2_keep_frac > 0.f;
  const uint64_t pk = hint ? l2_policy_keep(a.l2_keep_frac) : 0ull, ps = hint ? l2_policy_stream() : 0ull;
  const OpRows<T> opIG{a.IG, a.igoff, a.ldi, a.iseg_s, a.iseg_r0, a.iseg_r1, a.iseg_ptr[cta], a.iseg_ptr[cta + 1],
                       0, 0, 0, ps, hint};
  const OpRows<T> opH{a.H, a.hoff, a.ldb, a.hseg_s, a.hseg_r0, a.hseg_r1, a.hseg_ptr[cta], a.hseg_ptr[cta + 1],
                      0, 0, 0, pk, hint};
  const OpRows<T> opQ{a.Q, a.qoff, a.ldp, a.qseg_s, a.qseg_r0, a.qseg_r1, a.qseg_ptr[cta], a.qseg_ptr[cta + 1],
                      0, 0, 0, pk, hint};
  const OpRows<T> opP{a.P, a.poff, a.ldb, a.bseg_s, a.bseg_r0, a.bseg_r1, a.bseg_ptr[cta], a.bseg_ptr[cta + 1],
                      0, 0, 0, pk, hint};
  const OpRows<T> opGT{a.GT, a.gtoff, a.ldg, a.tseg_s, a.tseg_r0, a.tseg_r1, a.tseg_ptr[cta], a.tseg_ptr[cta + 1],
                       0, 0, 0, ps, hint};
  const OpRows<double> opS{a.Sinv, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, (int)cb, (int)ce, a.ldc,
                           pk, hint};
  // nested-dissection levels: 0 .. H-1 forward (Z rows), H .. H+D-2 backward (Lt rows, depth 1 ..)
  auto nd_op = [&](int lv) {
    if (lv < a.nd_H) {
      const int32_t *pp = a.ndf_ptr + (size_t)lv * (G + 1);
      return OpRows<double>{a.nd_Z, a.nd_zoff, a.nd_zld, a.ndf_s, a.ndf_r0, a.ndf_r1, pp[cta], pp[cta + 1],
                            0, 0, 0, pk, hint};
    }
    const int32_t *pp = a.ndb_ptr + (size_t)(lv - a.nd_H) * (G + 1);
    return OpRows<double>{a.nd_Lt, a.nd_ltoff, a.nd_ltld, a.ndb_s, a.ndb_r0, a.ndb_r1, pp[cta], pp[cta + 1],
                          0, 0, 0, pk, hint};
  };
  const int nd_levels = ND ? a.nd_H + max(a.nd_D - 1, 0) : 0;
  // the first coarse phase's rows (prefetched before the barrier that precedes it)
  auto coarse_first = [&]() {
    if constexpr (ND) return nd_op(0);
    else return opS;
  };

  // stage x_s[k] = f(k) (k < n), zero-padded to ld
  auto stage = [&](int n, int ld, auto f) {
    for (int k = threadIdx.x; k < ld; k += nthr) xs[k] = (T)(k < n ? f(k) : 0.0);
  };
  // stage u_s = B^T-type gather of patch s (ELL lists); keep it in ub for rows [r0, r1)
  auto gather = [&](int s, const double *w, int r0, int r1, double *store, auto val) {
    int nbs = a.nb[s], ld = a.ldb[s];
    int64_t b0 = a.bofs[s];
    constexpr int KP = 4;  // entries per thread per round, loads issued together
    for (int kb = threadIdx.x; kb < ld; kb += KP * nthr) {
      int lidx[KP][BT_W];
#pragma unroll
      for (int u = 0; u < KP; ++u) {
        int k = kb + u * nthr;
#pragma unroll
        for (int t = 0; t < BT_W; ++t) lidx[u][t] = (k < nbs) ? a.bt_lam[(b0 + k) * BT_W + t] : -1;
      }
      double vals[KP][BT_W];
#pragma unroll
      for (int u = 0; u < KP; ++u)
#pragma unroll
        for (int t = 0; t < BT_W; ++t) vals[u][t] = lidx[u][t] >= 0 ? val(lidx[u][t]) : 0.0;
#pragma unroll
      for (int u = 0; u < KP; ++u) {
        int k = kb + u * nthr;
        if (k >= ld) continue;
        double acc = 0;
        if (k < nbs) {
#pragma unroll
          for (int t = 0; t < BT_W; ++t)
            if (lidx[u][t] >= 0) acc += w[(b0 + k) * BT_W + t] * vals[u][t];
          if (store && k >= r0 && k < r1) store[b0 + k] = acc;
        }
        xs[k] = (T)acc;
      }
    }
  };
  auto jumpD = [&](const double *v, int64_t l) {
    double wp = a.lam_wp ? a.lam_wp[l] : 1.0, wm = a.lam_wm ? a.lam_wm[l] : 1.0;
    return wp * ldcg(v + a.lam_qp[l]) - wm * ldcg(v + a.lam_qm[l]);
  };
  auto jump = [&](const double *v, int64_t l) { return ldcg(v + a.lam_qp[l]) - ldcg(v + a.lam_qm[l]); };
  Cursor cur;  // producer cursor of the phase about to run (possibly prefetched)
  double *ub_old = a.ub1, *ub_new = a.ub;  // B^T p of the previous / current iteration
  double *yv_old = a.yv0, *yv_new = a.yv1;  // B_D^T r of the current / next iterate
  unsigned long long *tsub = nullptr;  // sub-phase timestamps of the traced iteration (or null)
  auto tsp = [&](int k) { return tsub ? tsub + 3 * k : nullptr; };
  // a barrier that gave up ends the launch: first the chunks this CTA still has in
  // flight into its shared memory are waited for (bounded), then every CTA returns
  auto sync = [&](unsigned long long *tr) {
    if (grid_sync(a.bar, G, target, a.spin_max, tr)) return true;
    if (threadIdx.x == 0)
      for (unsigned long long g = ring.consumed; g < ring.issued; ++g)
        mbar_wait(ring.bar + (g % ring.ns), (unsigned)((g / ring.ns) & 1ull));
    ring.consumed = ring.issued;
    __syncthreads();
    return false;
  };
  // H phase: [F; Psi^T] u_s -> zb, tpi, with a staging functor for u_s
  auto h_phase = [&](auto stage_u) -> bool {
    return stream_phase<4>(ring, opH, cur, xs, ybuf, errflag, [&](int s, int r0, int r1) { stage_u(s, r0, r1); },
                           [&](int s, int r, double v, double2) {
                             int nbs = a.nb[s];
                             if (r < nbs) a.zb[a.bofs[s] + r] = v;
                             else a.tpi[a.pofs[s] + (r - nbs)] = v;
                           },
                           NoPre(), tsp(0));
  };
  // coarse right-hand side c = sum_copies (g_p - tpi), chunk per CTA
  auto coarse_rhs = [&](bool with_g) {
    for (int64_t k = cb + threadIdx.x; k < ce; k += nthr) {
      double c = 0;
#pragma unroll
      for (int t = 0; t < CP_W; ++t) {
        int pos = a.cp_pos[k * CP_W + t];
        if (pos >= 0) c += (with_g ? ldcg(a.kg + a.p_kept[pos]) : 0.0) - ldcg(a.tpi + pos);
      }
      a.cc[k] = c;
    }
  };
  // the node of the coarse-level segment being processed (set by the stage functors,
  // read by the row epilogues of the segment)
  int nd_snk = 0, nd_sk0 = 0, nd_snch = 0;
  int64_t nd_sbase = 0, nd_suoff = 0;
  auto nd_seg = [&](int p) {
    nd_snk = a.nd_nk[p];
    nd_sk0 = a.nd_k0[p];
    nd_snch = a.nd_nch[p];
    nd_sbase = a.nd_srcoff[p];
    nd_suoff = a.nd_uoff[p];
  };
  // the child updates of front position i of the current node (the sum of its slots)
  auto nd_slots = [&](int i) -> double {
    if (nd_snch == 0) return 0.0;  // a leaf: no child updates
    const double *sl = a.nd_slot + nd_sbase + (int64_t)i * a.nd_cw;
    if (a.nd_cw == 2) {
      const double2 v = __ldcg(reinterpret_cast<const double2 *>(sl));
      return v.x + v.y;
    }
    double v = 0.0;
    for (int w = 0; w < a.nd_cw; ++w) v += ldcg(sl + w);
    return v;
  };
  // nested-dissection solve q = S_c^{-1} c: one phase per level, a grid barrier between
  // levels; the next level's rows are issued before the barrier
  // the mixed path's blocks are (hi, lo) FP32 pairs (double-FP32 rows), the FP64 path's FP64
  constexpr bool NDF = sizeof(T) == 4;
  unsigned nd_epoch = 0;  // coarse solves of this launch so far (the same in every CTA)
  // bounded wait of thread 0 until *ctr reaches target, then a CTA barrier
  auto nd_wait = [&](const unsigned *ctr, unsigned target) {
    if (threadIdx.x == 0) {
      long long spins = 0;
      while (ld_acquire(ctr) < target) {
        if (++spins > 64) __nanosleep(32);
        if (spins > a.spin_max) {
          atomicExch(errflag, 1u);
          break;
        }
        if ((spins & 1023) == 0 && *(volatile unsigned *)errflag) break;
      }
    }
    __syncthreads();
  };
  auto nd_signal = [&](unsigned *ctr) {
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(ctr, 1u);
    }
  };
  // counter of node p that marks q_K final: its backward rows if it has any, else its forward rows
  auto nd_final = [&](int p, const unsigned *&ctr, unsigned &target) {
    if (a.nd_nsegb[p] > 0) {
      ctr = a.nd_done + a.nd_nodes + p;
      target = nd_epoch * (unsigned)a.nd_nsegb[p];
    } else {
      ctr = a.nd_done + p;
      target = nd_epoch * (unsigned)a.nd_nsegf[p];
    }
  };
  auto coarse_solve_nd = [&]() -> bool {
    ++nd_epoch;
    double *xd = reinterpret_cast<double *>(smem_raw);
    float2 *xp = reinterpret_cast<float2 *>(smem_raw);
    double *yd = reinterpret_cast<double *>(ybuf_raw);
    auto put = [&](int k, double v) {
      if constexpr (NDF) {
        const float hi = (float)v;
        xp[k] = make_float2(hi, (float)(v - (double)hi));
      } else {
        xd[k] = v;
      }
    };
    for (int lv = 0; lv < nd_levels; ++lv) {
      const OpRows<double> op = nd_op(lv);
      bool ok;
      if (lv < a.nd_H) {
        auto stage_f = [&](int p, int, int) {
          if (a.nd_flow)
            for (int k = a.nd_cptr[p]; k < a.nd_cptr[p + 1]; ++k) {
              const int ch = a.nd_cidx[k];
              nd_wait(a.nd_done + ch, nd_epoch * (unsigned)a.nd_nsegf[ch]);
            }
          nd_seg(p);
          const int nk = nd_snk, ld = a.nd_zld[p];
          // f_K: four positions per thread and round, their loads issued together
          for (int kb = threadIdx.x; kb < ld; kb += 4 * nthr) {
            double f[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int k = kb + u * nthr;
              f[u] = k < nk ? ldcg(a.cc + nd_sk0 + k) + nd_slots(k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (kb + u * nthr < ld) put(kb + u * nthr, f[u]);
          }
        };
        auto out_f = [&](int, int r, double v, double2 pv) {
          if (r < nd_snk) a.q[nd_sk0 + r] = v;
          else a.nd_slot[(int64_t)pv.y] = pv.x - v;
        };
        // S rows: the child updates of the position and the slot of the row in the parent
        auto pre_f = [&](int, int r) {
          return r >= nd_snk ? make_double2(nd_slots(r), (double)a.nd_dst[nd_suoff + (r - nd_snk)])
                             : make_double2(0.0, 0.0);
        };
        unsigned long long *tl = (tsub && lv < TRACE_ND) ? tsub + 16 + 4 * lv : nullptr;
        if (a.nd_flow)
          ok = stream_phase<4, double, NDF>(ring, op, cur, xd, yd, errflag, stage_f, out_f, pre_f, tl,
                                            [&](int p) { nd_signal(a.nd_done + p); });
        else
          ok = stream_phase<4, double, NDF>(ring, op, cur, xd, yd, errflag, stage_f, out_f, pre_f, tl);
      } else {
        auto stage_b = [&](int p, int, int) {
          if (a.nd_flow) {
            const unsigned *ctr;
            unsigned target;
            nd_final(a.nd_parent[p], ctr, target);
            nd_wait(ctr, target);
          }
          nd_seg(p);
          const int ns = a.nd_ns[p], ld = a.nd_ltld[p];
          const int32_t *si = a.nd_sidx + a.nd_soff[p];
          // q_S: four positions per thread and round (the index loads, then the values)
          for (int kb = threadIdx.x; kb < ld; kb += 4 * nthr) {
            int idx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) idx[u] = kb + u * nthr < ns ? si[kb + u * nthr] : -1;
            double f[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) f[u] = idx[u] >= 0 ? ldcg(a.q + idx[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (kb + u * nthr < ld) put(kb + u * nthr, f[u]);
          }
        };
        auto out_b = [&](int, int r, double v, double2 pv) { a.q[nd_sk0 + r] = pv.x - v; };
        auto pre_b = [&](int, int r) { return make_double2(ldcg(a.q + nd_sk0 + r), 0.0); };
        unsigned long long *tl = (tsub && lv < TRACE_ND) ? tsub + 16 + 4 * lv : nullptr;
        if (a.nd_flow)
          ok = stream_phase<4, double, NDF>(ring, op, cur, xd, yd, errflag, stage_b, out_b, pre_b, tl,
                                            [&](int p) { nd_signal(a.nd_done + a.nd_nodes + p); });
        else
          ok = stream_phase<4, double, NDF>(ring, op, cur, xd, yd, errflag, stage_b, out_b, pre_b, tl);
      }
      if (!ok) return false;
      if (lv + 1 < nd_levels) {
        cur = prefetch(ring, nd_op(lv + 1));
        if (!a.nd_flow && !sync(nullptr)) return false;
      }
      if (tsub && threadIdx.x == 0 && lv < TRACE_ND) tsub[16 + 4 * lv + 3] = gtimer();  // tsub = trace row + 16
    }
    return true;
  };
  auto coarse_solve = [&]() -> bool {
    if constexpr (ND) {
      return coarse_solve_nd();
    } else if constexpr (sizeof(T) == 8) {
      return stream_phase<1>(ring, opS, cur, ccs, ybuf, errflag,
                             [&](int, int, int) {
                               for (int k = threadIdx.x; k < a.ldc; k += nthr)
                                 ccs[k] = k < a.nc ? ldcg(a.cc + k) : 0.0;
                             },
                             [&](int, int r, double v, double2) { a.q[r] = v; }, NoPre(), tsp(1));
    } else {
      // rows of (hi, lo) pairs, streamed as 8-byte entries, through the double-FP32 row
      // kernels of the ring loop
      float2 *xp = reinterpret_cast<float2 *>(smem_raw);
      return stream_phase<4, double, true>(ring, opS, cur, reinterpret_cast<const double *>(smem_raw),
                                           reinterpret_cast<double *>(ybuf_raw), errflag,
                                           [&](int, int, int) {
                                             for (int k = threadIdx.x; k < a.ldc; k += nthr) {
                                               const double c = k < a.nc ? ldcg(a.cc + k) : 0.0;
                                               const float hi = (float)c;
                                               xp[k] = make_float2(hi, (float)(c - (double)hi));
                                             }
                                           },
                                           [&](int, int r, double v, double2) { a.q[r] = v; }, NoPre(), tsp(1));
    }
  };
  // zf = zb - Psi q on the interface rows; out(global B index, zf, ub)
  auto psi_phase = [&](auto out) -> bool {
    return stream_phase<4>(
        ring, opQ, cur, xs, ybuf, errflag,
        [&](int s, int, int) {
          const int32_t *pcs = a.pc + a.pofs[s];
          stage(a.np[s], a.ldp[s], [&](int k) { return ldcg(a.q + pcs[k]); });
        },
        [&](int s, int r, double v, double2 pv) { out(a.bofs[s] + r, pv.x - v, pv.y); },
        [&](int s, int r) {
          int64_t q = a.bofs[s] + r;
          return make_double2(ldcg(a.zb + q), ldcg(ub_new + q));
        },
        tsp(2));
  };
  // S_bb rows against B_D^T r staged by gathering val(l) over the multipliers of each
  // copy; the segment owner keeps B_D^T r (store, B-space) for the next iteration
  auto precond_rows = [&](double *store, auto val) -> bool {
    return stream_phase<4>(ring, opP, cur, xs, ybuf, errflag,
                           [&](int s, int r0, int r1) { gather(s, wd, r0, r1, store, val); },
                           [&](int s, int r, double v, double2) { a.zp[a.bofs[s] + r] = v; }, NoPre(), tsp(3));
  };
  // the same with B_D^T r_new = B_D^T r_cur - alpha B_D^T B zf staged from the kept
  // B-space copy yo and the neighbour lists (two dependent loads instead of three)
  auto precond_rows_y = [&](double alpha, const double *yo, double *yn) -> bool {
    return stream_phase<4>(
        ring, opP, cur, xs, ybuf, errflag,
        [&](int s, int r0, int r1) {
          const int nbs = a.nb[s], ld = a.ldb[s];
          const int64_t b0 = a.bofs[s];
          for (int k = threadIdx.x; k < ld; k += nthr) {
            double y = 0.0;
            if (k < nbs) {
              const int64_t q = b0 + k;
              const int4 id = __ldg(reinterpret_cast<const int4 *>(a.nb_idx) + q);
              const double2 c01 = __ldg(reinterpret_cast<const double2 *>(a.nb_ca) + 2 * q);
              const double2 c23 = __ldg(reinterpret_cast<const double2 *>(a.nb_ca) + 2 * q + 1);
              const double yq = ldcg(yo + q);
              double acc = c01.x * ldcg(a.zf + id.x);
              if (id.y >= 0) acc += c01.y * ldcg(a.zf + id.y);
              if (id.z >= 0) acc += c23.x * ldcg(a.zf + id.z);
              if (id.w >= 0) acc += c23.y * ldcg(a.zf + id.w);
              y = yq - alpha * acc;
              if (k >= r0 && k < r1) yn[q] = y;
            }
            xs[k] = (T)y;
          }
        },
        [&](int s, int r, double v, double2) { a.zp[a.bofs[s] + r] = v; }, NoPre(), tsp(3));
  };
  // uz = B^T z on this CTA's chunk of interface copies (z recomputed on the fly)
  const int64_t qb = a.nbt * cta / G, qe = a.nbt * (cta + 1) / G;
  // uz = B^T B_D zp on this CTA's chunk (preconditioned runs), by the neighbour lists
  auto uz_chunk_nb = [&]() {
    for (int64_t q = qb + threadIdx.x; q < qe; q += nthr) {
      const int4 id = __ldg(reinterpret_cast<const int4 *>(a.nb_idx) + q);
      const double2 c01 = __ldg(reinterpret_cast<const double2 *>(a.nb_cb) + 2 * q);
      const double2 c23 = __ldg(reinterpret_cast<const double2 *>(a.nb_cb) + 2 * q + 1);
      double u = c01.x * ldcg(a.zp + id.x);
      if (id.y >= 0) u += c01.y * ldcg(a.zp + id.y);
      if (id.z >= 0) u += c23.x * ldcg(a.zp + id.z);
      if (id.w >= 0) u += c23.y * ldcg(a.zp + id.w);
      a.uz[q] = u;
    }
  };
  auto uz_chunk = [&](auto zf_of) {
    for (int64_t q = qb + threadIdx.x; q < qe; q += nthr) {
      double u = 0.0;
#pragma unroll
      for (int t = 0; t < BT_W; ++t) {
        int l = a.bt_lam[q * BT_W + t];
        if (l >= 0) u += a.bt_sgn[q * BT_W + t] * zf_of(l);
      }
      a.uz[q] = u;
    }
  };


  // ================= C: interior condensation  kg = [W_ii^{-1} f_i ; f_[bp] - G f_i]
  cur = prefetch(ring, opIG);
  if (!stream_phase<4>(ring, opIG, cur, xs, ybuf, errflag,
                       [&](int s, int, int) {
                         int64_t ko = a.kofs[s];
                         stage(a.ni[s], a.ldi[s], [&](int k) { return a.rhs[ko + k]; });
                       },
                       [&](int s, int r, double v, double2) {
                         int64_t ko = a.kofs[s];
                         a.kg[ko + r] = r < a.ni[s] ? v : a.rhs[ko + r] - v;
                       }))
    return;
  cur = prefetch(ring, opH);
  if (!sync(nullptr)) return;
  // ================= D: d = B zf with u = g_b, g_p
  if (!h_phase([&](int s, int, int) {
        int64_t kb = a.kofs[s] + a.ni[s];
        stage(a.nb[s], a.ldb[s], [&](int k) { return ldcg(a.kg + kb + k); });
      }))
    return;
  Cursor curS = prefetch(ring, coarse_first());
  if (!sync(nullptr)) return;
  coarse_rhs(true);
  if (!sync(nullptr)) return;
  cur = curS;
  if (!coarse_solve()) return;
  cur = prefetch(ring, opQ);
  if (!sync(nullptr)) return;
  if (!psi_phase([&](int64_t q, double v, double) { a.zf[q] = v; })) return;
  if (!a.precond_none) cur = prefetch(ring, opP);
  if (!sync(nullptr)) return;

  // ================= PCG: r = d, z = M^{-1} d
  double acc = 0;
  for (int64_t l = lb + threadIdx.x; l < le; l += nthr) {
    double dv = jump(a.zf, l);
    a.lam[l] = 0.0;
    a.r0[l] = dv;
    acc += dv * dv;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part_dd[cta] = acc;
  if (!a.precond_none && !precond_rows(a.yv0, [&](int l) { return jump(a.zf, l); })) return;
  cur = prefetch(ring, opH);
  if (!sync(nullptr)) return;
  const double dd = reduce_slot(part_dd, G, sh);
  if (cta == 0 && threadIdx.x == 0) *a.out_dd = dd;
  double rr = dd;
  int it = 0;
  if (dd > 0.0) {
    acc = 0;
    for (int64_t l = lb + threadIdx.x; l < le; l += nthr) {
      double rv = ldcg(a.r0 + l);
      double zv = a.precond_none ? rv : jumpD(a.zp, l);
      a.z[l] = zv;
      acc += rv * zv;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part_rz[cta] = acc;
    if (a.precond_none) uz_chunk([&](int l) { return ldcg(a.r0 + l); });
    else uz_chunk_nb();
    if (!sync(nullptr)) return;
    double rz_old = reduce_slot(part_rz, G, sh);
    double *rcur = a.r0, *rnxt = a.r1, *pcur = a.p0, *pnxt = a.p1;
    for (it = 1; it <= a.max_it; ++it) {
      unsigned long long *tr =
          (a.trace && cta == 0 && it <= TRACE_IT) ? a.trace + (size_t)(it - 1) * TRACE_SLOTS : nullptr;
      tsub = tr ? tr + 16 : nullptr;
      if (tr && threadIdx.x == 0) tr[14] = gtimer();
      // ---------------- P1: p_new, u = B^T p_new, [F; Psi^T] u
      double beta = 0.0;
      if (it > 1) {
        double rz_new = reduce_slot(part_rz, G, sh);
        beta = rz_new / rz_old;
        rz_old = rz_new;
      }
      for (int64_t l = lb + threadIdx.x; l < le; l += nthr) pnxt[l] = ldcg(a.z + l) + beta * ldcg(pcur + l);
      // u = B^T p_new = B^T z + beta B^T p_old  (uz from the previous phase, ub_old from the
      // previous iteration); this CTA stores u for its own rows into ub_new
      if (!h_phase([&](int s, int r0, int r1) {
            int64_t b0 = a.bofs[s];
            int nbs = a.nb[s];
            for (int k = threadIdx.x; k < a.ldb[s]; k += nthr) {
              double u = 0.0;
              if (k < nbs) {
                u = ldcg(a.uz + b0 + k) + (it > 1 ? beta * ldcg(ub_old + b0 + k) : 0.0);
                if (k >= r0 && k < r1) ub_new[b0 + k] = u;
              }
              xs[k] = (T)u;
            }
          }))
        return;
      curS = prefetch(ring, coarse_first());
      if (!sync(tr ? tr + 0 : nullptr)) return;
      // ---------------- P2, P3: coarse
      coarse_rhs(false);
      if (!sync(tr ? tr + 2 : nullptr)) return;
      cur = curS;
      if (!coarse_solve()) return;
      cur = prefetch(ring, opQ);
      if (!sync(tr ? tr + 4 : nullptr)) return;
      // ---------------- P4: zf = zb - Psi q; (p, F p) = (u, zf)
      acc = 0;
      if (!psi_phase([&](int64_t q, double v, double ubv) {  // ubv = B^T p_new (ub_new)
            a.zf[q] = v;
            acc += v * ubv;
          }))
        return;
      acc = block_sum(acc, sh);
      if (threadIdx.x == 0) part_pq[cta] = acc;
      if (!a.precond_none) cur = prefetch(ring, opP);
      if (!sync(tr ? tr + 6 : nullptr)) return;
      // ---------------- P5: alpha, owner updates, preconditioner
      double pq = reduce_slot(part_pq, G, sh);
      double alpha = rz_old / pq;
      acc = 0;
      for (int64_t l = lb + threadIdx.x; l < le; l += nthr) {
        double fp = jump(a.zf, l);
        a.lam[l] += alpha * ldcg(pnxt + l);
        double rv = ldcg(rcur + l) - alpha * fp;
        rnxt[l] = rv;
        acc += rv * rv;
      }
      acc = block_sum(acc, sh);
      if (threadIdx.x == 0) part_rr[cta] = acc;
      if (!a.precond_none && !precond_rows_y(alpha, yv_old, yv_new)) return;
      cur = prefetch(ring, opH);
      if (!sync(tr ? tr + 8 : nullptr)) return;
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
      if (a.precond_none) uz_chunk([&](int l) { return ldcg(rnxt + l); });
      else uz_chunk_nb();
      if (!sync(tr ? tr + 10 : nullptr)) return;
      double *t = rcur; rcur = rnxt; rnxt = t;
      t = pcur; pcur = pnxt; pnxt = t;
      t = ub_old; ub_old = ub_new; ub_new = t;
      t = yv_old; yv_old = yv_new; yv_new = t;
    }
  }
  tsub = nullptr;
  // ================= R: recovery with v_b = g_b - B^T lambda  (H rows prefetched)
  if (!h_phase([&](int s, int, int) {
        int64_t kb = a.kofs[s] + a.ni[s];
        int64_t b0 = a.bofs[s];
        int nbs = a.nb[s];
        for (int k = threadIdx.x; k < a.ldb[s]; k += nthr) {
          double v = 0;
          if (k < nbs) {
            const int32_t *L = a.bt_lam + (b0 + k) * BT_W;
            const double *W = a.bt_sgn + (b0 + k) * BT_W;
            v = ldcg(a.kg + kb + k);
#pragma unroll
            for (int t = 0; t < BT_W; ++t)
              if (L[t] >= 0) v -= W[t] * ldcg(a.lam + L[t]);
          }
          xs[k] = (T)v;
        }
      }))
    return;
  curS = prefetch(ring, coarse_first());
  if (!sync(nullptr)) return;
  coarse_rhs(true);
  if (!sync(nullptr)) return;
  cur = curS;
  if (!coarse_solve()) return;
  cur = prefetch(ring, opQ);
  if (!sync(nullptr)) return;
  if (!psi_phase([&](int64_t q, double v, double) { a.kx[a.b_kept[q]] = v; })) return;
  for (int64_t k = cb + threadIdx.x; k < ce; k += nthr) {  // a_p = q, every copy
#pragma unroll
    for (int t = 0; t < CP_W; ++t) {
      int pos = a.cp_pos[k * CP_W + t];
      if (pos >= 0) a.kx[a.p_kept[pos]] = ldcg(a.q + k);
    }
  }
  cur = prefetch(ring, opGT);
  if (!sync(nullptr)) return;
  // R5: a_i = z_i - G^T a_[bp]
  if (!stream_phase<4>(ring, opGT, cur, xs, ybuf, errflag,
                       [&](int s, int, int) {
                         int64_t ko = a.kofs[s] + a.ni[s];
                         stage(a.nb[s] + a.np[s], a.ldg[s], [&](int k) { return ldcg(a.kx + ko + k); });
                       },
                       [&](int s, int r, double v, double2) {
                         int64_t ko = a.kofs[s];
                         a.kx[ko + r] = ldcg(a.kg + ko + r) - v;
                       }))
    return;
  if (cta == 0 && threadIdx.x == 0) {
    *a.out_its = it > a.max_it ? a.max_it : it;
    *a.out_rr = rr;
  }
}

}  // namespace ieti
