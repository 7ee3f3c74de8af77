// Device part of the tree-cotree IETI-DP solver (Sec. 3 of the paper).
//
// Setup (once per problem): every patch's kept block W_s = M_s + dt K_s, ordered
// [interior i | interface b | primal p], is expanded densely and AUGMENTED by
// identity-coupled copies b' of its interface block and i' of its interior block:
//
//        [ W_ii  W_ib  W_ip  0  I ]
//        [ W_bi  W_bb  W_bp  I  0 ]   eliminating the i and b pivots (a partial
//        [ W_pi  W_pb  W_pp  0  0 ]   Cholesky) leaves in the trailing block
//        [ 0     I     0     0  0 ]   [[C_s, -Psi^T], [-Psi, -F_s]] and in the
//        [ I     0     0     0  0 ]   factor rows i' the block L_ii^{-T}
//
// with S_bb = W_bb - W_bi W_ii^{-1} W_ib (the Dirichlet-preconditioner block),
// F_s = S_bb^{-1} (the local dual operator B_s W_rr^{-1} B_s^T restricted to the
// interface), Psi_s = S_bb^{-1} S_bp (the primal basis on the interface) and
// C_s = S_pp - S_pb Psi_s (the local coarse Schur complement), i.e. the two
// sequential Schur complements of Sec. 3 computed explicitly by one batched dense
// kernel family.  The coarse S_c = sum_s A_s^T C_s A_s is inverted by the same
// trick ([[S_c, I], [I, 0]]).
//
// Step (Eq. (11)): f = M a^l + dt j; interior condensation with L_ii; PCG on the
// dual problem F lambda = d where every application of F and of the Dirichlet
// preconditioner is a batched dense GEMV with F_s, Psi_s, S_bb and S_c^{-1}
// (no triangular solve inside the CG iteration); recovery; interior
// back-substitution.  In mixed precision the local operators are FP32 and every
// step is wrapped in FP64 defect correction on the assembled system.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <type_traits>
#include <vector>

#include <unistd.h>

#include "chol_tc.cuh"
#include "device.h"
#include "nonlinear.cuh"
#include "pcg_kernel.cuh"
#include "coarse_nd.h"

namespace ieti {

#define CK(x)                                                                   \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      err = std::string(#x) + " failed: " + cudaGetErrorString(e_);             \
      return IETI_ERR_CUDA;                                                     \
    }                                                                           \
  } while (0)

constexpr int NB = 32;         // panel width of the partial Cholesky
constexpr int GEMV_BLOCK = 256;
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs for the deterministic reductions

template <class T> struct Acc { using type = T; };

// =============================================================================
// Setup kernels
// =============================================================================

// Expand the kept CSR rows into the augmented dense blocks (zeroed beforehand).
template <class TD>
__global__ void k_csr_to_dense(int64_t n_rows, const int32_t *row_patch, const int32_t *row_local,
                               const int64_t *rowptr, const int32_t *col_abs, const double *val,
                               const int64_t *kofs, const int64_t *doff, const int32_t *nn, TD *D) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n_rows) return;
  int s = row_patch[w];
  int r = row_local[w];
  int64_t ld = nn[s];
  TD *A = D + doff[s];
  for (int64_t t = rowptr[w] + lane; t < rowptr[w + 1]; t += 32) {
    int c = (int)(col_abs[t] - kofs[s]);
    A[r * ld + c] = (TD)val[t];
  }
}

// identity couplings of the augmented rows: b' (rows n..n+nb) to b, i' (rows
// n+nb..n+nb+ni) to i
template <class TD>
__global__ void k_augment(int n_patch, const int32_t *ni, const int32_t *nb, const int32_t *n,
                          const int32_t *nn, const int64_t *doff, TD *D) {
  int s = blockIdx.y;
  if (s >= n_patch) return;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int64_t ld = nn[s];
  TD *A = D + doff[s];
  if (k < nb[s]) {
    int64_t r = n[s] + k, c = ni[s] + k;
    A[r * ld + c] = 1.0;
    A[c * ld + r] = 1.0;
  }
  if (k < ni[s]) {
    int64_t r = n[s] + nb[s] + k, c = k;
    A[r * ld + c] = 1.0;
    A[c * ld + r] = 1.0;
  }
}

template <class T>
__global__ void k_potrf_diag(T *base, const int64_t *off, const int32_t *ldv, const int32_t *kbeg,
                             const int32_t *kend, int panel, int32_t *status) {
  int s = blockIdx.x;
  int j0 = kbeg[s] + panel * NB;
  int ke = kend[s];
  if (j0 >= ke) return;
  int jb = min(NB, ke - j0);
  int64_t ld = ldv[s];
  T *A = base + off[s];
  __shared__ double S[NB][NB + 1];
  for (int t = threadIdx.x; t < jb * jb; t += blockDim.x) {
    int r = t / jb, c = t % jb;
    S[r][c] = (c <= r) ? (double)A[(j0 + r) * ld + j0 + c] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < jb; ++k) {
    if (threadIdx.x == 0) {
      double d = S[k][k];
      if (!(d > 0.0) || !isfinite(d)) {
        if (status[s] == 0) status[s] = 1 + j0 + k;
        d = 1.0;  // keep the arithmetic finite; the host reports NOT_SPD
      }
      S[k][k] = sqrt(d);
    }
    __syncthreads();
    double piv = S[k][k];
    for (int i = k + 1 + threadIdx.x; i < jb; i += blockDim.x) S[i][k] /= piv;
    __syncthreads();
    int m = jb - k - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j <= i) S[i][j] -= S[i][k] * S[j][k];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < jb * jb; t += blockDim.x) {
    int r = t / jb, c = t % jb;
    if (c <= r) A[(j0 + r) * ld + j0 + c] = (T)S[r][c];
  }
}

// rows below the diagonal block: L_r = A_r L_jj^{-T} (one thread per row)

template <class T>
__global__ void k_trsm_panel(T *base, const int64_t *off, const int32_t *ldv, const int32_t *kbeg,
                             const int32_t *kend, const int32_t *nact, int panel, AugLimits lim) {
  using A_t = typename Acc<T>::type;
  int s = blockIdx.y;
  int j0 = kbeg[s] + panel * NB;
  int ke = kend[s];
  if (j0 >= ke) return;
  int jb = min(NB, ke - j0);
  int64_t ld = ldv[s];
  T *A = base + off[s];
  __shared__ A_t L[NB][NB + 1];
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    int i = t / NB, c = t % NB;
    L[i][c] = (i < jb && c <= i) ? (A_t)A[(j0 + i) * ld + j0 + c] : (A_t)(i == c ? 1 : 0);
  }
  __syncthreads();
  int r = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nact[s]) return;
  if (r >= lim.sk_lo[s] && r < lim.sk_hi[s]) return;
  T *row = A + r * ld + j0;
  A_t x[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    A_t v = (k < jb) ? (A_t)row[k] : (A_t)0;
#pragma unroll
    for (int m = 0; m < k; ++m) v -= x[m] * L[k][m];
    x[k] = v / L[k][k];
  }
#pragma unroll
  for (int k = 0; k < NB; ++k)
    if (k < jb) row[k] = (T)x[k];
}

// trailing lower update A[r][c] -= sum_k L[r][k] L[c][k] on 64x64 tiles.  With
// cend_panel >= 0 only the columns below kbeg + cend_panel * NB (and kend) are
// updated: the inner steps of a panel whose trailing part is updated separately.
template <class T>
__global__ void __launch_bounds__(256) k_syrk_update(T *base, const int64_t *off, const int32_t *ldv,
                                                     const int32_t *kbeg, const int32_t *kend,
                                                     const int32_t *nact, int panel, AugLimits lim,
                                                     int cend_panel = -1) {
  using A_t = typename Acc<T>::type;
  int s = blockIdx.y;
  int j0 = kbeg[s] + panel * NB;
  int ke = kend[s];
  if (j0 >= ke) return;
  int jb = min(NB, ke - j0);
  int t0 = j0 + jb;
  int na = nact[s];
  int m = na - t0;
  if (m <= 0) return;
  int T64 = (m + 63) / 64;
  int t = blockIdx.x;
  int ti, tj, cend = INT_MAX;
  if (cend_panel >= 0) {
    cend = min(kbeg[s] + cend_panel * NB, ke);
    int nc = (cend - t0 + 63) / 64;
    if (cend <= t0 || t >= T64 * nc) return;
    ti = t / nc;
    tj = t % nc;
    if (tj > ti) return;
  } else {
    if (t >= T64 * (T64 + 1) / 2) return;
    ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    tj = t - ti * (ti + 1) / 2;
  }
  int R0 = t0 + ti * 64, C0 = t0 + tj * 64;
  int sk_lo = lim.sk_lo[s], sk_hi = lim.sk_hi[s], rlim = lim.rlim[s], clim = lim.clim[s];
  if (R0 >= sk_lo && min(R0 + 64, na) <= sk_hi) return;   // rows with zero panel entries
  if (C0 >= sk_lo && min(C0 + 64, na) <= sk_hi) return;   // columns with zero panel entries
  if (R0 >= rlim && C0 >= clim) return;                   // block nobody reads
  int64_t ld = ldv[s];
  T *A = base + off[s];
  __shared__ A_t As[NB][64 + 1], Bs[NB][64 + 1];
  for (int idx = threadIdx.x; idx < 64 * NB; idx += 256) {
    int r = idx / NB, k = idx % NB;
    A_t a = 0, b = 0;
    if (k < jb) {
      if (R0 + r < na) a = (A_t)A[(R0 + r) * ld + j0 + k];
      if (C0 + r < na) b = (A_t)A[(C0 + r) * ld + j0 + k];
    }
    As[k][r] = a;
    Bs[k][r] = b;
  }
  __syncthreads();
  int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  A_t acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int k = 0; k < jb; ++k) {
    A_t a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = As[k][tr + 16 * i];
      b[i] = Bs[k][tc + 16 * i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = R0 + tr + 16 * i, c = C0 + tc + 16 * j;
      bool skip = (r >= sk_lo && r < sk_hi) || (r >= rlim && c >= clim) || c >= cend;
      if (r < na && c <= r && !skip) A[r * ld + c] = (T)((A_t)A[r * ld + c] - acc[i][j]);
    }
}

// P_s = S_bb (after the interior pivots), symmetrised from the lower triangle
template <class TD, class T>
__global__ void k_extract_P(const TD *D, const int64_t *doff, const int32_t *nn, const int32_t *ni,
                            const int32_t *nb, const int32_t *ldb, const int64_t *poff, T *P) {
  int s = blockIdx.y;
  int m = nb[s];
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  int r = (int)(idx / m), c = (int)(idx % m);
  int64_t ld = nn[s];
  const TD *A = D + doff[s];
  int rr = ni[s] + max(r, c), cc = ni[s] + min(r, c);
  P[poff[s] + (int64_t)r * ldb[s] + c] = (T)A[rr * ld + cc];
}

// H_s = [F_s; Psi_s^T] ((nb+np) x nb), Psi_s (nb x np), LY_s = first ni columns (n x ni)
template <class TD, class T>
__global__ void k_extract_ops(const TD *D, const int64_t *doff, const int32_t *nn, const int32_t *ni,
                              const int32_t *nb, const int32_t *np, const int32_t *ldb, const int32_t *ldp,
                              const int64_t *hoff, const int64_t *qoff, T *H, T *Q) {
  int s = blockIdx.y;
  int B = nb[s], Pn = np[s], I = ni[s];
  int n = I + B + Pn;
  int64_t ld = nn[s];
  const TD *A = D + doff[s];
  int64_t total = (int64_t)(B + Pn) * B;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(idx / B), c = (int)(idx % B);
    double v;
    if (r < B) {  // F = -(trailing b'b')
      int hi = max(r, c), lo = min(r, c);
      v = -A[(int64_t)(n + hi) * ld + n + lo];
    } else {      // Psi^T[r-B][c] = Psi[c][r-B] = -A[n + c][I + B + (r - B)]
      v = -A[(int64_t)(n + c) * ld + I + B + (r - B)];
      Q[qoff[s] + (int64_t)c * ldp[s] + (r - B)] = (T)v;
    }
    H[hoff[s] + (int64_t)r * ldb[s] + c] = (T)v;
  }
}

// IG_s (n x ldi): rows < ni hold W_ii^{-1} (= -trailing i'i'), rows >= ni hold
// G = W_[bp]i W_ii^{-1}; GT_s (ni x ldg) holds G^T.  After the interior pivots the
// trailing block of the augmented matrix has (i', i') = -W_ii^{-1} and
// (i', [b p]) = -W_ii^{-1} W_i[bp] = -G^T.
template <class TD, class T>
__global__ void k_extract_IG(const TD *D, const int64_t *doff, const int32_t *nn, const int32_t *ni,
                             const int32_t *nb, const int32_t *np, const int32_t *ldi, const int32_t *ldg,
                             const int64_t *igoff, const int64_t *gtoff, T *IG, T *GT) {
  int s = blockIdx.y;
  int I = ni[s], B = nb[s];
  int n = I + B + np[s];
  int64_t ld = nn[s];
  const TD *A = D + doff[s];
  int64_t total = (int64_t)n * I;
  int64_t ip = n + B;  // first i' row
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(idx / I), c = (int)(idx % I);
    double v;
    if (r < I) {
      int hi = max(r, c), lo = min(r, c);
      v = -A[(ip + hi) * ld + ip + lo];
    } else {
      v = -A[(ip + c) * ld + r];
      GT[gtoff[s] + (int64_t)c * ldg[s] + (r - I)] = (T)v;
    }
    IG[igoff[s] + (int64_t)r * ldi[s] + c] = (T)v;
  }
}

// coarse: Sc_aug[A[k]][A[l]] += C_s[k][l] (one launch per patch, in patch order)
template <class TD>
__global__ void k_coarse_add(const TD *D, int64_t doff, int nn, int ni, int nb, int np, const int32_t *A,
                             double *Sc, int64_t ldc) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)np * np) return;
  int k = (int)(idx / np), l = (int)(idx % np);
  int base = ni + nb;
  int hi = max(k, l), lo = min(k, l);
  double v = (double)D[doff + (int64_t)(base + hi) * nn + base + lo];
  Sc[(int64_t)A[k] * ldc + A[l]] += v;
}

__global__ void k_coarse_identity(int nc, double *Sc, int64_t ldc) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nc) return;
  Sc[(int64_t)(nc + r) * ldc + r] = 1.0;
  Sc[(int64_t)r * ldc + nc + r] = 1.0;
}

// (hi, lo) FP32 pairs of FP64 values: hi = fl32(x), lo = fl32(x - hi)
__global__ void k_split_pairs(int64_t n, const double *x, float2 *out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = x[i];
  float hi = (float)v;
  out[i] = make_float2(hi, (float)(v - (double)hi));
}

// C = alpha op(A) op(B) + beta C (row-major FP64; op = identity or transpose), 64 x 64
// tiles, 16-deep K slices in shared memory, 4 x 4 outputs per thread
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha, const double *A, int64_t lda,
                                               const double *B, int64_t ldb, double beta, double *C, int64_t ldc) {
  __shared__ double As[16][64 + 1], Bs[16][64 + 1];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
      int kk = idx / 64, ii = idx % 64;
      int k = k0 + kk, i = m0 + ii, j = n0 + ii;
      double a = 0, b = 0;
      if (k < K && i < M) a = TA ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k];
      if (k < K && j < N) b = TB ? B[(int64_t)j * ldb + k] : B[(int64_t)k * ldb + j];
      As[kk][ii] = a;
      Bs[kk][ii] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][tr + 16 * u];
        b[u] = Bs[kk][tc + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int i = m0 + tr + 16 * u, j = n0 + tc + 16 * v;
      if (i < M && j < N) {
        double *c = C + (int64_t)i * ldc + j;
        *c = alpha * acc[u][v] + (beta == 0.0 ? 0.0 : beta * *c);
      }
    }
}

// out[i][j] = S[ri[i]][ci[j]]  (gather of a sub-block of an ld-strided matrix)
__global__ void k_gather_block(int nr, int ncol, const int32_t *ri, const int32_t *ci, const double *S, int64_t ld,
                               double *out, int64_t ldo) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nr * ncol) return;
  int i = (int)(idx / ncol), j = (int)(idx % ncol);
  out[(int64_t)i * ldo + j] = S[(int64_t)ri[i] * ld + ci[j]];
}

// S[ri[i]][ci[j]] = sign * B[i][j]  (and, with tr, S[ci[j]][ri[i]] as well)
__global__ void k_scatter_block(int nr, int ncol, const int32_t *ri, const int32_t *ci, const double *B, int64_t ldb,
                                double sign, int tr, double *S, int64_t ld) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nr * ncol) return;
  int i = (int)(idx / ncol), j = (int)(idx % ncol);
  double v = sign * B[(int64_t)i * ldb + j];
  S[(int64_t)ri[i] * ld + ci[j]] = v;
  if (tr) S[(int64_t)ci[j] * ld + ri[i]] = v;
}

// aug = [[S, I], [I, 0]] (2n x 2n) from an n x n block S
__global__ void k_aug_identity_block(int n, const double *S, int64_t lds, double *aug) {
  int64_t ld = 2 * (int64_t)n;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ld * ld) return;
  int64_t r = idx / ld, c = idx % ld;
  double v = 0;
  if (r < n && c < n) v = S[r * lds + c];
  else if (r >= n && c == r - n) v = 1.0;
  else if (c >= n && r == c - n) v = 1.0;
  aug[idx] = v;
}

template <class TS>
__global__ void k_coarse_extract(int nc, const TS *Sc, int64_t ldc, double *Sinv, int ldo) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nc * nc) return;
  int r = (int)(idx / nc), c = (int)(idx % nc);
  int hi = max(r, c), lo = min(r, c);
  Sinv[(int64_t)r * ldo + c] = -(double)Sc[(int64_t)(nc + hi) * ldc + nc + lo];
}

// lower triangle of an FP64 matrix rounded to FP32 (leading dimensions ld, ldf)
__global__ void k_round_lower(int64_t n, const double *A, int64_t ld, float *F, int64_t ldf) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int64_t r = idx / n, c = idx % n;
  F[r * ldf + c] = c <= r ? (float)A[r * ld + c] : 0.f;
}

// ---- nested-dissection coarse factorization (multifrontal; fronts row-major, lower
// triangle, leading dimension na = 2 nk + ns: [K | S | K'] with K' = identity rows)

// original entries of S_c in the K columns of the front (rows K and S), identity rows K'
__global__ void k_front_init(const double *Sc, int64_t nc, const int32_t *fid, int nk, int ns, double *F,
                             int64_t ld) {
  const int m = nk + ns;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < (int64_t)m * nk) {
    const int i = (int)(idx / nk), j = (int)(idx % nk);
    if (i >= j) F[(int64_t)i * ld + j] = Sc[(int64_t)fid[i] * nc + fid[j]];
  }
  if (idx < nk) F[(int64_t)(m + idx) * ld + idx] = 1.0;
}

// F_parent[map[a]][map[b]] += U_child[a][b] (lower triangle; map ascending)
__global__ void k_extend_add(const double *Fc, int64_t ldc, int nkc, int nsc, const int32_t *map, double *Fp,
                             int64_t ldp) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nsc * nsc) return;
  const int a = (int)(idx / nsc), b = (int)(idx % nsc);
  if (b > a) return;
  Fp[(int64_t)map[a] * ldp + map[b]] += Fc[(int64_t)(nkc + a) * ldc + nkc + b];
}

// after the nk pivots: trailing [K' K'] = -D^{-1}, [K' S] = -Lbar^T.  Z = [D^{-1}; Lbar],
// Lt = Lbar^T (padding columns stay zero)
__global__ void k_front_extract(const double *F, int64_t ld, int nk, int ns, double *Z, int zld, double *Lt,
                                int ltld) {
  const int m = nk + ns;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nz = (int64_t)m * nk;
  if (idx < nz) {
    const int r = (int)(idx / nk), c = (int)(idx % nk);
    double v;
    if (r < nk) {
      const int hi = max(r, c), lo = min(r, c);
      v = -F[(int64_t)(m + hi) * ld + m + lo];
    } else {
      v = -F[(int64_t)(m + c) * ld + r];
    }
    Z[(int64_t)r * zld + c] = v;
  } else if (idx < nz + (int64_t)nk * ns) {
    const int64_t t = idx - nz;
    const int r = (int)(t / ns), j = (int)(t % ns);
    Lt[(int64_t)r * ltld + j] = -F[(int64_t)(m + r) * ld + nk + j];
  }
}

// =============================================================================
// Step kernels
// =============================================================================

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y[yidx] = alpha * A_row . x + beta * y0[yidx]    (warp per row)
template <class T>
__global__ void k_gemv_rows(int64_t n_rows, const int64_t *aoff, const int64_t *xoff, const int64_t *yidx,
                            const int32_t *ncol, const T *A, const double *x, double *y, const double *y0,
                            double alpha, double beta) {
  using A_t = typename Acc<T>::type;
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (; w < n_rows; w += nw) {
    const T *a = A + aoff[w];
    const double *xv = x + xoff[w];
    int nc = ncol[w];
    A_t acc = 0;
    for (int c = lane; c < nc; c += 32) acc += (A_t)a[c] * (A_t)xv[c];
    double sum = warp_sum((double)acc);
    if (lane == 0) {
      int64_t yi = yidx[w];
      double v = alpha * sum;
      if (y0) v += beta * y0[yi];
      y[yi] = v;
    }
  }
}

// kept-space gather of the global state: out[k] = a[glob[k]]
__global__ void k_gather_kept(int64_t nk, const int64_t *glob, const double *a, double *out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nk) out[k] = a[glob[k]];
}

// initial iterate of a step by extrapolation in time through the last two or three
// states: a = 2 a^l - a^{l-1}, or a = 3 a^l - 3 a^{l-1} + a^{l-2} (a_lm2 non-null);
// eliminated entries are 0 in all of them and stay 0
__global__ void k_extrapolate(int64_t n, const double *a_l, const double *a_lm1, const double *a_lm2, double *a) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  a[i] = a_lm2 ? 3.0 * (a_l[i] - a_lm1[i]) + a_lm2[i] : 2.0 * a_l[i] - a_lm1[i];
}

// f = M x + dt * w * j[glob]   (warp per CSR row)
__global__ void k_rhs(int64_t nk, const int64_t *ptr, const int32_t *col, const double *val, const double *x,
                      const int64_t *glob, const double *w, const double *j, double dt, double *f) {
  int lane = threadIdx.x & 31;
  int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (r >= nk) return;
  double acc = 0;
  for (int64_t t = ptr[r] + lane; t < ptr[r + 1]; t += 32) acc += val[t] * x[col[t]];
  acc = warp_sum(acc);
  if (lane == 0) f[r] = acc + dt * w[r] * j[glob[r]];
}

// r = f - W x
__global__ void k_resid(int64_t nk, const int64_t *ptr, const int32_t *col, const double *val, const double *x,
                        const double *f, double *r) {
  int lane = threadIdx.x & 31;
  int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (row >= nk) return;
  double acc = 0;
  for (int64_t t = ptr[row] + lane; t < ptr[row + 1]; t += 32) acc += val[t] * x[col[t]];
  acc = warp_sum(acc);
  if (lane == 0) r[row] = f[row] - acc;
}

// kept [b|p] parts -> B-space and Pi-space
__global__ void k_kept_to_bp(int64_t nbt, int64_t npt, const int64_t *b_kept, const int64_t *p_kept,
                             const double *kv, double *gb, double *gp) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nbt) gb[t] = kv[b_kept[t]];
  else if (t < nbt + npt) gp[t - nbt] = kv[p_kept[t - nbt]];
}

// u[q] = base[q] + sgn_mode * sum_t wt[t] * v[lam[t]]   (B^T or B_D^T, gather form)
__global__ void k_Bt(int64_t nbt, const int32_t *ptr, const int32_t *lam, const double *wt, const double *v,
                     const double *base, double sgn, double *u) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nbt) return;
  double acc = 0;
  for (int t = ptr[q]; t < ptr[q + 1]; ++t) acc += wt[t] * v[lam[t]];
  u[q] = (base ? base[q] : 0.0) + sgn * acc;
}

// out[lam] = wp * z[qp] - wm * z[qm]; optional partial dot with dotv
__global__ void k_jump(int64_t m, const int32_t *qp, const int32_t *qm, const double *wp, const double *wm,
                       const double *z, double *out, const double *dotv, double *part) {
  __shared__ double sh[32];
  double acc = 0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < m; l += (int64_t)gridDim.x * blockDim.x) {
    double a = wp ? wp[l] : 1.0, b = wm ? wm[l] : 1.0;
    double v = a * z[qp[l]] - b * z[qm[l]];
    out[l] = v;
    if (dotv) acc += v * dotv[l];
  }
  if (!part) return;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// cc[k] = sum over copies (gp[pos] - tp[pos])   (gp may be null)
__global__ void k_coarse_gather(int nc, const int32_t *ptr, const int32_t *pos, const double *gp, const double *tp,
                                double *cc) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc) return;
  double acc = 0;
  for (int t = ptr[k]; t < ptr[k + 1]; ++t) acc += (gp ? gp[pos[t]] : 0.0) - tp[pos[t]];
  cc[k] = acc;
}

__global__ void k_pgather(int64_t npt, const int32_t *pc, const double *q, double *qloc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < npt) qloc[t] = q[pc[t]];
}

// write the condensed solution into kept space: x[b] = zb, x[p] = q[pc]
__global__ void k_bp_to_kept(int64_t nbt, int64_t npt, const int64_t *b_kept, const int64_t *p_kept,
                             const int32_t *pc, const double *zb, const double *q, double *kx) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nbt) kx[b_kept[t]] = zb[t];
  else if (t < nbt + npt) kx[p_kept[t - nbt]] = q[pc[t - nbt]];
}

// a[glob[k]] += x[k] for owned kept entries
__global__ void k_owner_add(int64_t nk, const int64_t *glob, const uint8_t *own, const double *x, double *a) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nk && own[k]) a[glob[k]] += x[k];
}

// rg[fglob[f]] = sum over kept copies of v; partial sums of rg^2 (assembled residual)
__global__ void k_assemble_free(int64_t nf, const int64_t *ptr, const int64_t *pos, const int64_t *fglob,
                                const double *v, double *rg, double *part) {
  __shared__ double sh[32];
  double acc = 0;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int64_t t = ptr[f]; t < ptr[f + 1]; ++t) s += v[pos[t]];
    rg[fglob[f]] = s;
    acc += s * s;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    x = warp_sum(x);
    if (threadIdx.x == 0) part[blockIdx.x] = x;
  }
}

// local pieces of an assembled vector with the 1/k partition of unity: v[k] = w[k] rg[glob[k]]
__global__ void k_distribute(int64_t nk, const int64_t *glob, const double *w, const double *rg, double *v) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nk) v[k] = w[k] * rg[glob[k]];
}

__global__ void k_dot_partial(int64_t n, const double *x, const double *y, double *part) {
  __shared__ double sh[32];
  double acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i] * y[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// sc[idx] = sum(part); op 1: sc[4] = sc[1]/sc[2] (alpha); op 2: sc[5] = sc[6]/sc[1], sc[1] = sc[6] (beta)
enum { SC_DD = 0, SC_RZ = 1, SC_PQ = 2, SC_RR = 3, SC_ALPHA = 4, SC_BETA = 5, SC_RZNEW = 6, SC_TMP = 7, SC_FN = 8 };

// Device-side control of a step's refinement sweeps (graph mode): the decisions the
// host loop takes after reading the residual norm and the PCG status, taken on the
// device so that the whole sweep loop runs as one CUDA graph with a while node.
struct StepCtl {
  double prev, ores, rel;
  int sweeps, its, cg_fail, bar_err, status;  // status: 1 converged, 2 max sweeps, 3 stagnated, 4 barrier error
};

// after the residual norm of the current iterate: stop (converged, out of sweeps,
// stagnated, barrier error) or run one more sweep (the while node's condition)
__global__ void k_ctl_decide(StepCtl *c, const double *sc, cudaGraphConditionalHandle h, double outer_tol,
                             int max_sweeps, int first) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (first) {
    c->prev = -1.0;
    c->rel = 0.0;
    c->sweeps = c->its = c->cg_fail = c->bar_err = c->status = 0;
  }
  const double fn = sqrt(sc[SC_FN]), rn = sqrt(sc[SC_TMP]);
  const double ores = fn > 0.0 ? rn / fn : 0.0;
  c->ores = ores;
  unsigned cont = 0;
  if (c->bar_err) c->status = 4;
  else if (ores <= outer_tol || fn == 0.0) c->status = 1;
  else if (c->sweeps >= max_sweeps) c->status = 2;
  else if (c->sweeps >= 2 && rn > 0.9 * c->prev) c->status = 3;
  else {
    cont = 1;
    c->prev = rn;
  }
  cudaGraphSetConditional(h, cont);
}

// after a dual-primal solve: its iterations, barrier status and convergence
__global__ void k_ctl_solved(StepCtl *c, const int *its, const unsigned *bar, const double *rr, const double *dd,
                             double tol2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  c->sweeps++;
  c->its += *its;
  if (bar[1]) c->bar_err = 1;
  const double r = *rr, q = *dd;
  if (q > 0.0) {
    c->rel = sqrt(r / q);
    if (!isfinite(r) || r > tol2 * q) c->cg_fail = 1;
  }
}
// partial sums of sum_k own[k] x[k]^2 (each global DOF once)
__global__ void k_owner_sq(int64_t n, const uint8_t *own, const double *x, double *part) {
  __shared__ double sh[32];
  double acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (own[i]) acc += x[i] * x[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void k_dot_final(int nparts, const double *part, double *sc, int idx, int op) {
  __shared__ double sh[32];
  double acc = 0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w];
    sc[idx] = v;
    if (op == 1) sc[SC_ALPHA] = sc[SC_RZ] / sc[SC_PQ];
    if (op == 2) {
      sc[SC_BETA] = sc[SC_RZNEW] / sc[SC_RZ];
      sc[SC_RZ] = sc[SC_RZNEW];
    }
  }
}

// lam += alpha p; r -= alpha q; partial (r, r)
__global__ void k_cg_update(int64_t m, const double *sc, const double *p, const double *q, double *lam, double *r,
                            double *part) {
  __shared__ double sh[32];
  double alpha = sc[SC_ALPHA];
  double acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    lam[i] += alpha * p[i];
    double v = r[i] - alpha * q[i];
    r[i] = v;
    acc += v * v;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void k_p_update(int64_t m, const double *sc, const double *z, double *p) {
  double beta = sc[SC_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// =============================================================================
// Host-side state
// =============================================================================

template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
};

struct DeviceState {
  ieti_options opt{};
  double *a_prev = nullptr, *a_old = nullptr;  // a^{l-1} and a^l of the step in progress (predictor)
  double *a_prev2 = nullptr;                   // a^{l-2} (quadratic predictor)
  int n_hist = 0;                              // previous states held: a_prev (1), and a_prev2 (2)
  int device = 0;
  cudaStream_t stream = nullptr;
  bool mixed = false;
  std::vector<void *> allocs;
  int64_t bytes = 0;
  int64_t launches_setup = 0;
  double t_setup_ms = 0;
  // sizes
  int np_ = 0;
  int64_t n_edges = 0, NK = 0, NBt = 0, NPt = 0, M = 0, NC = 0, NF = 0;
  int64_t bytes_iter = 0;
  int max_ni = 0;
  std::vector<int32_t> h_ni, h_nb, h_np;
  // per patch device arrays
  int32_t *ni = nullptr, *nb = nullptr, *npp = nullptr;
  int64_t *kofs = nullptr, *igoff = nullptr, *gtoff = nullptr, *hoff = nullptr, *qoff = nullptr, *poff = nullptr;
  // kept space
  int64_t *kglob = nullptr;
  double *kw = nullptr;
  uint8_t *kown = nullptr;
  int64_t *wptr = nullptr, *mptr = nullptr;
  int32_t *wcol = nullptr, *mcol = nullptr;
  double *wval = nullptr, *mval = nullptr;
  // B / Pi / lambda / coarse maps
  int64_t *b_kept = nullptr, *p_kept = nullptr;
  int32_t *bt_ptr = nullptr, *bt_lam = nullptr;
  double *bt_sgn = nullptr, *bt_wd = nullptr;
  int32_t *lam_qp = nullptr, *lam_qm = nullptr;
  double *lam_wp = nullptr, *lam_wm = nullptr;
  int32_t *pc = nullptr, *cptr = nullptr, *cpos = nullptr;
  int64_t *fptr = nullptr, *fpos = nullptr, *fglob = nullptr;
  double *rglob = nullptr;
  // operators (T = double or float)
  void *IG = nullptr, *GT = nullptr, *H = nullptr, *Q = nullptr, *P = nullptr;
  double *Sinv = nullptr;
  // GEMV descriptors
  struct Desc {
    int64_t n = 0;
    int64_t *aoff = nullptr, *xoff = nullptr, *yidx = nullptr;
    int32_t *ncol = nullptr;
  } dH, dQ, dP, dS, dIGi, dIGg, dGT;
  // vectors
  double *a = nullptr, *j = nullptr, *kf = nullptr, *kx = nullptr, *kr = nullptr, *kz = nullptr, *ka = nullptr,
         *kt = nullptr;
  double *bp = nullptr, *ub = nullptr, *gb = nullptr, *gp = nullptr, *cc = nullptr, *q = nullptr, *qloc = nullptr;
  double *lam = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *Fp = nullptr, *dvec = nullptr;
  double *part = nullptr, *sc = nullptr, *h_sc = nullptr;
  // persistent PCG
  int G = 0, ldc = 0;
  size_t pcg_smem = 0;
  int32_t *ldb = nullptr, *ldp = nullptr, *ldi = nullptr, *ldg = nullptr, *bpatch = nullptr;
  int64_t *bofs_d = nullptr, *pofs_d = nullptr;
  int32_t *hseg_ptr = nullptr, *hseg_s = nullptr, *hseg_r0 = nullptr, *hseg_r1 = nullptr;
  int32_t *bseg_ptr = nullptr, *bseg_s = nullptr, *bseg_r0 = nullptr, *bseg_r1 = nullptr;
  int32_t *qseg_ptr = nullptr, *qseg_s = nullptr, *qseg_r0 = nullptr, *qseg_r1 = nullptr;
  int psi_overhead = 0;  // > 0: the Psi rows have their own partition (per-row overhead in elements)
  int seg_overhead = 0;  // per-segment weight of the row partitions (elements)
  int32_t *iseg_ptr = nullptr, *iseg_s = nullptr, *iseg_r0 = nullptr, *iseg_r1 = nullptr;
  int32_t *tseg_ptr = nullptr, *tseg_s = nullptr, *tseg_r0 = nullptr, *tseg_r1 = nullptr;
  double *kg = nullptr, *ub1 = nullptr, *uz = nullptr;
  // balanced (deflated) preconditioner: k patch pairs, the pair of every multiplier,
  // the multipliers of every pair (CSR), F U (k rows of length m), E^{-1} (k x k, FP64)
  int defl_k = 0;
  int32_t *defl_pair = nullptr, *defl_ptr = nullptr, *defl_lam = nullptr;
  double *defl_FUt = nullptr, *defl_Einv = nullptr, *defl_ur = nullptr, *defl_c = nullptr, *defl_fw = nullptr;
  double *defl_rh = nullptr, *defl_w = nullptr;
  double *Sdf = nullptr;  // mixed path: S_c^{-1} as (hi, lo) FP32 pairs, viewed as doubles
  // per-iteration operators (H, Q, P, coarse) share one arena, the L2 access-policy window
  unsigned char *iter_arena = nullptr;
  double *Scoarse_slot = nullptr;  // coarse operator used by the PCG kernel (inside iter_arena)
  size_t iter_bytes = 0, l2_window = 0;
  float l2_hit_ratio = 0.f;
  float l2_keep_frac = 0.f;  // l2_persist = 2: fraction of the arena's lines loaded evict-last
  bool l2_set = false;
  size_t l2_prev_limit = 0;
  int n_stages = 3;
  int32_t *ell_lam = nullptr, *cp_pos = nullptr;
  double *ell_sgn = nullptr, *ell_wd = nullptr;
  int32_t *nb_idx = nullptr;               // [NBt][NB_W] interface-copy neighbours (self first)
  double *nb_ca = nullptr, *nb_cb = nullptr;  // their B_D^T B and B^T B_D coefficients
  double *yv0 = nullptr, *yv1 = nullptr;    // B_D^T r of the current / next PCG iterate
  double *p1 = nullptr, *r1 = nullptr, *zb = nullptr, *zf = nullptr, *ubp = nullptr, *tpi = nullptr, *zp = nullptr,
         *ccg = nullptr, *ppart = nullptr;
  unsigned *bar = nullptr;
  int *pcg_its = nullptr;
  unsigned long long *trace = nullptr;
  double trace_acc[8] = {};   // summed per-phase time (us) over traced iterations: work P1..P6, waits
  double trace_wait[8] = {};
  double trace_sub[4][3] = {};  // P1, P3, P4, P5: staging, first chunk, rows (us)
  double trace_nd[TRACE_ND][4] = {};  // nested-dissection levels: staging, first chunk, rows, barrier (us)
  int64_t trace_nd_n = 0;
  int64_t trace_sub_n[4] = {};
  int64_t trace_n = 0;
  double *pcg_rr = nullptr, *pcg_dd = nullptr;
  double bytes_iter_alg = 0, bytes_sweep_alg = 0;
  unsigned xs_bytes = 0, stage_bytes = 0;
  // graph mode: the sweep loop of a step as one CUDA graph (while node)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  StepCtl *ctl = nullptr, *h_ctl = nullptr;
  // schedule of the persistent kernel: host copies of the per-patch row counts and
  // leading dimensions of its four partitions (re-planned by the autotuner)
  std::vector<int32_t> plan_rows[5], plan_ld[5];
  int ldmax = 4, n_sm = 0, cps = 1;
  int sched_source = 0, tune_candidates = 0;
  double tune_ms = 0, tune_us[2] = {0, 0};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double dt = 0;
  // kernel-class profiler (options.profile)
  ieti_kernel_stat kstat[IETI_K_NCLASS] = {};
  std::vector<cudaEvent_t> ev_pool;
  struct Pend { int cls; int e0; double bytes; };
  std::vector<Pend> pend;
  int ev_used = 0;
  double gemv_bytes[IETI_K_NCLASS] = {};  // algorithmic bytes of one launch per GEMV class
  int64_t nlaunch = 0;                    // kernels launched by the current step
  // setup factorization
  int factor = IETI_FACTOR_FP64;
  double t_factor_ms = 0;                 // both partial-Cholesky phases of the patch blocks
  double tc_ms = 0, tc_flops = 0, tc_useful_flops = 0;  // tensor-core trailing updates
  int64_t tc_launches = 0;
  double factor_flops = 0;                // useful flops of both phases (all factor modes)
  // coarse factorization descriptors (one matrix), kept for refactorizations
  int64_t *c_off = nullptr;
  int32_t *c_ld = nullptr, *c_kb = nullptr, *c_ke = nullptr, *c_na = nullptr, *c_st = nullptr, *c_z = nullptr,
          *c_big = nullptr;
  // nonlinear reluctivity: Newton with refactorization of the patches holding
  // nonlinear elements (the "nl batch") and of the coarse block
  bool nonlinear = false;
  NlLaw law{};
  int nl_np = 0;
  int64_t nl_ne = 0;
  int nl_max_nloc = 0, nl_max_nq = 0;
  double *nl_G = nullptr, *nl_cq = nullptr;
  int32_t *nl_kept = nullptr, *nl_nloc = nullptr, *nl_nq = nullptr, *nl_bpos = nullptr;
  int64_t *nl_glob = nullptr, *nl_goff = nullptr, *nl_qoff = nullptr, *nl_doff = nullptr;
  float4 *nl_tq = nullptr;
  void *nl_base = nullptr, *nl_work = nullptr;  // dense augmented blocks of the batch: W without the law, + dt K_t
  std::vector<int32_t> nlh_ids, nlh_nn, nlh_n, nlh_ni, nlh_nb, nlh_np;
  std::vector<int64_t> nlh_doff, nlh_pofs;
  int64_t nl_arena = 0;
  int64_t *nlb_doff = nullptr, *nlb_kofs = nullptr, *nlb_hoff = nullptr, *nlb_qoff = nullptr, *nlb_poff = nullptr,
          *nlb_igoff = nullptr, *nlb_gtoff = nullptr;
  int32_t *nlb_nn = nullptr, *nlb_ni = nullptr, *nlb_nb = nullptr, *nlb_np = nullptr, *nlb_ldb = nullptr,
          *nlb_ldp = nullptr, *nlb_ldi = nullptr, *nlb_ldg = nullptr, *nlb_n = nullptr;
  int32_t *nlb_kb = nullptr, *nlb_ke = nullptr, *nlb_na = nullptr, *nlb_st = nullptr, *nlb_sklo = nullptr,
          *nlb_skhi = nullptr, *nlb_rlim = nullptr, *nlb_clim = nullptr;
  double *sc_lin = nullptr, *sc_aug = nullptr;  // coarse: sum over the linear patches (nc x nc); work (2nc)^2
  int64_t refactors = 0;
  int32_t step_refactors = 0;
  double t_refactor_ms[4] = {};
  float *sc_aug32 = nullptr;             // FP32 copy of the augmented coarse block (mixed Newton refactors)
  int64_t ld32 = 0;          // tangent, local factorization + extraction, coarse, total (profile)
  // coarse block update: coarse unknowns split into L (untouched by the nonlinear
  // patches) and N; constants inv(S_LL), X = inv(S_LL) S_LN, Z0 = S_NN(linear) - S_NL X
  int cL = 0, cN = 0;
  int32_t *c_idxL = nullptr, *c_idxN = nullptr, *nl_pcN = nullptr;
  std::vector<int64_t> nlh_pcN;     // per batch patch: offset into nl_pcN
  double *c_SLLinv = nullptr, *c_X = nullptr, *c_Z0 = nullptr, *c_Zaug = nullptr, *c_Zinv = nullptr,
         *c_Y = nullptr, *c_Ltmp = nullptr;
  // coarse solve by nested dissection of the patch grid (coarse_nd = 1): per node the
  // operators Z = [D^{-1}; Lbar] and Lt = Lbar^T in the per-iteration arena, the
  // update buffer, the gather lists, and the rows of every level per CTA
  int coarse_nd = 0, nd_cw = 1, nd_H = 0, nd_D = 0, nd_nodes = 0, nd_zmax = 0;
  int32_t *nd_k0 = nullptr, *nd_nk = nullptr, *nd_ns = nullptr, *nd_zld = nullptr, *nd_ltld = nullptr,
          *nd_sidx = nullptr, *nd_dst = nullptr, *nd_nch = nullptr;
  int64_t *nd_zoff = nullptr, *nd_ltoff = nullptr, *nd_soff = nullptr, *nd_uoff = nullptr, *nd_srcoff = nullptr;
  double *nd_Z = nullptr, *nd_Lt = nullptr, *nd_slot = nullptr;
  int32_t *ndf_ptr = nullptr, *ndf_s = nullptr, *ndf_r0 = nullptr, *ndf_r1 = nullptr;
  int32_t *ndb_ptr = nullptr, *ndb_s = nullptr, *ndb_r0 = nullptr, *ndb_r1 = nullptr;
  int nd_flow = 0;                                      // levels wait on per-node counters, not grid barriers
  const CoarseTree *nd_tree = nullptr;                  // kept by the context; Newton refactorizations reuse it
  int32_t *nd_cptr = nullptr, *nd_cidx = nullptr, *nd_parent = nullptr, *nd_nsegf = nullptr, *nd_nsegb = nullptr;
  unsigned *nd_done = nullptr;
  std::vector<std::vector<int32_t>> ndh_fwd, ndh_bwd;   // node ids per forward / backward level
  std::vector<int32_t> ndh_nk, ndh_ns, ndh_zld, ndh_ltld;
  int64_t nd_z_elems = 0, nd_lt_elems = 0;              // padded sizes of the two operator blocks
  double nd_bytes = 0;                                  // algorithmic bytes of one coarse solve
  double t_coarse_ms = 0;                               // device time of the coarse factorization
  int factor_batches = 1;                               // patch batches of the setup factorization
};

// event pair around one launch of a kernel class (no-op unless profiling)
static void prof_begin(DeviceState *d, int cls, double bytes) {
  if (!d->opt.profile) return;
  if (d->ev_used + 2 > (int)d->ev_pool.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      d->ev_pool.push_back(e);
    }
  }
  d->pend.push_back({cls, d->ev_used, bytes});
  cudaEventRecord(d->ev_pool[d->ev_used], d->stream);
  d->ev_used += 2;
}
static void prof_end(DeviceState *d) {
  if (!d->opt.profile) return;
  cudaEventRecord(d->ev_pool[d->pend.back().e0 + 1], d->stream);
}
static void prof_set_bytes(DeviceState *d, double bytes) {
  if (d->opt.profile && !d->pend.empty()) d->pend.back().bytes = bytes;
}
static void prof_collect(DeviceState *d) {
  if (!d->opt.profile || d->pend.empty()) return;
  cudaStreamSynchronize(d->stream);
  for (auto &p : d->pend) {
    float ms = 0;
    cudaEventElapsedTime(&ms, d->ev_pool[p.e0], d->ev_pool[p.e0 + 1]);
    d->kstat[p.cls].launches++;
    d->kstat[p.cls].total_ms += ms;
    d->kstat[p.cls].bytes += p.bytes;
  }
  d->pend.clear();
  d->ev_used = 0;
}

template <class T>
static int dalloc(DeviceState *d, T **ptr, size_t n, std::string &err) {
  *ptr = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)ptr, n * sizeof(T));
  if (e != cudaSuccess) {
    err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
    return IETI_ERR_OOM;
  }
  d->allocs.push_back((void *)*ptr);
  d->bytes += (int64_t)(n * sizeof(T));
  return IETI_OK;
}

template <class T>
static int upload(DeviceState *d, T **ptr, const std::vector<T> &h, std::string &err) {
  int rc = dalloc(d, ptr, h.size(), err);
  if (rc) return rc;
  if (!h.empty()) CK(cudaMemcpyAsync(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return IETI_OK;
}

static int upload_desc(DeviceState *d, DeviceState::Desc &D, const std::vector<int64_t> &aoff,
                        const std::vector<int64_t> &xoff, const std::vector<int64_t> &yidx,
                        const std::vector<int32_t> &ncol, std::string &err) {
  D.n = (int64_t)aoff.size();
  int rc;
  if ((rc = upload(d, &D.aoff, aoff, err)) || (rc = upload(d, &D.xoff, xoff, err)) ||
      (rc = upload(d, &D.yidx, yidx, err)) || (rc = upload(d, &D.ncol, ncol, err)))
    return rc;
  return IETI_OK;
}

static inline unsigned grid_for(int64_t n, int block) { return (unsigned)std::max<int64_t>(1, (n + block - 1) / block); }

template <class T>
static void gemv(DeviceState *d, const DeviceState::Desc &D, const void *A, const double *x, double *y,
                 const double *y0, double alpha, double beta, int cls) {
  if (D.n == 0) return;
  prof_begin(d, cls, d->gemv_bytes[cls]);
  int64_t warps = D.n;
  unsigned blocks = (unsigned)std::min<int64_t>((warps * 32 + GEMV_BLOCK - 1) / GEMV_BLOCK, 152 * 16);
  k_gemv_rows<T><<<blocks, GEMV_BLOCK, 0, d->stream>>>(D.n, D.aoff, D.xoff, D.yidx, D.ncol, (const T *)A, x, y, y0,
                                                        alpha, beta);
  d->nlaunch++;
  prof_end(d);
}

// partial Cholesky over all patches (host loop over panels)
template <class T>
static int potrf_partial(DeviceState *d, T *base, const int64_t *off, const int32_t *ld, const std::vector<int32_t> &hkb,
                         const std::vector<int32_t> &hke, const std::vector<int32_t> &hna, int32_t *dkb, int32_t *dke,
                         int32_t *dna, int32_t *status, AugLimits lim, std::string &err) {
  int nbatch = (int)hkb.size();
  int max_panels = 0;
  for (int s = 0; s < nbatch; ++s) max_panels = std::max(max_panels, (hke[s] - hkb[s] + NB - 1) / NB);
  for (int j = 0; j < max_panels; ++j) {
    int max_rows = 0, max_tiles = 0;
    for (int s = 0; s < nbatch; ++s) {
      int j0 = hkb[s] + j * NB;
      if (j0 >= hke[s]) continue;
      int jb = std::min(NB, hke[s] - j0);
      int m = hna[s] - (j0 + jb);
      if (m <= 0) continue;
      max_rows = std::max(max_rows, m);
      int T64 = (m + 63) / 64;
      max_tiles = std::max(max_tiles, T64 * (T64 + 1) / 2);
    }
    k_potrf_diag<T><<<nbatch, 256, 0, d->stream>>>(base, off, ld, dkb, dke, j, status);
    d->nlaunch++;
    d->launches_setup++;
    if (max_rows > 0) {
      dim3 g1(grid_for(max_rows, 128), nbatch);
      k_trsm_panel<T><<<g1, 128, 0, d->stream>>>(base, off, ld, dkb, dke, dna, j, lim);
      d->nlaunch++;
      dim3 g2(max_tiles, nbatch);
      k_syrk_update<T><<<g2, 256, 0, d->stream>>>(base, off, ld, dkb, dke, dna, j, lim);
      d->nlaunch++;
      d->launches_setup += 2;
    }
  }
  CK(cudaGetLastError());
  return IETI_OK;
}

// ---------------------------------------------------------------------------
// Partial Cholesky of FP32 blocks with tensor-core trailing updates.
//
// Outer panels of TC_KP columns.  Each is factored by the SIMT kernels in NB-wide
// steps that update only the panel's own columns, then its rows below the panel
// are split into TF32 hi/lo planes (k_panel_split) and the whole trailing lower
// triangle is updated once on the tensor cores (k_syrk_tc).

// cuTensorMapEncodeTiled, resolved from the driver at run time (the library links
// only the CUDA runtime, so it loads on machines without a driver)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled(std::string &err) {
  static std::mutex mu;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      err = "cuTensorMapEncodeTiled is not available from the driver";
      return nullptr;
    }
    fn = (EncodeTiledFn)p;
  }
  return fn;
}

// host copies of the per-patch limits, for building the tile list
struct TcHost {
  std::vector<int64_t> off;
  std::vector<int32_t> ld, sk_lo, sk_hi, rlim, clim;
};

// The output tiles of every outer panel (patch-major, lower triangle, restricted by
// the limits), their useful flops, and each panel's slice of the list.
static void tc_plan(const TcHost &th, const std::vector<int32_t> &hkb, const std::vector<int32_t> &hke,
                    const std::vector<int32_t> &hna, int kch, std::vector<TcItem> &items, std::vector<int64_t> &pofs,
                    double &flops) {
  const int nb = (int)hkb.size();
  int max_outer = 0;
  for (int s = 0; s < nb; ++s) max_outer = std::max(max_outer, (hke[s] - hkb[s] + TC_KP - 1) / TC_KP);
  items.clear();
  pofs.assign(1, 0);
  flops = 0;
  for (int P = 0; P < max_outer; ++P) {
    for (int s = 0; s < nb; ++s) {
      const int J = hkb[s] + P * TC_KP;
      if (J >= hke[s]) continue;
      const int Je = std::min(J + TC_KP, hke[s]), t0 = Je, na = hna[s];
      if (t0 >= na) continue;
      const int t0a = t0 & ~3, nk = (Je - J + kch - 1) / kch;
      const int sklo = th.sk_lo[s], skhi = th.sk_hi[s], rlim = th.rlim[s], clim = th.clim[s];
      for (int R0 = t0; R0 < na; R0 += TC_BM) {
        const int Rend = std::min(R0 + TC_BM, na);
        if (R0 >= sklo && Rend <= skhi) continue;
        for (int C0 = t0a; C0 < Rend; C0 += TC_BN) {
          const int cf = std::max(C0, t0), cl = std::min(C0 + TC_BN, Rend) - 1;
          if (cf > cl) continue;
          if (cf >= sklo && cl < skhi) continue;
          if (R0 >= rlim && cf >= clim) continue;
          items.push_back({s, R0, C0, t0, nk, 0});
        }
      }
      // useful multiply-adds: every updated (r, c) with K = Je - J
      for (int r = t0; r < na; ++r) {
        if (r >= sklo && r < skhi) continue;
        int cmax = (r >= rlim) ? std::min(r, clim - 1) : r;
        if (cmax >= t0) flops += 2.0 * (double)(cmax - t0 + 1) * (Je - J);
      }
    }
    pofs.push_back((int64_t)items.size());
  }
}

// Useful flops of a partial Cholesky phase: for every pivot k, the scaled column and the
// rank-1 update of the active rows below it (rows in the skip range hold zeros there,
// rows >= rlim stop at column clim).
static double partial_chol_flops(const TcHost &th, const std::vector<int32_t> &hkb, const std::vector<int32_t> &hke,
                                 const std::vector<int32_t> &hna) {
  double f = 0;
  for (size_t s = 0; s < hkb.size(); ++s) {
    const int sklo = th.sk_lo[s], skhi = th.sk_hi[s], rlim = th.rlim[s], clim = th.clim[s];
    for (int k = hkb[s]; k < hke[s]; ++k) {
      // active rows r in (k, na) outside [sklo, skhi)
      const int lo = k + 1, hi = hna[s];
      if (lo >= hi) continue;
      int m = hi - lo - std::max(0, std::min(hi, skhi) - std::max(lo, sklo));
      double upd = 0.5 * (double)m * (m + 1);  // lower-triangle entries (r, c), k < c <= r
      if (rlim < hi && clim <= hi) {            // rows >= rlim only reach columns < clim
        int mr = hi - std::max(lo, rlim);
        int mc = std::max(0, hi - std::max(lo, clim));
        upd -= 0.5 * (double)std::min(mr, mc) * (std::min(mr, mc) + 1);
      }
      f += (double)m + 2.0 * upd;
    }
  }
  return f;
}

template <int X3, int BF>
static int potrf_partial_tc(DeviceState *d, float *base, const int64_t *off, const int32_t *ld, const TcHost &th,
                            const std::vector<int32_t> &hkb, const std::vector<int32_t> &hke,
                            const std::vector<int32_t> &hna, int32_t *dkb, int32_t *dke, int32_t *dna,
                            int32_t *status, AugLimits lim, std::string &err) {
  const int nbatch = (int)hkb.size();
  constexpr int IN = TC_KP / NB;  // inner steps per outer panel
  std::vector<TcItem> items;
  std::vector<int64_t> pofs;
  double flops = 0;
  using E = TcElem<BF>;
  tc_plan(th, hkb, hke, hna, E::KCH, items, pofs, flops);
  const int max_outer = (int)pofs.size() - 1;
  if (max_outer <= 0) return IETI_OK;
  // stacked panel buffer: patch s owns rows [ro[s], ro[s] + nact[s])
  std::vector<int64_t> hro(nbatch);
  int64_t R = 0;
  for (int s = 0; s < nbatch; ++s) {
    hro[s] = R;
    R += std::max(hna[s], 1);
  }
  if (R + 2 * TC_BN >= (int64_t)INT32_MAX) {
    err = "the stacked panel buffer exceeds 2^31 rows";
    return IETI_ERR_TOO_LARGE;
  }
  EncodeTiledFn enc = encode_tiled(err);
  if (!enc) return IETI_ERR_CUDA;
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaFuncSetAttribute(k_syrk_tc<X3, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<X3>::SMEM));
  // scratch: tile list, panel planes, row offsets, error word (freed before returning)
  typename E::T *PB = nullptr;
  TcItem *ditems = nullptr;
  int64_t *dro = nullptr;
  int32_t *derr = nullptr;
  auto release = [&]() {
    cudaStreamSynchronize(d->stream);
    cudaFree(PB);
    cudaFree(ditems);
    cudaFree(dro);
    cudaFree(derr);
  };
  size_t pb_bytes = (size_t)2 * R * TC_KP * sizeof(typename E::T);
  if (cudaMalloc((void **)&PB, pb_bytes) != cudaSuccess ||
      cudaMalloc((void **)&ditems, std::max<size_t>(items.size(), 1) * sizeof(TcItem)) != cudaSuccess ||
      cudaMalloc((void **)&dro, nbatch * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc((void **)&derr, sizeof(int32_t)) != cudaSuccess) {
    release();
    err = "cudaMalloc failed for the tensor-core factorization scratch";
    return IETI_ERR_OOM;
  }
  if (cudaMemsetAsync(PB, 0, pb_bytes, d->stream) != cudaSuccess ||
      cudaMemsetAsync(derr, 0, sizeof(int32_t), d->stream) != cudaSuccess ||
      cudaMemcpyAsync(ditems, items.data(), items.size() * sizeof(TcItem), cudaMemcpyHostToDevice, d->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(dro, hro.data(), nbatch * sizeof(int64_t), cudaMemcpyHostToDevice, d->stream) != cudaSuccess ||
      cudaStreamSynchronize(d->stream) != cudaSuccess) {
    release();
    err = "upload of the tensor-core factorization plan failed";
    return IETI_ERR_CUDA;
  }
  CUtensorMap tm;
  {
    const cuuint64_t esz = sizeof(typename E::T);
    cuuint64_t gdim[3] = {(cuuint64_t)TC_KP, (cuuint64_t)R, 2};
    cuuint64_t gstr[2] = {(cuuint64_t)TC_KP * esz, (cuuint64_t)R * TC_KP * esz};
    cuuint32_t box[3] = {(cuuint32_t)E::KCH, (cuuint32_t)TC_BM, 1};  // 128 bytes of K per row
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(&tm, BF ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, PB, gdim, gstr,
                     box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      release();
      err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
      return IETI_ERR_CUDA;
    }
  }
  std::vector<cudaEvent_t> evs;
  for (int P = 0; P < max_outer; ++P) {
    for (int q = 0; q < IN; ++q) {
      const int j = P * IN + q;
      bool any = false;
      int max_rows = 0, max_tiles = 0;
      for (int s = 0; s < nbatch; ++s) {
        const int j0 = hkb[s] + j * NB;
        const int Je = std::min(hkb[s] + (P + 1) * TC_KP, hke[s]);
        if (j0 >= Je) continue;
        any = true;
        const int jb = std::min(NB, hke[s] - j0);
        const int m = hna[s] - (j0 + jb);
        if (m <= 0) continue;
        max_rows = std::max(max_rows, m);
        const int nc = (Je - (j0 + jb) + 63) / 64;
        if (nc > 0) max_tiles = std::max(max_tiles, ((m + 63) / 64) * nc);
      }
      if (!any) continue;
      k_potrf_diag<float><<<nbatch, 256, 0, d->stream>>>(base, off, ld, dkb, dke, j, status);
      d->launches_setup++;
      if (max_rows > 0) {
        dim3 g1(grid_for(max_rows, 128), nbatch);
        k_trsm_panel<float><<<g1, 128, 0, d->stream>>>(base, off, ld, dkb, dke, dna, j, lim);
        d->launches_setup++;
        if (max_tiles > 0) {
          dim3 g2(max_tiles, nbatch);
          k_syrk_update<float><<<g2, 256, 0, d->stream>>>(base, off, ld, dkb, dke, dna, j, lim, (P + 1) * IN);
          d->launches_setup++;
        }
      }
    }
    const int64_t n_it = pofs[P + 1] - pofs[P];
    if (n_it == 0) continue;
    int max_m = 0;
    for (int s = 0; s < nbatch; ++s) {
      const int J = hkb[s] + P * TC_KP;
      if (J < hke[s]) max_m = std::max(max_m, hna[s] - std::min(J + TC_KP, hke[s]));
    }
    dim3 gs(std::min<unsigned>(grid_for(max_m, 8), 512), nbatch);
    k_panel_split<X3, BF><<<gs, 256, 0, d->stream>>>(base, off, ld, dkb, dke, dna, P, dro, R, PB);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    evs.push_back(e0);
    evs.push_back(e1);
    cudaEventRecord(e0, d->stream);
    const unsigned grid = (unsigned)std::min<int64_t>(n_it, nsm);
    k_syrk_tc<X3, BF><<<grid, TC_THREADS, TcCfg<X3>::SMEM, d->stream>>>(tm, ditems + pofs[P], (int)n_it, base, off,
                                                                       ld, dro, dna, lim, derr);
    cudaEventRecord(e1, d->stream);
    d->launches_setup += 2;
    d->tc_launches++;
  }
  cudaError_t e = cudaGetLastError();
  int32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int32_t), cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  for (size_t k = 0; k + 1 < evs.size(); k += 2) {
    float ms = 0;
    if (e == cudaSuccess && cudaEventElapsedTime(&ms, evs[k], evs[k + 1]) == cudaSuccess) d->tc_ms += ms;
    cudaEventDestroy(evs[k]);
    cudaEventDestroy(evs[k + 1]);
  }
  d->tc_flops += flops * (X3 ? 3.0 : 1.0);
  d->tc_useful_flops += flops;
  release();
  if (e != cudaSuccess) {
    err = std::string("tensor-core partial Cholesky failed: ") + cudaGetErrorString(e);
    return IETI_ERR_CUDA;
  }
  if (herr) {
    err = "tensor-core trailing update gave up waiting (stage " + std::to_string(herr) + ")";
    return IETI_ERR_CUDA;
  }
  return IETI_OK;
}

// one partial-Cholesky phase of an FP32 batch in a reduced factor arithmetic
// (IETI_FACTOR_FP32 on the SIMT pipe, the others with tensor-core trailing updates)
static int potrf_partial_f32(DeviceState *d, int factor, float *base, const int64_t *off, const int32_t *ld,
                             const TcHost &th, const std::vector<int32_t> &hkb, const std::vector<int32_t> &hke,
                             const std::vector<int32_t> &hna, int32_t *dkb, int32_t *dke, int32_t *dna,
                             int32_t *status, AugLimits lim, std::string &err) {
  switch (factor) {
    case IETI_FACTOR_FP32:
      return potrf_partial<float>(d, base, off, ld, hkb, hke, hna, dkb, dke, dna, status, lim, err);
    case IETI_FACTOR_TF32X3:
      return potrf_partial_tc<1, 0>(d, base, off, ld, th, hkb, hke, hna, dkb, dke, dna, status, lim, err);
    case IETI_FACTOR_TF32:
      return potrf_partial_tc<0, 0>(d, base, off, ld, th, hkb, hke, hna, dkb, dke, dna, status, lim, err);
    case IETI_FACTOR_BF16X3:
      return potrf_partial_tc<1, 1>(d, base, off, ld, th, hkb, hke, hna, dkb, dke, dna, status, lim, err);
    case IETI_FACTOR_BF16:
      return potrf_partial_tc<0, 1>(d, base, off, ld, th, hkb, hke, hna, dkb, dke, dna, status, lim, err);
    default:
      err = "unknown factor arithmetic";
      return IETI_ERR_INVALID_ARG;
  }
}

// one partial-Cholesky phase of a batch in the context's factor arithmetic
template <class TD>
static int run_partial(DeviceState *d, TD *D, const int64_t *doff, const int32_t *ld, const TcHost &th,
                       const std::vector<int32_t> &hkb, const std::vector<int32_t> &hke,
                       const std::vector<int32_t> &hna, int32_t *dkb, int32_t *dke, int32_t *dna, int32_t *dst,
                       AugLimits lim, std::string &err) {
  if constexpr (std::is_same<TD, double>::value) {
    return potrf_partial<double>(d, D, doff, ld, hkb, hke, hna, dkb, dke, dna, dst, lim, err);
  } else {
    return potrf_partial_f32(d, d->factor, D, doff, ld, th, hkb, hke, hna, dkb, dke, dna, dst, lim, err);
  }
}

static int coarse_publish(DeviceState *d, std::string &err);

static int nd_ld(int n) {  // leading dimension of an FP64 operator block: an odd number of 16-byte units
  if (n <= 0) return 0;
  int l = (n + 3) / 4 * 4;
  if ((l / 2) % 2 == 0) l += 2;
  return l;
}

// Host part of the nested-dissection coarse solve: node tables, the gather lists of
// the child updates, the per-level node lists and the operator layout (Z and Lt
// blocks, offsets into d->nd_Z / d->nd_Lt).  Sizes only; the operators come from
// coarse_nd_factor.
static int coarse_nd_tables(DeviceState *d, const CoarseTree &t, std::string &err) {
  const int NN = t.n_nodes;
  d->nd_nodes = NN;
  d->nd_H = t.n_height;
  d->nd_D = t.n_depth;
  d->ndh_nk.assign(t.nk.begin(), t.nk.end());
  d->ndh_ns.assign(t.ns.begin(), t.ns.end());
  d->ndh_zld.resize(NN);
  d->ndh_ltld.resize(NN);
  std::vector<int64_t> zoff(NN), ltoff(NN), uoff(NN), srcoff(NN);
  int64_t z = 0, lt = 0, u = 0, sr = 0;
  d->nd_zmax = 4;
  d->nd_bytes = 0;
  for (int p = 0; p < NN; ++p) {
    const int nk = t.nk[p], ns = t.ns[p];
    d->ndh_zld[p] = nd_ld(nk);
    d->ndh_ltld[p] = nd_ld(ns);
    zoff[p] = z;
    ltoff[p] = lt;
    uoff[p] = u;
    srcoff[p] = sr;
    z += (int64_t)(nk + ns) * d->ndh_zld[p];
    lt += (int64_t)nk * d->ndh_ltld[p];
    u += ns;
    sr += nk + ns;
    d->nd_zmax = std::max({d->nd_zmax, d->ndh_zld[p], d->ndh_ltld[p]});
    // every entry of Z read once forward, of Lt once backward; the staged vectors once per node
    d->nd_bytes += 8.0 * ((double)(nk + ns) * nk + (double)nk * ns) + 8.0 * (3.0 * nk + 2.0 * ns);
  }
  d->nd_z_elems = z;
  d->nd_lt_elems = lt;
  // child updates per front position
  std::vector<std::vector<int32_t>> lists(sr);
  int cw = 1;
  for (int p = 0; p < NN; ++p)
    for (int k = t.child_ptr[p]; k < t.child_ptr[p + 1]; ++k) {
      const int ch = t.child_idx[k];
      for (int j = 0; j < t.ns[ch]; ++j) {
        const int i = t.front_index(p, t.s_idx[t.s_off[ch] + j]);
        if (i < 0) {
          err = "nested dissection: a child update has no place in its parent's front";
          return IETI_ERR_INVALID_ARG;
        }
        auto &L = lists[srcoff[p] + i];
        L.push_back((int32_t)(uoff[ch] + j));
        cw = std::max(cw, (int)L.size());
      }
    }
  if (u >= (int64_t)INT32_MAX || z >= ((int64_t)1 << 40)) {
    err = "coarse problem too large for the nested-dissection solver";
    return IETI_ERR_TOO_LARGE;
  }
  d->nd_cw = cw;
  if ((int64_t)sr * cw >= (int64_t)INT32_MAX) {
    err = "coarse problem too large for the nested-dissection solver";
    return IETI_ERR_TOO_LARGE;
  }
  // slot w of front position i of node p receives the update of the w-th child that
  // contributes there (child order): every update row of every node has one slot in
  // its parent's front (dst), so that a parent reads its positions' updates
  // contiguously; slots that no child fills stay zero
  std::vector<int32_t> dst(std::max<int64_t>(u, 1), 0);
  for (int64_t i = 0; i < sr; ++i)
    for (size_t w = 0; w < lists[i].size(); ++w) dst[lists[i][w]] = (int32_t)(i * cw + (int64_t)w);
  std::vector<int64_t> srcoff_w(NN), soff(t.s_off.begin(), t.s_off.end() - 1);
  for (int p = 0; p < NN; ++p) srcoff_w[p] = srcoff[p] * cw;
  d->ndh_fwd.assign(d->nd_H, {});
  d->ndh_bwd.assign(std::max(d->nd_D - 1, 0), {});
  for (int p = 0; p < NN; ++p) {
    d->ndh_fwd[t.height[p]].push_back(p);
    if (t.depth[p] > 0 && t.ns[p] > 0 && t.nk[p] > 0) d->ndh_bwd[t.depth[p] - 1].push_back(p);
  }
  std::vector<int32_t> sidx(t.s_idx), nch(NN);
  if (sidx.empty()) sidx.push_back(0);
  for (int p = 0; p < NN; ++p) nch[p] = t.child_ptr[p + 1] - t.child_ptr[p];
  int rc;
  if ((rc = upload(d, &d->nd_k0, t.k0, err)) || (rc = upload(d, &d->nd_nk, d->ndh_nk, err)) ||
      (rc = upload(d, &d->nd_ns, d->ndh_ns, err)) || (rc = upload(d, &d->nd_zld, d->ndh_zld, err)) ||
      (rc = upload(d, &d->nd_ltld, d->ndh_ltld, err)) || (rc = upload(d, &d->nd_sidx, sidx, err)) ||
      (rc = upload(d, &d->nd_dst, dst, err)) || (rc = upload(d, &d->nd_nch, nch, err)) ||
      (rc = upload(d, &d->nd_zoff, zoff, err)) ||
      (rc = upload(d, &d->nd_ltoff, ltoff, err)) || (rc = upload(d, &d->nd_soff, soff, err)) ||
      (rc = upload(d, &d->nd_uoff, uoff, err)) || (rc = upload(d, &d->nd_srcoff, srcoff_w, err)) ||
      (rc = dalloc(d, &d->nd_slot, (size_t)std::max<int64_t>(sr * cw, 2), err)))
    return rc;
  CK(cudaMemsetAsync(d->nd_slot, 0, (size_t)std::max<int64_t>(sr * cw, 2) * sizeof(double), d->stream));
  std::vector<int32_t> cidx(t.child_idx);
  if (cidx.empty()) cidx.push_back(0);
  if ((rc = upload(d, &d->nd_cptr, t.child_ptr, err)) || (rc = upload(d, &d->nd_cidx, cidx, err)) ||
      (rc = upload(d, &d->nd_parent, t.parent, err)) || (rc = dalloc(d, &d->nd_nsegf, (size_t)NN, err)) ||
      (rc = dalloc(d, &d->nd_nsegb, (size_t)NN, err)) || (rc = dalloc(d, &d->nd_done, (size_t)2 * NN, err)))
    return rc;
  return IETI_OK;
}

// Multifrontal FP64 factorization of S_c (nc x nc, rows and columns in elimination
// order) along the tree, level by level in height: each node's front [K | S | K'] is
// the original K columns of S_c, the children's update matrices added (in child
// order: deterministic), and identity rows K'; one batched partial Cholesky of the
// nk pivots of all fronts of a level leaves the update matrix in [S S], -Lbar^T in
// [K' S] and -D^{-1} in [K' K'], which are extracted into d->nd_Z / d->nd_Lt.
static int coarse_nd_factor(DeviceState *d, const CoarseTree &t, const double *Sc, std::string &err) {
  const int NN = t.n_nodes;
  const int64_t nc = d->NC;
  cudaStream_t st = d->stream;
  std::vector<int64_t> foff(NN + 1, 0), fidoff(NN + 1, 0), eaoff(NN + 1, 0);
  std::vector<int32_t> na(NN), fid, ea;
  for (int p = 0; p < NN; ++p) {
    na[p] = 2 * t.nk[p] + t.ns[p];
    foff[p + 1] = foff[p] + (int64_t)na[p] * na[p];
    for (int k = 0; k < t.nk[p]; ++k) fid.push_back(t.k0[p] + k);
    for (int64_t k = t.s_off[p]; k < t.s_off[p + 1]; ++k) fid.push_back(t.s_idx[k]);
    fidoff[p + 1] = (int64_t)fid.size();
    if (t.parent[p] >= 0)
      for (int64_t k = t.s_off[p]; k < t.s_off[p + 1]; ++k) ea.push_back(t.front_index(t.parent[p], t.s_idx[k]));
    eaoff[p + 1] = (int64_t)ea.size();
  }
  if (fid.empty()) fid.push_back(0);
  if (ea.empty()) ea.push_back(0);
  double *F = nullptr;
  int32_t *dfid = nullptr, *dea = nullptr;
  unsigned char *blk = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(F);
    cudaFree(dfid);
    cudaFree(dea);
    cudaFree(blk);
  };
  const size_t fbytes = (size_t)std::max<int64_t>(foff[NN], 1) * sizeof(double);
  if (cudaMalloc((void **)&F, fbytes) != cudaSuccess || cudaMalloc((void **)&dfid, fid.size() * 4) != cudaSuccess ||
      cudaMalloc((void **)&dea, ea.size() * 4) != cudaSuccess ||
      cudaMalloc((void **)&blk, (size_t)NN * (8 + 9 * 4)) != cudaSuccess) {
    cleanup();
    err = "cudaMalloc failed for the nested-dissection fronts (" + std::to_string(fbytes >> 20) + " MiB)";
    return IETI_ERR_OOM;
  }
  int64_t *doff = (int64_t *)blk;
  int32_t *dld = (int32_t *)(doff + NN), *dkb = dld + NN, *dke = dkb + NN, *dna = dke + NN, *dstat = dna + NN,
          *dz = dstat + NN, *dbig = dz + NN, *dz2 = dbig + NN;
  cudaError_t e = cudaMemsetAsync(F, 0, fbytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dfid, fid.data(), fid.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dea, ea.data(), ea.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dstat, 0, (size_t)NN * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dz, 0, (size_t)NN * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dz2, 0, (size_t)NN * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dbig, 0x7f, (size_t)NN * 4, st);
  if (e != cudaSuccess) {
    cleanup();
    err = std::string("nested-dissection setup failed: ") + cudaGetErrorString(e);
    return IETI_ERR_CUDA;
  }
  for (int p = 0; p < NN; ++p) {
    const int64_t cnt = std::max<int64_t>((int64_t)(t.nk[p] + t.ns[p]) * t.nk[p], t.nk[p]);
    if (cnt > 0)
      k_front_init<<<grid_for(cnt, 256), 256, 0, st>>>(Sc, nc, dfid + fidoff[p], t.nk[p], t.ns[p], F + foff[p],
                                                       na[p]);
    d->launches_setup++;
  }
  AugLimits lim{dz, dz2, dbig, dz};
  int rc = IETI_OK;
  for (int h = 0; h < d->nd_H && rc == IETI_OK; ++h) {
    const std::vector<int32_t> &L = d->ndh_fwd[h];
    std::vector<int64_t> hoff;
    std::vector<int32_t> hld, hkb, hke, hna;
    for (int p : L) {
      for (int k = t.child_ptr[p]; k < t.child_ptr[p + 1]; ++k) {
        const int ch = t.child_idx[k];
        const int64_t cnt = (int64_t)t.ns[ch] * t.ns[ch];
        if (cnt == 0) continue;
        k_extend_add<<<grid_for(cnt, 256), 256, 0, st>>>(F + foff[ch], na[ch], t.nk[ch], t.ns[ch], dea + eaoff[ch],
                                                         F + foff[p], na[p]);
        d->launches_setup++;
      }
      hoff.push_back(foff[p]);
      hld.push_back(na[p]);
      hkb.push_back(0);
      hke.push_back(t.nk[p]);
      hna.push_back(na[p]);
    }
    const int nb = (int)L.size();
    e = cudaMemcpyAsync(doff, hoff.data(), nb * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dld, hld.data(), nb * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dkb, hkb.data(), nb * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dke, hke.data(), nb * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dna, hna.data(), nb * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      err = std::string("nested-dissection setup failed: ") + cudaGetErrorString(e);
      rc = IETI_ERR_CUDA;
      break;
    }
    rc = potrf_partial<double>(d, F, doff, dld, hkb, hke, hna, dkb, dke, dna, dstat, lim, err);
    if (rc == IETI_OK) {
      std::vector<int32_t> hst(nb);
      e = cudaMemcpyAsync(hst.data(), dstat, nb * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        err = std::string("nested-dissection factorization failed: ") + cudaGetErrorString(e);
        rc = IETI_ERR_CUDA;
      }
      for (int b = 0; b < nb && rc == IETI_OK; ++b)
        if (hst[b]) {
          err = "coarse Schur complement is not positive definite (nested-dissection node " + std::to_string(L[b]) +
                ", pivot " + std::to_string(hst[b] - 1) + ")";
          rc = IETI_ERR_NOT_SPD;
        }
    }
  }
  if (rc == IETI_OK) {
    int64_t zo = 0, lo = 0;
    for (int p = 0; p < NN; ++p) {
      const int64_t cnt = (int64_t)(t.nk[p] + t.ns[p]) * t.nk[p] + (int64_t)t.nk[p] * t.ns[p];
      if (cnt > 0)
        k_front_extract<<<grid_for(cnt, 256), 256, 0, st>>>(F + foff[p], na[p], t.nk[p], t.ns[p], d->nd_Z + zo,
                                                            d->ndh_zld[p], d->nd_Lt + lo, d->ndh_ltld[p]);
      d->launches_setup++;
      zo += (int64_t)(t.nk[p] + t.ns[p]) * d->ndh_zld[p];
      lo += (int64_t)t.nk[p] * d->ndh_ltld[p];
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      err = std::string("nested-dissection extraction failed: ") + cudaGetErrorString(e);
      rc = IETI_ERR_CUDA;
    }
  }
  cleanup();
  return rc;
}

// FP64 partial Cholesky of the assembled [[S_c, I], [I, 0]] (2 nc x 2 nc, row-major)
// and extraction of S_c^{-1} into the per-iteration slot (FP32 (hi, lo) pairs in the
// mixed path).  The descriptor words are allocated once and reused.
static int coarse_factor(DeviceState *d, double *Sc, std::string &err) {
  const int64_t nc = d->NC, ldc = 2 * nc;
  int rc;
  if (!d->c_off) {
    std::vector<int64_t> hcoff{0};
    std::vector<int32_t> hcld{(int32_t)ldc}, hckb{0}, hcke{(int32_t)nc}, hcna{(int32_t)ldc}, hz{0},
        hbig{INT32_MAX};
    if ((rc = upload(d, &d->c_off, hcoff, err)) || (rc = upload(d, &d->c_ld, hcld, err)) ||
        (rc = upload(d, &d->c_kb, hckb, err)) || (rc = upload(d, &d->c_ke, hcke, err)) ||
        (rc = upload(d, &d->c_na, hcna, err)) || (rc = upload(d, &d->c_st, hz, err)) ||
        (rc = upload(d, &d->c_z, hz, err)) || (rc = upload(d, &d->c_big, hbig, err)))
      return rc;
  }
  CK(cudaMemsetAsync(d->c_st, 0, 4, d->stream));
  std::vector<int32_t> hckb{0}, hcke{(int32_t)nc}, hcna{(int32_t)ldc};
  AugLimits clim_{d->c_z, d->c_z, d->c_big, d->c_z};
  if ((rc = potrf_partial<double>(d, Sc, d->c_off, d->c_ld, hckb, hcke, hcna, d->c_kb, d->c_ke, d->c_na, d->c_st,
                                  clim_, err)))
    return rc;
  int32_t cstat = 0;
  CK(cudaMemcpyAsync(&cstat, d->c_st, 4, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  if (cstat) {
    err = "coarse Schur complement is not positive definite (pivot " + std::to_string(cstat - 1) + ")";
    return IETI_ERR_NOT_SPD;
  }
  if (!d->Sinv) {
    if ((rc = dalloc(d, &d->Sinv, (size_t)(nc * d->ldc), err))) return rc;
    CK(cudaMemsetAsync(d->Sinv, 0, (size_t)(nc * d->ldc) * sizeof(double), d->stream));
  }
  k_coarse_extract<double><<<grid_for(nc * nc, 256), 256, 0, d->stream>>>((int)nc, Sc, ldc, d->Sinv, d->ldc);
  return coarse_publish(d, err);
}

// S_c^{-1} (d->Sinv) -> the per-iteration slot: FP32 (hi, lo) pairs (mixed) or FP64
static int coarse_publish(DeviceState *d, std::string &err) {
  const int64_t nc = d->NC;
  if (d->mixed) {
    d->Sdf = d->Scoarse_slot;
    k_split_pairs<<<grid_for(nc * d->ldc, 256), 256, 0, d->stream>>>(nc * d->ldc, d->Sinv, (float2 *)d->Sdf);
  } else {
    CK(cudaMemcpyAsync(d->Scoarse_slot, d->Sinv, (size_t)(nc * d->ldc) * sizeof(double), cudaMemcpyDeviceToDevice,
                       d->stream));
  }
  d->launches_setup += 2;
  CK(cudaGetLastError());
  return IETI_OK;
}

// inverse of an SPD n x n block from its assembled augmentation aug = [[S, I], [I, 0]]
// (2n x 2n, row-major): FP64 partial Cholesky of the first n pivots leaves -S^{-1}
// in the trailing block; out (n x n, leading dimension ldo) receives S^{-1}
static int spd_inverse(DeviceState *d, double *aug, int n, double *out, int ldo, std::string &err) {
  static_assert(sizeof(int64_t) == 8, "");
  int64_t *off = nullptr;
  int32_t *w = nullptr;
  CK(cudaMalloc((void **)&off, sizeof(int64_t) + 8 * sizeof(int32_t)));
  w = (int32_t *)(off + 1);
  int32_t hw[8] = {2 * n, 0, n, 2 * n, 0, 0, INT32_MAX, 0};  // ld, kb, ke, na, status, zero, big, zero
  int64_t h0 = 0;
  cudaError_t e = cudaMemcpyAsync(off, &h0, 8, cudaMemcpyHostToDevice, d->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w, hw, sizeof(hw), cudaMemcpyHostToDevice, d->stream);
  if (e != cudaSuccess) {
    cudaFree(off);
    err = "spd_inverse upload failed";
    return IETI_ERR_CUDA;
  }
  std::vector<int32_t> hkb{0}, hke{n}, hna{2 * n};
  AugLimits lim{w + 5, w + 5, w + 6, w + 7};
  int rc = potrf_partial<double>(d, aug, off, w, hkb, hke, hna, w + 1, w + 2, w + 3, w + 4, lim, err);
  int32_t st = 0;
  if (rc == IETI_OK) {
    e = cudaMemcpyAsync(&st, w + 4, 4, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) {
      err = std::string("spd_inverse failed: ") + cudaGetErrorString(e);
      rc = IETI_ERR_CUDA;
    } else if (st) {
      err = "coarse block is not positive definite (pivot " + std::to_string(st - 1) + ")";
      rc = IETI_ERR_NOT_SPD;
    }
  }
  if (rc == IETI_OK)
    k_coarse_extract<double><<<grid_for((int64_t)n * n, 256), 256, 0, d->stream>>>(n, aug, 2 * n, out, ldo);
  cudaStreamSynchronize(d->stream);
  cudaFree(off);
  return rc;
}

static void dgemm(DeviceState *d, bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int64_t lda,
                  const double *B, int64_t ldb, double beta, double *C, int64_t ldc) {
  dim3 g((N + 63) / 64, (M + 63) / 64);
  if (!ta && !tb) k_dgemm<false, false><<<g, 256, 0, d->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (ta && !tb) k_dgemm<true, false><<<g, 256, 0, d->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (!ta && tb) k_dgemm<false, true><<<g, 256, 0, d->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else k_dgemm<true, true><<<g, 256, 0, d->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// Split of the coarse unknowns for the Newton refactorizations: N = the primal
// unknowns of the patches holding nonlinear elements (only S_NN changes between
// refactorizations), L = the rest.  Precomputes inv(S_LL), X = inv(S_LL) S_LN and
// Z0 = S_NN(linear part) - S_NL X from the linear patches' part of S_c.
static int coarse_block_setup(DeviceState *d, const std::vector<int32_t> &hpc, std::string &err) {
  const int64_t nc = d->NC;
  std::vector<int32_t> posN(nc, -1), idxL, idxN, pcN;
  for (int b = 0; b < d->nl_np; ++b)
    for (int k = 0; k < d->nlh_np[b]; ++k) posN[hpc[d->nlh_pofs[b] + k]] = 0;
  for (int64_t c = 0; c < nc; ++c) {
    if (posN[c] == 0) {
      posN[c] = (int32_t)idxN.size();
      idxN.push_back((int32_t)c);
    } else {
      idxL.push_back((int32_t)c);
    }
  }
  for (int b = 0; b < d->nl_np; ++b) {
    d->nlh_pcN.push_back((int64_t)pcN.size());
    for (int k = 0; k < d->nlh_np[b]; ++k) pcN.push_back(posN[hpc[d->nlh_pofs[b] + k]]);
  }
  const int cL = (int)idxL.size(), cN = (int)idxN.size();
  // the split pays only when the changing block is a minor part of S_c: its cost is
  // that of inverting Z (cN) plus GEMMs of cL^2 cN, against a factorization of 2 nc
  if (cL == 0 || cN == 0 || 2 * cN > nc) return IETI_OK;  // full refactorizations
  int rc;
  if ((rc = upload(d, &d->c_idxL, idxL, err)) || (rc = upload(d, &d->c_idxN, idxN, err)) ||
      (rc = upload(d, &d->nl_pcN, pcN, err)) || (rc = dalloc(d, &d->c_SLLinv, (size_t)cL * cL, err)) ||
      (rc = dalloc(d, &d->c_X, (size_t)cL * cN, err)) || (rc = dalloc(d, &d->c_Z0, (size_t)cN * cN, err)) ||
      (rc = dalloc(d, &d->c_Zaug, (size_t)4 * cN * cN, err)) || (rc = dalloc(d, &d->c_Zinv, (size_t)cN * cN, err)) ||
      (rc = dalloc(d, &d->c_Y, (size_t)cL * cN, err)) || (rc = dalloc(d, &d->c_Ltmp, (size_t)cL * cL, err)))
    return rc;
  double *tmpL = nullptr, *augL = nullptr, *SLN = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(d->stream);
    cudaFree(tmpL);
    cudaFree(augL);
    cudaFree(SLN);
  };
  if (cudaMalloc((void **)&tmpL, (size_t)cL * cL * 8) != cudaSuccess ||
      cudaMalloc((void **)&augL, (size_t)4 * cL * cL * 8) != cudaSuccess ||
      cudaMalloc((void **)&SLN, (size_t)cL * cN * 8) != cudaSuccess) {
    cleanup();
    err = "cudaMalloc failed for the coarse block split";
    return IETI_ERR_OOM;
  }
  cudaStream_t st = d->stream;
  k_gather_block<<<grid_for((int64_t)cL * cL, 256), 256, 0, st>>>(cL, cL, d->c_idxL, d->c_idxL, d->sc_lin, nc, tmpL,
                                                                   cL);
  k_aug_identity_block<<<grid_for((int64_t)4 * cL * cL, 256), 256, 0, st>>>(cL, tmpL, cL, augL);
  if ((rc = spd_inverse(d, augL, cL, d->c_SLLinv, cL, err))) {
    cleanup();
    return rc;
  }
  k_gather_block<<<grid_for((int64_t)cL * cN, 256), 256, 0, st>>>(cL, cN, d->c_idxL, d->c_idxN, d->sc_lin, nc, SLN,
                                                                   cN);
  dgemm(d, false, false, cL, cN, cL, 1.0, d->c_SLLinv, cL, SLN, cN, 0.0, d->c_X, cN);
  k_gather_block<<<grid_for((int64_t)cN * cN, 256), 256, 0, st>>>(cN, cN, d->c_idxN, d->c_idxN, d->sc_lin, nc,
                                                                   d->c_Z0, cN);
  dgemm(d, true, false, cN, cN, cL, -1.0, SLN, cN, d->c_X, cN, 1.0, d->c_Z0, cN);
  cudaError_t e = cudaGetLastError();
  cleanup();
  if (e != cudaSuccess) {
    err = std::string("coarse block split failed: ") + cudaGetErrorString(e);
    return IETI_ERR_CUDA;
  }
  d->cL = cL;
  d->cN = cN;
  return IETI_OK;
}

// S_c^{-1} after a refactorization of the nonlinear patches, by the block formula
// with Z = Z0 + sum over those patches of their C_s (on N):
// S^{-1} = [[inv(S_LL) + X inv(Z) X^T, -X inv(Z)], [-inv(Z) X^T, inv(Z)]]
template <class TD>
static int coarse_block_refactor(DeviceState *d, const TD *W, std::string &err) {
  cudaStream_t st = d->stream;
  const int cL = d->cL, cN = d->cN;
  const int64_t ldz = 2 * (int64_t)cN;
  k_aug_identity_block<<<grid_for(ldz * ldz, 256), 256, 0, st>>>(cN, d->c_Z0, cN, d->c_Zaug);
  for (int b = 0; b < d->nl_np; ++b) {
    if (d->nlh_np[b] == 0) continue;
    int64_t cnt = (int64_t)d->nlh_np[b] * d->nlh_np[b];
    k_coarse_add<TD><<<grid_for(cnt, 256), 256, 0, st>>>(W, d->nlh_doff[b], d->nlh_nn[b], d->nlh_ni[b], d->nlh_nb[b],
                                                         d->nlh_np[b], d->nl_pcN + d->nlh_pcN[b], d->c_Zaug, ldz);
  }
  int rc;
  if ((rc = spd_inverse(d, d->c_Zaug, cN, d->c_Zinv, cN, err))) return rc;
  dgemm(d, false, false, cL, cN, cN, 1.0, d->c_X, cN, d->c_Zinv, cN, 0.0, d->c_Y, cN);
  CK(cudaMemcpyAsync(d->c_Ltmp, d->c_SLLinv, (size_t)cL * cL * 8, cudaMemcpyDeviceToDevice, st));
  dgemm(d, false, true, cL, cL, cN, 1.0, d->c_Y, cN, d->c_X, cN, 1.0, d->c_Ltmp, cL);
  k_scatter_block<<<grid_for((int64_t)cL * cL, 256), 256, 0, st>>>(cL, cL, d->c_idxL, d->c_idxL, d->c_Ltmp, cL, 1.0,
                                                                    0, d->Sinv, d->ldc);
  k_scatter_block<<<grid_for((int64_t)cL * cN, 256), 256, 0, st>>>(cL, cN, d->c_idxL, d->c_idxN, d->c_Y, cN, -1.0,
                                                                    1, d->Sinv, d->ldc);
  k_scatter_block<<<grid_for((int64_t)cN * cN, 256), 256, 0, st>>>(cN, cN, d->c_idxN, d->c_idxN, d->c_Zinv, cN, 1.0,
                                                                    0, d->Sinv, d->ldc);
  CK(cudaGetLastError());
  return coarse_publish(d, err);
}

// ---------------------------------------------------------------------------
// Nonlinear reluctivity: refactorization of the patches holding nonlinear elements
// at the current state d->a (their blocks W (without the law) + dt K_t(a)), then the
// coarse block S_c = (sum over the linear patches, kept from setup) + theirs.
template <class TD, class TO>  // dense arena type, operator type
static int nl_refactor(DeviceState *d, std::string &err) {
  cudaStream_t st = d->stream;
  cudaEvent_t ev[4] = {};
  if (d->opt.profile)
    for (auto &e : ev) {
      cudaEventCreate(&e);
    }
  if (ev[0]) cudaEventRecord(ev[0], st);
  const int nb = d->nl_np;
  TD *W = (TD *)d->nl_work;
  CK(cudaMemcpyAsync(d->nl_work, d->nl_base, (size_t)d->nl_arena * sizeof(TD), cudaMemcpyDeviceToDevice, st));
  {
    size_t sm = (size_t)(d->nl_max_nloc + 4 * d->nl_max_nq) * sizeof(double);
    k_nl_eval<<<(unsigned)d->nl_ne, 128, sm, st>>>(d->nl_G, d->nl_cq, d->nl_kept, d->nl_glob, d->nl_goff,
                                                   d->nl_qoff, d->nl_doff, d->nl_nloc, d->nl_nq, d->nl_bpos,
                                                   d->nlb_kofs, d->a, d->law, d->dt, nullptr, d->nl_tq, 2);
    size_t sm2 = (size_t)NL_QC * d->nl_max_nloc * sizeof(float4);
    k_nl_tangent<TD><<<(unsigned)d->nl_ne, NL_TB, sm2, st>>>(d->nl_G, d->nl_kept, d->nl_goff, d->nl_qoff,
                                                             d->nl_doff, d->nl_nloc, d->nl_nq, d->nl_bpos, d->nl_tq,
                                                             d->nlb_doff, d->nlb_nn, d->dt, W);
    d->nlaunch += 2;
  }
  CK(cudaGetLastError());
  if (ev[1]) cudaEventRecord(ev[1], st);
  // phase A: interior pivots; copy S_bb
  std::vector<int32_t> hkb(nb), hke(nb), hna(nb);
  TcHost th;
  th.off = d->nlh_doff;
  th.ld = d->nlh_nn;
  th.sk_lo.resize(nb);
  th.sk_hi.resize(nb);
  th.rlim.assign(nb, INT32_MAX);
  th.clim.assign(nb, 0);
  for (int b = 0; b < nb; ++b) {
    hkb[b] = 0;
    hke[b] = d->nlh_ni[b];
    hna[b] = d->nlh_nn[b];
    th.sk_lo[b] = d->nlh_n[b];
    th.sk_hi[b] = d->nlh_n[b] + d->nlh_nb[b];
  }
  auto put = [&](int32_t *dst, const std::vector<int32_t> &h) -> int {
    CK(cudaMemcpyAsync(dst, h.data(), nb * 4, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return IETI_OK;
  };
  int rc;
  if ((rc = put(d->nlb_kb, hkb)) || (rc = put(d->nlb_ke, hke)) || (rc = put(d->nlb_na, hna)) ||
      (rc = put(d->nlb_sklo, th.sk_lo)) || (rc = put(d->nlb_skhi, th.sk_hi)) || (rc = put(d->nlb_rlim, th.rlim)) ||
      (rc = put(d->nlb_clim, th.clim)))
    return rc;
  CK(cudaMemsetAsync(d->nlb_st, 0, nb * 4, st));
  AugLimits lim{d->nlb_sklo, d->nlb_skhi, d->nlb_rlim, d->nlb_clim};
  if ((rc = run_partial<TD>(d, W, d->nlb_doff, d->nlb_nn, th, hkb, hke, hna, d->nlb_kb, d->nlb_ke, d->nlb_na,
                            d->nlb_st, lim, err)))
    return rc;
  int maxnb = 1, maxnp = 1;
  int64_t maxH = 1, maxIG = 1;
  for (int b = 0; b < nb; ++b) {
    maxnb = std::max(maxnb, d->nlh_nb[b]);
    maxnp = std::max(maxnp, d->nlh_np[b]);
    maxH = std::max(maxH, (int64_t)(d->nlh_nb[b] + d->nlh_np[b]) * d->nlh_nb[b]);
    maxIG = std::max(maxIG, (int64_t)d->nlh_n[b] * d->nlh_ni[b]);
  }
  {
    dim3 g(grid_for((int64_t)maxnb * maxnb, 256), nb);
    k_extract_P<TD, TO><<<g, 256, 0, st>>>(W, d->nlb_doff, d->nlb_nn, d->nlb_ni, d->nlb_nb, d->nlb_ldb,
                                           d->nlb_poff, (TO *)d->P);
  }
  // phase B: interface pivots
  for (int b = 0; b < nb; ++b) {
    hkb[b] = d->nlh_ni[b];
    hke[b] = d->nlh_ni[b] + d->nlh_nb[b];
    hna[b] = d->nlh_n[b] + d->nlh_nb[b];
    th.sk_lo[b] = th.sk_hi[b] = 0;
  }
  if ((rc = put(d->nlb_kb, hkb)) || (rc = put(d->nlb_ke, hke)) || (rc = put(d->nlb_na, hna)) ||
      (rc = put(d->nlb_sklo, th.sk_lo)) || (rc = put(d->nlb_skhi, th.sk_hi)))
    return rc;
  if ((rc = run_partial<TD>(d, W, d->nlb_doff, d->nlb_nn, th, hkb, hke, hna, d->nlb_kb, d->nlb_ke, d->nlb_na,
                            d->nlb_st, lim, err)))
    return rc;
  {
    std::vector<int32_t> hst(nb);
    CK(cudaMemcpyAsync(hst.data(), d->nlb_st, nb * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int b = 0; b < nb; ++b)
      if (hst[b]) {
        err = "Newton tangent block of patch " + std::to_string(d->nlh_ids[b]) +
              " is not positive definite (pivot " + std::to_string(hst[b] - 1) + ")";
        return IETI_ERR_NOT_SPD;
      }
  }
  {
    dim3 g((unsigned)std::min<int64_t>(grid_for(maxH, 256), 4096), nb);
    k_extract_ops<TD, TO><<<g, 256, 0, st>>>(W, d->nlb_doff, d->nlb_nn, d->nlb_ni, d->nlb_nb, d->nlb_np, d->nlb_ldb,
                                             d->nlb_ldp, d->nlb_hoff, d->nlb_qoff, (TO *)d->H, (TO *)d->Q);
    dim3 g2((unsigned)std::min<int64_t>(grid_for(maxIG, 256), 4096), nb);
    k_extract_IG<TD, TO><<<g2, 256, 0, st>>>(W, d->nlb_doff, d->nlb_nn, d->nlb_ni, d->nlb_nb, d->nlb_np, d->nlb_ldi,
                                             d->nlb_ldg, d->nlb_igoff, d->nlb_gtoff, (TO *)d->IG, (TO *)d->GT);
  }
  if (ev[2]) cudaEventRecord(ev[2], st);
  // coarse: along the nested dissection (linear part + the refactored patches, the
  // multifrontal FP64 factorization), by the block formula when the split exists, else
  // linear part + the refactored patches and a full factorization of the augmented block
  if (d->NC > 0 && d->coarse_nd) {
    const int64_t nc = d->NC;
    CK(cudaMemcpyAsync(d->sc_aug, d->sc_lin, (size_t)(nc * nc) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int b = 0; b < nb; ++b) {
      if (d->nlh_np[b] == 0) continue;
      int64_t cnt = (int64_t)d->nlh_np[b] * d->nlh_np[b];
      k_coarse_add<TD><<<grid_for(cnt, 256), 256, 0, st>>>(W, d->nlh_doff[b], d->nlh_nn[b], d->nlh_ni[b],
                                                           d->nlh_nb[b], d->nlh_np[b], d->pc + d->nlh_pofs[b],
                                                           d->sc_aug, nc);
    }
    if ((rc = coarse_nd_factor(d, *d->nd_tree, d->sc_aug, err))) return rc;
    if (d->mixed) {
      const int64_t n = d->nd_z_elems + d->nd_lt_elems;
      k_split_pairs<<<grid_for(n, 256), 256, 0, st>>>(n, d->nd_Z, (float2 *)d->nd_Z);
    }
  } else if (d->NC > 0 && d->cN > 0) {
    if ((rc = coarse_block_refactor<TD>(d, W, err))) return rc;
  } else if (d->NC > 0 && d->mixed && d->factor != IETI_FACTOR_FP64) {
    // the Newton iterate's coarse block in the factor arithmetic of the patches (a
    // Newton step is an inexact solve; its residual stays FP64): assembled in FP64,
    // rounded, factored by the batched FP32 / tensor-core partial Cholesky
    const int64_t nc = d->NC, ldc = 2 * nc;
    CK(cudaMemsetAsync(d->sc_aug, 0, (size_t)(ldc * ldc) * sizeof(double), st));
    CK(cudaMemcpy2DAsync(d->sc_aug, ldc * sizeof(double), d->sc_lin, nc * sizeof(double), nc * sizeof(double), nc,
                         cudaMemcpyDeviceToDevice, st));
    for (int b = 0; b < nb; ++b) {
      if (d->nlh_np[b] == 0) continue;
      int64_t cnt = (int64_t)d->nlh_np[b] * d->nlh_np[b];
      k_coarse_add<TD><<<grid_for(cnt, 256), 256, 0, st>>>(W, d->nlh_doff[b], d->nlh_nn[b], d->nlh_ni[b],
                                                           d->nlh_nb[b], d->nlh_np[b], d->pc + d->nlh_pofs[b],
                                                           d->sc_aug, ldc);
    }
    k_coarse_identity<<<grid_for(nc, 256), 256, 0, st>>>((int)nc, d->sc_aug, ldc);
    if (!d->sc_aug32) {
      d->ld32 = (ldc + 3) / 4 * 4;
      float *p = nullptr;
      if ((rc = dalloc(d, &p, (size_t)(ldc * d->ld32), err))) return rc;
      d->sc_aug32 = p;
    }
    k_round_lower<<<grid_for(ldc * ldc, 256), 256, 0, st>>>(ldc, d->sc_aug, ldc, d->sc_aug32, d->ld32);
    std::vector<int32_t> ckb{0}, cke{(int32_t)nc}, cna{(int32_t)ldc};
    TcHost cth;
    cth.off = {0};
    cth.ld = {(int32_t)d->ld32};
    cth.sk_lo = {0};
    cth.sk_hi = {0};
    cth.rlim = {INT32_MAX};
    cth.clim = {0};
    int32_t hld = (int32_t)d->ld32;
    CK(cudaMemcpyAsync(d->c_ld, &hld, 4, cudaMemcpyHostToDevice, st));  // coarse descriptor: FP32 leading dim
    CK(cudaMemsetAsync(d->c_st, 0, 4, st));
    AugLimits clim_{d->c_z, d->c_z, d->c_big, d->c_z};
    rc = run_partial<float>(d, d->sc_aug32, d->c_off, d->c_ld, cth, ckb, cke, cna, d->c_kb, d->c_ke, d->c_na,
                            d->c_st, clim_, err);
    int32_t hld2 = (int32_t)ldc;
    CK(cudaMemcpyAsync(d->c_ld, &hld2, 4, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (rc) return rc;
    int32_t cstat = 0;
    CK(cudaMemcpyAsync(&cstat, d->c_st, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (cstat) {
      err = "Newton coarse block is not positive definite in FP32 (pivot " + std::to_string(cstat - 1) + ")";
      return IETI_ERR_NOT_SPD;
    }
    k_coarse_extract<float><<<grid_for(nc * nc, 256), 256, 0, st>>>((int)nc, d->sc_aug32, d->ld32, d->Sinv, d->ldc);
    if ((rc = coarse_publish(d, err))) return rc;
  } else if (d->NC > 0) {
    const int64_t nc = d->NC, ldc = 2 * nc;
    CK(cudaMemsetAsync(d->sc_aug, 0, (size_t)(ldc * ldc) * sizeof(double), st));
    CK(cudaMemcpy2DAsync(d->sc_aug, ldc * sizeof(double), d->sc_lin, nc * sizeof(double), nc * sizeof(double), nc,
                         cudaMemcpyDeviceToDevice, st));
    for (int b = 0; b < nb; ++b) {
      if (d->nlh_np[b] == 0) continue;
      int64_t cnt = (int64_t)d->nlh_np[b] * d->nlh_np[b];
      k_coarse_add<TD><<<grid_for(cnt, 256), 256, 0, st>>>(W, d->nlh_doff[b], d->nlh_nn[b], d->nlh_ni[b],
                                                           d->nlh_nb[b], d->nlh_np[b], d->pc + d->nlh_pofs[b],
                                                           d->sc_aug, ldc);
    }
    k_coarse_identity<<<grid_for(nc, 256), 256, 0, st>>>((int)nc, d->sc_aug, ldc);
    if ((rc = coarse_factor(d, d->sc_aug, err))) return rc;
  }
  CK(cudaGetLastError());
  if (ev[3]) {
    cudaEventRecord(ev[3], st);
    cudaEventSynchronize(ev[3]);
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    cudaEventElapsedTime(&c, ev[2], ev[3]);
    d->t_refactor_ms[0] += a;
    d->t_refactor_ms[1] += b;
    d->t_refactor_ms[2] += c;
    d->t_refactor_ms[3] += a + b + c;
    for (auto &e : ev) cudaEventDestroy(e);
  }
  d->refactors++;
  d->step_refactors++;
  return IETI_OK;
}

static int nl_refactor_any(DeviceState *d, std::string &err) {
  if (!d->mixed) return nl_refactor<double, double>(d, err);
  if (d->factor == IETI_FACTOR_FP64) return nl_refactor<double, float>(d, err);
  return nl_refactor<float, float>(d, err);
}

// ---------------------------------------------------------------------------
// the condensed interface solve: given u (B-space) and gp (Pi-space, may be
// null): bp[0:NBt] = F u - Psi q, q = S_c^{-1} sum_s A_s^T (gp - Psi^T u)
template <class T>
static void condensed(DeviceState *d, const double *u, const double *gp) {
  cudaStream_t st = d->stream;
  gemv<T>(d, d->dH, d->H, u, d->bp, nullptr, 1.0, 0.0, IETI_K_GEMV_H);
  if (d->NC > 0) {
    k_coarse_gather<<<grid_for(d->NC, 256), 256, 0, st>>>((int)d->NC, d->cptr, d->cpos, gp, d->bp + d->NBt, d->cc);
    d->nlaunch++;
    gemv<double>(d, d->dS, d->Sinv, d->cc, d->q, nullptr, 1.0, 0.0, IETI_K_GEMV_S);
    k_pgather<<<grid_for(d->NPt, 256), 256, 0, st>>>(d->NPt, d->pc, d->q, d->qloc);
    d->nlaunch++;
    gemv<T>(d, d->dQ, d->Q, d->qloc, d->bp, d->bp, -1.0, 1.0, IETI_K_GEMV_Q);
  }
}

template <class T>
static void apply_F(DeviceState *d, const double *v, double *out, const double *dotv, double *part) {
  cudaStream_t st = d->stream;
  k_Bt<<<grid_for(d->NBt, 256), 256, 0, st>>>(d->NBt, d->bt_ptr, d->bt_lam, d->bt_sgn, v, nullptr, 1.0, d->ub);
  d->nlaunch++;
  condensed<T>(d, d->ub, nullptr);
  k_jump<<<RED_BLOCKS, 256, 0, st>>>(d->M, d->lam_qp, d->lam_qm, nullptr, nullptr, d->bp, out, dotv, part);
  d->nlaunch++;
}

// ---- balanced (deflated) preconditioner  M_bal = (I - P) M (I - P)^T + U E^{-1} U^T,
// P = U E^{-1} U^T F, E = U^T F U, U the patch-pair indicator space of the multipliers

// ur[j] = sum of v over the multipliers of pair j (one block per pair)
__global__ void k_pair_sums(int k, const int32_t *ptr, const int32_t *lam, const double *v, double *ur) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  if (j >= k) return;
  double acc = 0.0;
  for (int t = ptr[j] + threadIdx.x; t < ptr[j + 1]; t += blockDim.x) acc += v[lam[t]];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    ur[j] = t;
  }
}

// c = Einv (a - b)   (b may be null; k x k row-major, thread per row)
__global__ void k_small_gemv(int k, const double *Einv, const double *a, const double *b, double *c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double acc = 0.0;
  for (int j = 0; j < k; ++j) acc += Einv[(int64_t)i * k + j] * (b ? a[j] - b[j] : a[j]);
  c[i] = acc;
}

// out[l] = v[l] - sum_j FUt[j][l] c[j]   (thread per multiplier, the k rows read coalesced)
__global__ void k_defl_sub(int64_t m, int k, const double *FUt, const double *c, const double *v, double *out) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= m) return;
  double acc = v[l];
  for (int j = 0; j < k; ++j) acc -= FUt[(int64_t)j * m + l] * c[j];
  out[l] = acc;
}

// fw[j] = FUt[j] . w   (one block per row)
__global__ void k_defl_dots(int64_t m, int k, const double *FUt, const double *w, double *fw) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  if (j >= k) return;
  const double *row = FUt + (int64_t)j * m;
  double acc = 0.0;
  for (int64_t l = threadIdx.x; l < m; l += blockDim.x) acc += row[l] * w[l];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    fw[j] = t;
  }
}

// out[l] = w[l] + c[pair[l]]; partial sums of out . dotv (PCG's (r, z))
__global__ void k_defl_finish(int64_t m, const int32_t *pair, const double *w, const double *c, double *out,
                              const double *dotv, double *part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < m; l += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[l] + c[pair[l]];
    out[l] = v;
    if (dotv) acc += v * dotv[l];
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// v[l] = (pair[l] == j)
__global__ void k_pair_indicator(int64_t m, const int32_t *pair, int j, double *v) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l < m) v[l] = pair[l] == j ? 1.0 : 0.0;
}

template <class T>
static void apply_dirichlet(DeviceState *d, const double *rv, double *out, const double *dotv, double *part);

template <class T>
static void apply_precond(DeviceState *d, const double *rv, double *out, const double *dotv, double *part) {
  if (d->defl_k == 0) {
    apply_dirichlet<T>(d, rv, out, dotv, part);
    return;
  }
  cudaStream_t st = d->stream;
  const int64_t m = d->M;
  const int k = d->defl_k;
  k_pair_sums<<<k, 128, 0, st>>>(k, d->defl_ptr, d->defl_lam, rv, d->defl_ur);          // U^T r
  k_small_gemv<<<grid_for(k, 128), 128, 0, st>>>(k, d->defl_Einv, d->defl_ur, nullptr, d->defl_c);
  k_defl_sub<<<grid_for(m, 256), 256, 0, st>>>(m, k, d->defl_FUt, d->defl_c, rv, d->defl_rh);  // (I - P)^T r
  apply_dirichlet<T>(d, d->defl_rh, d->defl_w, rv, part);                                 // w = M (...)
  k_defl_dots<<<k, 256, 0, st>>>(m, k, d->defl_FUt, d->defl_w, d->defl_fw);              // (F U)^T w
  k_small_gemv<<<grid_for(k, 128), 128, 0, st>>>(k, d->defl_Einv, d->defl_ur, d->defl_fw, d->defl_c);
  k_defl_finish<<<RED_BLOCKS, 256, 0, st>>>(m, d->defl_pair, d->defl_w, d->defl_c, out, dotv, part);
  d->nlaunch += 6;
}

template <class T>
static void apply_dirichlet(DeviceState *d, const double *rv, double *out, const double *dotv, double *part) {
  cudaStream_t st = d->stream;
  int pcnd = d->opt.precond;
  if (pcnd == IETI_PRECOND_NONE) {
    cudaMemcpyAsync(out, rv, d->M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    k_dot_partial<<<RED_BLOCKS, 256, 0, st>>>(d->M, out, dotv, part);
    d->nlaunch++;
    return;
  }
  bool scaled = pcnd != IETI_PRECOND_DIRICHLET;
  k_Bt<<<grid_for(d->NBt, 256), 256, 0, st>>>(d->NBt, d->bt_ptr, d->bt_lam, scaled ? d->bt_wd : d->bt_sgn, rv,
                                               nullptr, 1.0, d->ub);
  d->nlaunch++;
  gemv<T>(d, d->dP, d->P, d->ub, d->bp, nullptr, 1.0, 0.0, IETI_K_GEMV_P);
  k_jump<<<RED_BLOCKS, 256, 0, st>>>(d->M, d->lam_qp, d->lam_qm, scaled ? d->lam_wp : nullptr,
                                     scaled ? d->lam_wm : nullptr, d->bp, out, dotv, part);
  d->nlaunch++;
}

static int read_scalar(DeviceState *d, int idx, double *out, std::string &err) {
  CK(cudaMemcpyAsync(d->h_sc, d->sc + idx, sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  *out = *d->h_sc;
  return IETI_OK;
}

// PCG on F lambda = d (Sec. 4: Dirichlet-preconditioned CG, lambda_0 = 0)
template <class T>
static int pcg(DeviceState *d, int *its, double *rel, std::string &err) {
  cudaStream_t st = d->stream;
  int64_t m = d->M;
  *its = 0;
  *rel = 0.0;
  if (m == 0) return IETI_OK;
  CK(cudaMemsetAsync(d->lam, 0, m * sizeof(double), st));
  CK(cudaMemcpyAsync(d->r, d->dvec, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  k_dot_partial<<<RED_BLOCKS, 256, 0, st>>>(m, d->r, d->r, d->part);
  d->nlaunch++;
  k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_DD, 0);
  d->nlaunch++;
  double dd;
  int rc = read_scalar(d, SC_DD, &dd, err);
  if (rc) return rc;
  if (!(dd > 0.0)) return IETI_OK;
  double tol2 = d->opt.cg_tol * d->opt.cg_tol * dd;
  apply_precond<T>(d, d->r, d->z, d->r, d->part);
  k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_RZ, 0);
  d->nlaunch++;
  CK(cudaMemcpyAsync(d->p, d->z, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double rr = dd;
  for (int it = 1; it <= d->opt.cg_max_it; ++it) {
    apply_F<T>(d, d->p, d->Fp, d->p, d->part);
    k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_PQ, 1);
    d->nlaunch++;
    k_cg_update<<<RED_BLOCKS, 256, 0, st>>>(m, d->sc, d->p, d->Fp, d->lam, d->r, d->part);
    d->nlaunch++;
    k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_RR, 0);
    d->nlaunch++;
    rc = read_scalar(d, SC_RR, &rr, err);
    if (rc) return rc;
    *its = it;
    if (!std::isfinite(rr)) {
      err = "PCG breakdown (non-finite residual)";
      return IETI_ERR_CG_NOT_CONVERGED;
    }
    if (rr <= tol2) break;
    apply_precond<T>(d, d->r, d->z, d->r, d->part);
    k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_RZNEW, 2);
    d->nlaunch++;
    k_p_update<<<RED_BLOCKS, 256, 0, st>>>(m, d->sc, d->z, d->p);
    d->nlaunch++;
  }
  *rel = std::sqrt(rr / dd);
  CK(cudaGetLastError());
  if (rr > tol2) {
    err = "PCG did not reach cg_tol within cg_max_it";
    return IETI_ERR_CG_NOT_CONVERGED;
  }
  return IETI_OK;
}

// the whole dual-primal solve of a sweep as one persistent cooperative launch
// (pcg_kernel.cuh): condensation, d, PCG, recovery
// launch only (stream-ordered, no host synchronisation; usable under stream capture):
// barrier reset, trace reset, the cooperative launch on stream st
template <class T>
static int pcg_launch(DeviceState *d, const double *rhs, cudaStream_t st, std::string &err) {
  CK(cudaMemsetAsync(d->bar, 0, 3 * sizeof(unsigned), st));
  PcgArgs<T> a;
  a.m = d->M;
  a.nc = (int)d->NC;
  a.ldc = d->ldc;
  a.precond_none = d->opt.precond == IETI_PRECOND_NONE;
  a.scaled = d->opt.precond == IETI_PRECOND_DIRICHLET_MULT || d->opt.precond == IETI_PRECOND_DIRICHLET_STIFF;
  a.max_it = d->opt.cg_max_it;
  a.tol2 = d->opt.cg_tol * d->opt.cg_tol;
  a.bt_lam = d->ell_lam; a.bt_sgn = d->ell_sgn; a.bt_wd = d->ell_wd;
  a.nb_idx = d->nb_idx; a.nb_ca = d->nb_ca; a.nb_cb = d->nb_cb; a.yv0 = d->yv0; a.yv1 = d->yv1;
  a.lam_qp = d->lam_qp; a.lam_qm = d->lam_qm;
  a.lam_wp = a.scaled ? d->lam_wp : nullptr;
  a.lam_wm = a.scaled ? d->lam_wm : nullptr;
  a.kofs = d->kofs; a.bofs = d->bofs_d; a.pofs = d->pofs_d; a.hoff = d->hoff; a.qoff = d->qoff; a.poff = d->poff;
  a.igoff = d->igoff; a.gtoff = d->gtoff;
  a.ni = d->ni; a.nb = d->nb; a.np = d->npp; a.ldb = d->ldb; a.ldp = d->ldp; a.ldi = d->ldi; a.ldg = d->ldg;
  a.pc = d->pc; a.cp_pos = d->cp_pos; a.p_kept = d->p_kept; a.b_kept = d->b_kept;
  a.IG = (const T *)d->IG; a.GT = (const T *)d->GT;
  a.H = (const T *)d->H; a.Q = (const T *)d->Q; a.P = (const T *)d->P; a.Sinv = d->Sinv;
  a.hseg_ptr = d->hseg_ptr; a.hseg_s = d->hseg_s; a.hseg_r0 = d->hseg_r0; a.hseg_r1 = d->hseg_r1;
  a.bseg_ptr = d->bseg_ptr; a.bseg_s = d->bseg_s; a.bseg_r0 = d->bseg_r0; a.bseg_r1 = d->bseg_r1;
  if (d->psi_overhead > 0) {
    a.qseg_ptr = d->qseg_ptr; a.qseg_s = d->qseg_s; a.qseg_r0 = d->qseg_r0; a.qseg_r1 = d->qseg_r1;
  } else {
    a.qseg_ptr = d->bseg_ptr; a.qseg_s = d->bseg_s; a.qseg_r0 = d->bseg_r0; a.qseg_r1 = d->bseg_r1;
  }
  a.iseg_ptr = d->iseg_ptr; a.iseg_s = d->iseg_s; a.iseg_r0 = d->iseg_r0; a.iseg_r1 = d->iseg_r1;
  a.tseg_ptr = d->tseg_ptr; a.tseg_s = d->tseg_s; a.tseg_r0 = d->tseg_r0; a.tseg_r1 = d->tseg_r1;
  a.rhs = rhs; a.kg = d->kg; a.kx = d->kx; a.ub1 = d->ub1; a.uz = d->uz; a.nbt = d->NBt;
  a.Sinv = d->Scoarse_slot;
  a.lam = d->lam; a.p0 = d->p; a.p1 = d->p1; a.r0 = d->r; a.r1 = d->r1; a.z = d->z;
  a.ub = d->ubp; a.zb = d->zb; a.zf = d->zf; a.tpi = d->tpi; a.cc = d->ccg; a.q = d->q; a.zp = d->zp;
  a.part = d->ppart;
  a.bar = d->bar; a.out_its = d->pcg_its; a.out_rr = d->pcg_rr; a.out_dd = d->pcg_dd;
  a.trace = d->opt.profile ? d->trace : nullptr;
  a.stage_bytes = d->stage_bytes;
  a.xs_bytes = d->xs_bytes;
  a.n_stages = d->n_stages;
  a.l2_keep_frac = d->l2_keep_frac;
  a.spin_max = d->opt.wait_limit > 0 ? (long long)d->opt.wait_limit : (1ll << 25);
  a.coarse_nd = d->coarse_nd;
  a.nd_cw = d->nd_cw; a.nd_H = d->nd_H; a.nd_D = d->nd_D;
  a.nd_k0 = d->nd_k0; a.nd_nk = d->nd_nk; a.nd_ns = d->nd_ns; a.nd_zld = d->nd_zld; a.nd_ltld = d->nd_ltld;
  a.nd_sidx = d->nd_sidx; a.nd_dst = d->nd_dst; a.nd_nch = d->nd_nch;
  a.nd_zoff = d->nd_zoff; a.nd_ltoff = d->nd_ltoff; a.nd_soff = d->nd_soff; a.nd_uoff = d->nd_uoff;
  a.nd_srcoff = d->nd_srcoff;
  a.nd_Z = d->nd_Z; a.nd_Lt = d->nd_Lt; a.nd_slot = d->nd_slot;
  a.ndf_ptr = d->ndf_ptr; a.ndf_s = d->ndf_s; a.ndf_r0 = d->ndf_r0; a.ndf_r1 = d->ndf_r1;
  a.ndb_ptr = d->ndb_ptr; a.ndb_s = d->ndb_s; a.ndb_r0 = d->ndb_r0; a.ndb_r1 = d->ndb_r1;
  a.nd_nodes = d->nd_nodes; a.nd_flow = d->nd_flow;
  a.nd_cptr = d->nd_cptr; a.nd_cidx = d->nd_cidx; a.nd_parent = d->nd_parent;
  a.nd_nsegf = d->nd_nsegf; a.nd_nsegb = d->nd_nsegb; a.nd_done = d->nd_done;
  if (d->nd_flow) CK(cudaMemsetAsync(d->nd_done, 0, 2 * (size_t)d->nd_nodes * sizeof(unsigned), st));
  if (a.trace) CK(cudaMemsetAsync(d->trace, 0, TRACE_IT * TRACE_SLOTS * sizeof(unsigned long long), st));
  void *args[] = {&a};
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(d->G);
    cfg.blockDim = dim3(PCG_THREADS);
    cfg.dynamicSmemBytes = d->pcg_smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    int nattr = 1;
    if (d->l2_window > 0) {
      attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
      attr[1].val.accessPolicyWindow.base_ptr = d->iter_arena;
      attr[1].val.accessPolicyWindow.num_bytes = d->l2_window;
      attr[1].val.accessPolicyWindow.hitRatio = d->l2_hit_ratio;
      attr[1].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
      attr[1].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
      nattr = 2;
    }
    cfg.attrs = attr;
    cfg.numAttrs = nattr;
    const void *fn = d->coarse_nd ? (const void *)k_ddsolve<T, true> : (const void *)k_ddsolve<T, false>;
    CK(cudaLaunchKernelExC(&cfg, fn, args));
  }
  return IETI_OK;
}

template <class T>
static int pcg_persistent(DeviceState *d, const double *rhs, int *its, double *rel, std::string &err) {
  cudaStream_t st = d->stream;
  *its = 0;
  *rel = 0.0;
  prof_begin(d, IETI_K_PCG, 0.0);
  int lrc = pcg_launch<T>(d, rhs, st, err);
  if (lrc) return lrc;
  d->nlaunch++;
  prof_end(d);
  const double tol2 = d->opt.cg_tol * d->opt.cg_tol;
  const bool traced = d->opt.profile != 0;
  struct {
    int its;
    unsigned bar[3];
    double rr, dd;
  } h;
  CK(cudaMemcpyAsync(&h.its, d->pcg_its, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h.bar, d->bar, 3 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h.rr, d->pcg_rr, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h.dd, d->pcg_dd, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h.bar[1]) {
    err = "persistent PCG: a grid barrier timed out";
    return IETI_ERR_TIMEOUT;
  }
  *its = h.its;
  prof_set_bytes(d, d->bytes_iter_alg * (h.its + 2) + d->bytes_sweep_alg);
  if (traced) {
    unsigned long long tr[TRACE_IT * TRACE_SLOTS];
    CK(cudaMemcpy(tr, d->trace, sizeof(tr), cudaMemcpyDeviceToHost));
    for (int i = 0; i < std::min(h.its - 1, TRACE_IT); ++i) {
      unsigned long long *t = tr + i * TRACE_SLOTS;
      if (!t[14] || !t[11]) continue;
      unsigned long long prev = t[14];
      // phase starts: P1 at the iteration start, P3 after the P2 wait, P4, P5 after theirs
      const unsigned long long start_of[4] = {t[14], t[3], t[5], t[7]};
      for (int ph = 0; ph < 6; ++ph) {
        d->trace_acc[ph] += (t[2 * ph] - prev) * 1e-3;
        d->trace_wait[ph] += (t[2 * ph + 1] - t[2 * ph]) * 1e-3;
        prev = t[2 * ph + 1];
      }
      if (d->coarse_nd && t[35]) {
        unsigned long long prev_nd = t[3];  // the coarse phase starts after the P2 barrier
        const int nl = std::min(TRACE_ND, d->nd_H + std::max(d->nd_D - 1, 0));
        for (int lv = 0; lv < nl && t[32 + 4 * lv + 3]; ++lv) {
          const unsigned long long *u = t + 32 + 4 * lv;
          if (u[0] && u[1] && u[2]) {  // a CTA without rows in a level leaves the first three empty
            d->trace_nd[lv][0] += (u[0] - prev_nd) * 1e-3;
            d->trace_nd[lv][1] += (u[1] - u[0]) * 1e-3;
            d->trace_nd[lv][2] += (u[2] - u[1]) * 1e-3;
            d->trace_nd[lv][3] += (u[3] - u[2]) * 1e-3;
          } else {
            d->trace_nd[lv][3] += (u[3] - prev_nd) * 1e-3;
          }
          prev_nd = u[3];
        }
        d->trace_nd_n++;
      }
      for (int k = 0; k < 4; ++k) {
        const unsigned long long *u = t + 16 + 3 * k;
        if (!u[0] || !u[1] || !u[2]) continue;
        d->trace_sub[k][0] += (u[0] - start_of[k]) * 1e-3;
        d->trace_sub[k][1] += (u[1] - u[0]) * 1e-3;
        d->trace_sub[k][2] += (u[2] - u[1]) * 1e-3;
        d->trace_sub_n[k]++;
      }
      d->trace_n++;
    }
  }
  if (!(h.dd > 0.0)) return IETI_OK;
  *rel = std::sqrt(h.rr / h.dd);
  if (!std::isfinite(h.rr)) {
    err = "PCG breakdown (non-finite residual)";
    return IETI_ERR_CG_NOT_CONVERGED;
  }
  if (h.rr > tol2 * h.dd) {
    err = "PCG did not reach cg_tol within cg_max_it";
    return IETI_ERR_CG_NOT_CONVERGED;
  }
  return IETI_OK;
}

// contiguous byte-balanced row ranges per CTA, split into per-patch segments
// (a row weighs its leading dimension plus `overhead` elements: the per-row epilogue;
// every segment a CTA starts weighs `seg` elements more: its vector staging)
static void partition_rows(const std::vector<int32_t> &rows_per_patch, const std::vector<int32_t> &ld, int G,
                           std::vector<int32_t> &sptr, std::vector<int32_t> &ss, std::vector<int32_t> &r0,
                           std::vector<int32_t> &r1, int overhead = 16, int seg = 0) {
  int np_ = (int)rows_per_patch.size();
  double W = 0;
  int nonempty = 0;
  for (int s = 0; s < np_; ++s) {
    W += (double)rows_per_patch[s] * (ld[s] + overhead);
    nonempty += rows_per_patch[s] > 0;
  }
  W += (double)seg * (nonempty + G);  // about one segment per patch plus one split per CTA
  sptr.assign(1, 0);
  ss.clear(); r0.clear(); r1.clear();
  int s = 0, r = 0;
  double acc = 0;
  for (int c = 0; c < G; ++c) {
    double target = W * (c + 1) / G;
    while (s < np_ && (acc < target || c == G - 1)) {
      if (r >= rows_per_patch[s]) { ++s; r = 0; continue; }
      // take rows of patch s until the target is reached
      int take = rows_per_patch[s] - r;
      double per = ld[s] + overhead;
      acc += seg;
      if (c < G - 1) {
        int need = (int)std::ceil((target - acc) / per);
        take = std::max(1, std::min(take, need));
      }
      ss.push_back(s); r0.push_back(r); r1.push_back(r + take);
      acc += take * per;
      r += take;
      if (r >= rows_per_patch[s]) { ++s; r = 0; }
    }
    sptr.push_back((int32_t)ss.size());
  }
}

// dual-primal solve of the gauged step system for kept-space right-hand sides
// rhs (per patch, Sec. 3), solution into d->kx (kept space)
template <class T>
static int pcg_persistent(DeviceState *d, const double *rhs, int *its, double *rel, std::string &err);

// dual-primal solve of the gauged step system for kept-space right-hand sides rhs
// (per patch, Sec. 3), solution into d->kx (kept space)
template <class T>
static int dd_solve(DeviceState *d, const double *rhs, int *its, double *rel, std::string &err) {
  if (d->opt.pcg_mode == 0) return pcg_persistent<T>(d, rhs, its, rel, err);
  cudaStream_t st = d->stream;
  // interior condensation: z_i = W_ii^{-1} f_i, g_[bp] = f_[bp] - G f_i  (kg)
  gemv<T>(d, d->dIGi, d->IG, rhs, d->kg, nullptr, 1.0, 0.0, IETI_K_TRI);
  gemv<T>(d, d->dIGg, d->IG, rhs, d->kg, rhs, -1.0, 1.0, IETI_K_GEMV_Y);
  k_kept_to_bp<<<grid_for(d->NBt + d->NPt, 256), 256, 0, st>>>(d->NBt, d->NPt, d->b_kept, d->p_kept, d->kg, d->gb,
                                                                 d->gp);
  d->nlaunch++;
  // d = B (F g_b - Psi S_c^{-1} sum A^T (g_p - Psi^T g_b))
  condensed<T>(d, d->gb, d->gp);
  k_jump<<<RED_BLOCKS, 256, 0, st>>>(d->M, d->lam_qp, d->lam_qm, nullptr, nullptr, d->bp, d->dvec, nullptr, nullptr);
  d->nlaunch++;
  int rc = pcg<T>(d, its, rel, err);
  if (rc && rc != IETI_ERR_CG_NOT_CONVERGED) return rc;
  int cg_rc = rc;
  // recovery: v_b = g_b - B^T lambda; a_b = F v_b - Psi q, a_p = q
  k_Bt<<<grid_for(d->NBt, 256), 256, 0, st>>>(d->NBt, d->bt_ptr, d->bt_lam, d->bt_sgn, d->lam, d->gb, -1.0, d->ub);
  d->nlaunch++;
  condensed<T>(d, d->ub, d->gp);
  k_bp_to_kept<<<grid_for(d->NBt + d->NPt, 256), 256, 0, st>>>(d->NBt, d->NPt, d->b_kept, d->p_kept, d->pc, d->bp,
                                                                 d->q, d->kx);
  d->nlaunch++;
  // interior: a_i = z_i - G^T a_[bp]
  gemv<T>(d, d->dGT, d->GT, d->kx, d->kx, d->kg, -1.0, 1.0, IETI_K_GEMV_Y);
  CK(cudaGetLastError());
  return cg_rc;
}

// assemble a kept-space vector over the free global DOFs (rglob), return its norm
static int assemble_norm(DeviceState *d, const double *v, double *out, std::string &err) {
  k_assemble_free<<<RED_BLOCKS, 256, 0, d->stream>>>(d->NF, d->fptr, d->fpos, d->fglob, v, d->rglob, d->part);
  d->nlaunch++;
  k_dot_final<<<1, 256, 0, d->stream>>>(RED_BLOCKS, d->part, d->sc, SC_TMP, 0);
  d->nlaunch++;
  int rc = read_scalar(d, SC_TMP, out, err);
  *out = std::sqrt(*out);
  return rc;
}

// residual of the assembled system at the current iterate and its squared norm
// (kernels only, no host read): kr, rglob, sc[SC_TMP]
static void resid_norm_launch(DeviceState *d, cudaStream_t st) {
  k_resid<<<grid_for(d->NK * 32, 256), 256, 0, st>>>(d->NK, d->wptr, d->wcol, d->wval, d->ka, d->kf, d->kr);
  k_assemble_free<<<RED_BLOCKS, 256, 0, st>>>(d->NF, d->fptr, d->fpos, d->fglob, d->kr, d->rglob, d->part);
  k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_TMP, 0);
}

static void graph_release(DeviceState *d) {
  if (d->gexec) cudaGraphExecDestroy(d->gexec);
  if (d->graph) cudaGraphDestroy(d->graph);
  d->gexec = nullptr;
  d->graph = nullptr;
}

// Build the sweep loop of a linear step as one CUDA graph:
//   residual + norm, decide  ->  while (condition) { distribute, dual-primal solve,
//   solve status, owner update, gather, residual + norm, decide }
// captured on a private stream (the legacy default stream cannot be captured).
// Returns non-zero (graph mode off, state unchanged) when any graph call fails.
template <class T>
static int graph_build(DeviceState *d, std::string &err) {
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  auto bad = [&](const char *what, cudaError_t e) {
    if (cs) {
      cudaStreamCaptureStatus stt;
      if (cudaStreamIsCapturing(cs, &stt) == cudaSuccess && stt != cudaStreamCaptureStatusNone) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(cs, &junk);
        if (junk) cudaGraphDestroy(junk);
      }
      cudaStreamDestroy(cs);
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    err = std::string("graph mode unavailable: ") + what + ": " + cudaGetErrorString(e);
    return IETI_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return bad("stream", e);
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return bad("graph", e);
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, 0)) != cudaSuccess) return bad("conditional handle", e);
  const double outer_tol = d->opt.outer_tol, tol2 = d->opt.cg_tol * d->opt.cg_tol;
  const int max_sweeps = std::max(1, d->opt.max_sweeps);
  // the part before the loop
  if ((e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return bad("capture", e);
  resid_norm_launch(d, cs);
  k_ctl_decide<<<1, 32, 0, cs>>>(d->ctl, d->sc, h, outer_tol, max_sweeps, 1);
  if ((e = cudaStreamEndCapture(cs, &g)) != cudaSuccess) return bad("end capture", e);
  // its last node (the part is a chain: the node without dependents)
  size_t nn = 0;
  if ((e = cudaGraphGetNodes(g, nullptr, &nn)) != cudaSuccess || nn == 0) return bad("nodes", e);
  std::vector<cudaGraphNode_t> nodes(nn);
  if ((e = cudaGraphGetNodes(g, nodes.data(), &nn)) != cudaSuccess) return bad("nodes", e);
  cudaGraphNode_t leaf = nullptr;
  for (cudaGraphNode_t x : nodes) {
    size_t nd = 0;
    if ((e = cudaGraphNodeGetDependentNodes(x, nullptr, nullptr, &nd)) != cudaSuccess) return bad("dependents", e);
    if (nd == 0) leaf = x;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  if ((e = cudaGraphAddNode(&cnode, g, &leaf, nullptr, 1, &cp)) != cudaSuccess) return bad("while node", e);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return bad("body capture", e);
  k_distribute<<<grid_for(d->NK, 256), 256, 0, cs>>>(d->NK, d->kglob, d->kw, d->rglob, d->kr);
  std::string e2;
  if (pcg_launch<T>(d, d->kr, cs, e2) != IETI_OK) return bad("dual-primal launch", cudaGetLastError());
  k_ctl_solved<<<1, 32, 0, cs>>>(d->ctl, d->pcg_its, d->bar, d->pcg_rr, d->pcg_dd, tol2);
  k_owner_add<<<grid_for(d->NK, 256), 256, 0, cs>>>(d->NK, d->kglob, d->kown, d->kx, d->a);
  k_gather_kept<<<grid_for(d->NK, 256), 256, 0, cs>>>(d->NK, d->kglob, d->a, d->ka);
  resid_norm_launch(d, cs);
  k_ctl_decide<<<1, 32, 0, cs>>>(d->ctl, d->sc, h, outer_tol, max_sweeps, 0);
  if ((e = cudaStreamEndCapture(cs, &body)) != cudaSuccess) return bad("end body capture", e);
  if ((e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess) return bad("instantiate", e);
  cudaStreamDestroy(cs);
  d->graph = g;
  d->gexec = ge;
  return IETI_OK;
}

// the sweep loop of a linear step through the graph: one launch, one read of the
// control block afterwards
static int graph_sweeps(DeviceState *d, int *its_total, int *sweeps, double *rel, double *ores, std::string &err) {
  CK(cudaGraphLaunch(d->gexec, d->stream));
  CK(cudaMemcpyAsync(d->h_ctl, d->ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  const StepCtl c = *d->h_ctl;
  *its_total = c.its;
  *sweeps = c.sweeps;
  *rel = c.rel;
  *ores = c.ores;
  d->nlaunch += 4 + 9 * (int64_t)c.sweeps;
  if (c.bar_err) {
    err = "persistent PCG: a grid barrier timed out";
    return IETI_ERR_TIMEOUT;
  }
  if (c.status == 2 && d->opt.max_sweeps > 1 && !c.cg_fail) {
    err = "refinement did not reach outer_tol within max_sweeps";
    return IETI_ERR_CG_NOT_CONVERGED;
  }
  if (c.status == 3) {
    err = c.cg_fail ? "PCG did not reach cg_tol within cg_max_it" : "refinement stagnated above outer_tol";
    return IETI_ERR_CG_NOT_CONVERGED;
  }
  if (c.cg_fail) {
    err = "PCG did not reach cg_tol within cg_max_it";
    return IETI_ERR_CG_NOT_CONVERGED;
  }
  return IETI_OK;
}

template <class T>
static int step_impl(DeviceState *d, ieti_stats *stats, std::string &err) {
  cudaStream_t st = d->stream;
  int64_t NK = d->NK;
  // f = M a^l + dt j^{l+1}  (kept space, load split 1/k over the k patches holding a DOF)
  k_gather_kept<<<grid_for(NK, 256), 256, 0, st>>>(NK, d->kglob, d->a, d->ka);
  d->nlaunch++;
  k_rhs<<<grid_for(NK * 32, 256), 256, 0, st>>>(NK, d->mptr, d->mcol, d->mval, d->ka, d->kglob, d->kw, d->j, d->dt,
                                                 d->kf);
  d->nlaunch++;
  double fn = 0.0;
  int rc;
  if (d->gexec) {
    // ||f||^2 stays on the device (sc[SC_FN]) for the graph's decisions
    k_assemble_free<<<RED_BLOCKS, 256, 0, st>>>(d->NF, d->fptr, d->fpos, d->fglob, d->kf, d->rglob, d->part);
    k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_FN, 0);
    d->nlaunch += 2;
  } else if ((rc = assemble_norm(d, d->kf, &fn, err))) {
    return rc;
  }
  if (d->opt.predictor) {
    // keep a^l; with a^{l-1} known, start the sweeps from the extrapolated iterate
    CK(cudaMemcpyAsync(d->a_old, d->a, d->n_edges * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (d->n_hist > 0) {
      const double *a2 = (d->opt.predictor == 2 && d->n_hist > 1) ? d->a_prev2 : nullptr;
      k_extrapolate<<<grid_for(d->n_edges, 256), 256, 0, st>>>(d->n_edges, d->a_old, d->a_prev, a2, d->a);
      k_gather_kept<<<grid_for(NK, 256), 256, 0, st>>>(NK, d->kglob, d->a, d->ka);
      d->nlaunch += 2;
    }
  }
  int its_total = 0, sweeps = 0, cg_rc = IETI_OK;
  double rel = 0, ores = -1.0, prev = -1.0;
  int max_sweeps = std::max(1, d->opt.max_sweeps);
  const bool newton = d->nl_np > 0;
  bool update_small = false;
  d->step_refactors = 0;
  if (d->gexec) {
    cg_rc = graph_sweeps(d, &its_total, &sweeps, &rel, &ores, err);
    if (cg_rc != IETI_OK && cg_rc != IETI_ERR_CG_NOT_CONVERGED) return cg_rc;
  }
  for (int sweep = 0; !d->gexec; ++sweep) {
    // defect of the ASSEMBLED system at the current iterate, in FP64: r = f - W_g a,
    // redistributed over the patches with the 1/k weights (so that the local
    // right-hand sides of the correction are as small as the defect itself)
    prof_begin(d, IETI_K_SPMV, d->gemv_bytes[IETI_K_SPMV]);
    k_resid<<<grid_for(NK * 32, 256), 256, 0, st>>>(NK, d->wptr, d->wcol, d->wval, d->ka, d->kf, d->kr);
    d->nlaunch++;
    prof_end(d);
    if (newton) {
      // Newton residual of the nonlinear system: r -= dt N(a) over the nonlinear elements
      size_t sm = (size_t)(d->nl_max_nloc + 4 * d->nl_max_nq) * sizeof(double);
      k_nl_eval<<<(unsigned)d->nl_ne, 128, sm, st>>>(d->nl_G, d->nl_cq, d->nl_kept, d->nl_glob, d->nl_goff,
                                                     d->nl_qoff, d->nl_doff, d->nl_nloc, d->nl_nq, d->nl_bpos,
                                                     d->nlb_kofs, d->a, d->law, d->dt, d->kr, d->nl_tq, 1);
      d->nlaunch++;
    }
    double rn;
    if ((rc = assemble_norm(d, d->kr, &rn, err))) return rc;
    ores = fn > 0 ? rn / fn : 0.0;
    if (ores <= d->opt.outer_tol || fn == 0.0 || update_small) break;
    if (sweep >= max_sweeps) {
      if (max_sweeps > 1 && cg_rc == IETI_OK) {
        err = "refinement did not reach outer_tol within max_sweeps";
        cg_rc = IETI_ERR_CG_NOT_CONVERGED;
      }
      break;
    }
    // stagnation at the rounding floor of the FP64 defect (Newton with a frozen tangent
    // contracts linearly, possibly slowly: only a residual that stops falling ends it)
    if (sweep >= (newton ? 6 : 2) && rn > (newton ? 1.0 : 0.9) * prev) {
      if (cg_rc == IETI_OK) {
        err = "refinement stagnated above outer_tol";
        cg_rc = IETI_ERR_CG_NOT_CONVERGED;
      }
      break;
    }
    prev = rn;
    if (newton && (d->opt.refactor == IETI_REFACTOR_EVERY || (d->opt.refactor == IETI_REFACTOR_STEP && sweep == 0)))
      if ((rc = nl_refactor_any(d, err))) return rc;
    k_distribute<<<grid_for(NK, 256), 256, 0, st>>>(NK, d->kglob, d->kw, d->rglob, d->kr);
    d->nlaunch++;
    int its = 0;
    rc = dd_solve<T>(d, d->kr, &its, &rel, err);
    its_total += its;
    sweeps++;
    if (rc == IETI_ERR_CG_NOT_CONVERGED) cg_rc = rc;
    else if (rc) return rc;
    k_owner_add<<<grid_for(NK, 256), 256, 0, st>>>(NK, d->kglob, d->kown, d->kx, d->a);
    d->nlaunch++;
    k_gather_kept<<<grid_for(NK, 256), 256, 0, st>>>(NK, d->kglob, d->a, d->ka);
    d->nlaunch++;
    if (newton && d->opt.newton_tol > 0.0) {
      // relative update ||d|| / ||a|| of this Newton iteration
      k_owner_sq<<<RED_BLOCKS, 256, 0, st>>>(NK, d->kown, d->kx, d->part);
      k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_TMP, 0);
      double dn2, an2;
      if ((rc = read_scalar(d, SC_TMP, &dn2, err))) return rc;
      k_owner_sq<<<RED_BLOCKS, 256, 0, st>>>(NK, d->kown, d->ka, d->part);
      k_dot_final<<<1, 256, 0, st>>>(RED_BLOCKS, d->part, d->sc, SC_TMP, 0);
      if ((rc = read_scalar(d, SC_TMP, &an2, err))) return rc;
      d->nlaunch += 4;
      update_small = dn2 <= d->opt.newton_tol * d->opt.newton_tol * an2;
    }
  }
  CK(cudaGetLastError());
  if (d->opt.predictor) {
    // a^l becomes the previous state, a^{l-1} the one before (quadratic predictor)
    if (d->opt.predictor == 2) std::swap(d->a_prev2, d->a_prev);
    std::swap(d->a_prev, d->a_old);
    d->n_hist = std::min(d->n_hist + 1, d->opt.predictor);
  }
  if (stats) {
    stats->refactors = d->step_refactors;
    stats->cg_its = its_total;
    stats->sweeps = sweeps;
    stats->rel_res = rel;
    stats->outer_res = ores;
  }
  return cg_rc;
}

// =============================================================================
// Setup orchestration
// =============================================================================
// return the L2 lines of the per-iteration operator arena to normal eviction priority
// (they were loaded evict-last during the step), so that later traffic can evict them
__global__ void k_l2_demote(const unsigned char *base, int64_t lines) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < lines; i += (int64_t)gridDim.x * blockDim.x)
    asm volatile("applypriority.global.L2::evict_normal [%0], 128;" ::"l"(base + 128 * i) : "memory");
}

// ---------------------------------------------------------------------------
// Schedule of the persistent dual-primal kernel and its autotuner.
//
// A schedule fixes the CTAs per SM (grid = cps x SMs, every CTA resident: the launch
// is cooperative), the number of TMA ring stages and the bytes per stage.  The
// four row partitions of the kernel (H rows, interface rows, IG rows, GT rows) are
// cut into cps x SMs byte-balanced ranges for it.  Results depend on the schedule
// only through the rounding order of the cross-CTA reductions.
constexpr int PCG_MAX_CPS = 2;

struct PcgSched {
  int cps = 1, ns = 3;
  size_t stage = 0;
  int psi = 0;  // 0: the Psi rows share the S_bb partition; > 0: own partition, per-row overhead
  int seg = 0;  // per-segment weight of the row partitions (elements)
  int flow = 0;  // nested-dissection levels wait on per-node counters instead of grid barriers
};

// widest FP64 coarse row / staged coarse vector: the dense S_c^{-1} row, or the widest
// nested-dissection block
static size_t pcg_coarse_width(const DeviceState *d) {
  return (size_t)(d->coarse_nd ? d->nd_zmax : std::max(d->ldc, 4));
}
static size_t pcg_xs_bytes(const DeviceState *d) {
  const size_t esz = d->mixed ? 4 : 8;
  return (std::max((size_t)d->ldmax * esz, pcg_coarse_width(d) * sizeof(double)) + 127) / 128 * 128;
}
static size_t pcg_row_max(const DeviceState *d) {
  const size_t esz = d->mixed ? 4 : 8;
  return (std::max((size_t)d->ldmax * esz, pcg_coarse_width(d) * sizeof(double)) + 127) / 128 * 128;
}
// dynamic shared memory per CTA at cps CTAs per SM (227 KB per CTA at most, the
// kernel's static arrays and the per-CTA reservation taken off)
static size_t pcg_budget(int cps) { return cps == 1 ? 212 * 1024 : 100 * 1024; }

// the rule: one CTA per SM, three stages (two when three rows do not fit) of at most 64 KB
static int pcg_rule(const DeviceState *d, PcgSched *out, std::string &err) {
  const size_t xs = pcg_xs_bytes(d), row_max = pcg_row_max(d), budget = pcg_budget(1);
  if (xs + 2 * row_max > budget) {
    err = "a patch block is too wide for the shared-memory staging of the dual-primal kernel";
    return IETI_ERR_TOO_LARGE;
  }
  out->cps = 1;
  out->ns = (xs + 3 * row_max <= budget) ? 3 : 2;
  size_t stage = std::min<size_t>(64 * 1024, (budget - xs) / out->ns) / 128 * 128;
  out->stage = std::max(stage, row_max);
  return IETI_OK;
}

template <class T>
static int upload_cap(DeviceState *d, T **ptr, size_t cap, const std::vector<T> &h, std::string &err) {
  if (!*ptr) {
    int rc = dalloc(d, ptr, cap, err);
    if (rc) return rc;
  }
  if (h.size() > cap) {
    err = "persistent PCG plan exceeds its preallocated size";
    return IETI_ERR_INVALID_ARG;
  }
  if (!h.empty()) CK(cudaMemcpyAsync(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return IETI_OK;
}

// apply a schedule: shared-memory layout, grid, row partitions.  IETI_ERR_TOO_LARGE
// (state unchanged) when it does not fit the shared memory or the occupancy.
static int pcg_plan(DeviceState *d, const PcgSched &sc, std::string &err) {
  const size_t xs = pcg_xs_bytes(d), row_max = pcg_row_max(d);
  if (sc.cps < 1 || sc.cps > PCG_MAX_CPS || sc.ns < 2 || sc.ns > NS_MAX || sc.stage % 128 || sc.stage < row_max ||
      xs + sc.ns * sc.stage > pcg_budget(sc.cps)) {
    err = "schedule does not fit the dual-primal kernel's shared memory";
    return IETI_ERR_TOO_LARGE;
  }
  const size_t smem = xs + sc.ns * sc.stage;
  const void *fn = d->mixed ? (d->coarse_nd ? (const void *)k_ddsolve<float, true> : (const void *)k_ddsolve<float, false>)
                            : (d->coarse_nd ? (const void *)k_ddsolve<double, true> : (const void *)k_ddsolve<double, false>);
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PCG_THREADS, smem));
  if (per_sm < sc.cps) {
    err = "schedule exceeds the occupancy of the dual-primal kernel";
    return IETI_ERR_TOO_LARGE;
  }
  d->n_stages = sc.ns;
  d->xs_bytes = (unsigned)xs;
  d->stage_bytes = (unsigned)sc.stage;
  d->pcg_smem = smem;
  d->cps = sc.cps;
  d->G = sc.cps * d->n_sm;
  const size_t cap_ptr = (size_t)PCG_MAX_CPS * d->n_sm + 1, cap_seg = (size_t)PCG_MAX_CPS * d->n_sm + d->np_ + 1;
  int32_t **ptrs[4][4] = {{&d->hseg_ptr, &d->hseg_s, &d->hseg_r0, &d->hseg_r1},
                          {&d->bseg_ptr, &d->bseg_s, &d->bseg_r0, &d->bseg_r1},
                          {&d->iseg_ptr, &d->iseg_s, &d->iseg_r0, &d->iseg_r1},
                          {&d->tseg_ptr, &d->tseg_s, &d->tseg_r0, &d->tseg_r1}};
  std::vector<int32_t> sp, ss, r0v, r1v;
  for (int k = 0; k < 4; ++k) {
    partition_rows(d->plan_rows[k], d->plan_ld[k], d->G, sp, ss, r0v, r1v, 16, sc.seg);
    int rc;
    if ((rc = upload_cap(d, ptrs[k][0], cap_ptr, sp, err)) || (rc = upload_cap(d, ptrs[k][1], cap_seg, ss, err)) ||
        (rc = upload_cap(d, ptrs[k][2], cap_seg, r0v, err)) || (rc = upload_cap(d, ptrs[k][3], cap_seg, r1v, err)))
      return rc;
  }
  if (d->coarse_nd) {
    // rows of every nested-dissection level, partitioned like the patch operators
    // (segment s = node id); pointer rows of all levels concatenated
    for (int dir = 0; dir < 2; ++dir) {
      const auto &levels = dir == 0 ? d->ndh_fwd : d->ndh_bwd;
      std::vector<int32_t> P, S, R0, R1;
      for (const auto &L : levels) {
        std::vector<int32_t> rows, ld;
        for (int nd : L) {
          rows.push_back(dir == 0 ? d->ndh_nk[nd] + d->ndh_ns[nd] : d->ndh_nk[nd]);
          ld.push_back(dir == 0 ? d->ndh_zld[nd] : d->ndh_ltld[nd]);
        }
        partition_rows(rows, ld, d->G, sp, ss, r0v, r1v, 16, sc.seg);
        const int32_t base = (int32_t)S.size();
        for (int32_t v : sp) P.push_back(base + v);
        for (int32_t v : ss) S.push_back(L[v]);
        R0.insert(R0.end(), r0v.begin(), r0v.end());
        R1.insert(R1.end(), r1v.begin(), r1v.end());
      }
      const size_t nl = std::max<size_t>(levels.size(), 1);
      const size_t cp = nl * ((size_t)PCG_MAX_CPS * d->n_sm + 1), cs = nl * (size_t)PCG_MAX_CPS * d->n_sm + d->nd_nodes + 1;
      std::vector<int32_t> nseg(d->nd_nodes, 0);  // segments of every node over all CTAs
      for (int32_t v : S) nseg[v]++;
      CK(cudaMemcpyAsync(dir == 0 ? d->nd_nsegf : d->nd_nsegb, nseg.data(), nseg.size() * 4, cudaMemcpyHostToDevice,
                         d->stream));
      if (P.empty()) P.push_back(0);
      int rc;
      if (dir == 0 ? ((rc = upload_cap(d, &d->ndf_ptr, cp, P, err)) || (rc = upload_cap(d, &d->ndf_s, cs, S, err)) ||
                      (rc = upload_cap(d, &d->ndf_r0, cs, R0, err)) || (rc = upload_cap(d, &d->ndf_r1, cs, R1, err)))
                   : ((rc = upload_cap(d, &d->ndb_ptr, cp, P, err)) || (rc = upload_cap(d, &d->ndb_s, cs, S, err)) ||
                      (rc = upload_cap(d, &d->ndb_r0, cs, R0, err)) || (rc = upload_cap(d, &d->ndb_r1, cs, R1, err))))
        return rc;
    }
  }
  d->psi_overhead = sc.psi;
  d->seg_overhead = sc.seg;
  d->nd_flow = d->coarse_nd ? sc.flow : 0;
  if (sc.psi > 0) {
    partition_rows(d->plan_rows[4], d->plan_ld[4], d->G, sp, ss, r0v, r1v, sc.psi, sc.seg);
    int rc;
    if ((rc = upload_cap(d, &d->qseg_ptr, cap_ptr, sp, err)) || (rc = upload_cap(d, &d->qseg_s, cap_seg, ss, err)) ||
        (rc = upload_cap(d, &d->qseg_r0, cap_seg, r0v, err)) || (rc = upload_cap(d, &d->qseg_r1, cap_seg, r1v, err)))
      return rc;
  }
  return IETI_OK;
}

// synthetic kept-space right-hand side of the tuning solves (a fixed bounded pattern)
__global__ void k_tune_rhs(double *x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t h = (uint32_t)i * 2654435761u;
    x[i] = (double)(h >> 8) * (1.0 / 16777216.0) - 0.5;
  }
}

// time per PCG iteration (us) of the current schedule: `iters` iterations (no
// convergence stop), the best of two runs after one untimed run
template <class T>
static int pcg_time(DeviceState *d, const double *rhs, int iters, double *us, std::string &err) {
  const ieti_options keep = d->opt;
  d->opt.profile = 0;
  d->opt.cg_tol = 0.0;
  d->opt.cg_max_it = iters;
  double best = 1e300;
  int rc = IETI_OK;
  for (int rep = 0; rep < 3 && rc == IETI_OK; ++rep) {
    int its = 0;
    double rel = 0;
    std::string e2;
    cudaEventRecord(d->ev0, d->stream);
    rc = pcg_persistent<T>(d, rhs, &its, &rel, e2);
    cudaEventRecord(d->ev1, d->stream);
    if (rc == IETI_ERR_CG_NOT_CONVERGED) rc = IETI_OK;  // the iteration count is fixed on purpose
    if (rc != IETI_OK) {
      err = "autotuning solve failed: " + e2;
      break;
    }
    float ms = 0;
    if (cudaEventSynchronize(d->ev1) != cudaSuccess || cudaEventElapsedTime(&ms, d->ev0, d->ev1) != cudaSuccess) {
      err = "autotuning: event timing failed";
      rc = IETI_ERR_CUDA;
      break;
    }
    if (rep > 0) best = std::min(best, 1e3 * ms / std::max(its + 2, 1));
  }
  d->opt = keep;
  d->nlaunch = 0;
  *us = best;
  return rc;
}

static std::string tune_key(const DeviceState *d) {
  cudaDeviceProp prop{};
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, d->device) == cudaSuccess) name = prop.name;
  for (char &c : name)
    if (c == ' ' || c == '\t' || c == '\n') c = '_';
  std::ostringstream k;
  k << name << "|sm" << d->n_sm << "|" << (d->mixed ? "mixed" : "fp64") << "|np" << d->np_ << "|nk" << d->NK << "|nb"
    << d->NBt << "|npi" << d->NPt << "|m" << d->M << "|nc" << d->NC << "|ld" << d->ldmax;
  return k.str();
}

// cache lines: "ieti_tune2 <key> <cps> <stages> <stage bytes> <psi overhead>"
static bool tune_cache_lookup(const std::string &path, const std::string &key, PcgSched *out) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream ls(line);
    std::string tag, k;
    long cps = 0, ns = 0, stage = 0, psi = -1, seg = 0;
    // ieti_tune3 lines carry the segment weight; ieti_tune2 lines (without it) read as 0
    if (!(ls >> tag >> k >> cps >> ns >> stage >> psi) || (tag != "ieti_tune2" && tag != "ieti_tune3") || k != key)
      continue;
    long flow = 0;
    if (tag == "ieti_tune3" && !(ls >> seg >> flow)) continue;
    if (flow != 0 && flow != 1) continue;
    if (cps < 1 || cps > PCG_MAX_CPS || ns < 2 || ns > NS_MAX || stage < 128 || stage > 227 * 1024 || psi < 0 ||
        psi > 4096 || seg < 0 || seg > (1 << 20))
      continue;
    out->cps = (int)cps;
    out->ns = (int)ns;
    out->stage = (size_t)stage;
    out->psi = (int)psi;
    out->seg = (int)seg;
    out->flow = (int)flow;
    found = true;  // the last valid entry of the key wins
  }
  return found;
}

static bool tune_cache_store(const std::string &path, const std::string &key, const PcgSched &sc) {
  std::vector<std::string> keep;
  {
    std::ifstream f(path);
    std::string line;
    while (f && std::getline(f, line)) {
      std::istringstream ls(line);
      std::string tag, k;
      if ((ls >> tag >> k) && (tag == "ieti_tune2" || tag == "ieti_tune3") && k == key) continue;
      if (!line.empty()) keep.push_back(line);
    }
  }
  const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
  {
    std::ofstream f(tmp, std::ios::trunc);
    if (!f) return false;
    for (auto &l : keep) f << l << "\n";
    f << "ieti_tune3 " << key << " " << sc.cps << " " << sc.ns << " " << sc.stage << " " << sc.psi << " " << sc.seg
      << " " << sc.flow << "\n";
    if (!f.good()) return false;
  }
  return std::rename(tmp.c_str(), path.c_str()) == 0;
}

// pick the schedule: from the cache, else by timing every feasible candidate
template <class T>
static int pcg_autotune(DeviceState *d, std::string &err) {
  auto t0 = std::chrono::steady_clock::now();
  const std::string key = tune_key(d);
  const char *cache = d->opt.tune_cache;
  PcgSched rule, best;
  int rc = pcg_rule(d, &rule, err);
  if (rc) return rc;
  if (cache && *cache && tune_cache_lookup(cache, key, &best)) {
    std::string e2;
    if (pcg_plan(d, best, e2) == IETI_OK) {
      d->sched_source = 3;
      d->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      return IETI_OK;
    }
  }
  double *rhs = nullptr;
  if ((rc = dalloc(d, &rhs, (size_t)d->NK, err))) return rc;
  k_tune_rhs<<<grid_for(d->NK, 256), 256, 0, d->stream>>>(rhs, d->NK);
  CK(cudaGetLastError());
  const int iters = 16;
  std::vector<PcgSched> cand;
  for (int cps = 1; cps <= PCG_MAX_CPS; ++cps)
    for (int ns : {2, 3, 4, 6})
      for (size_t kb : {16, 24, 32, 48, 64, 96}) cand.push_back({cps, ns, kb * 1024});
  cand.push_back(rule);
  double best_us = 1e300, rule_us = 1e300;
  best = rule;
  PcgSched fastest = rule;
  for (size_t c = 0; c < cand.size(); ++c) {
    std::string e2;
    const int prc = pcg_plan(d, cand[c], e2);
    if (prc == IETI_ERR_TOO_LARGE) continue;  // does not fit: not a candidate
    if (prc) {
      err = e2;
      rc = prc;
      break;
    }
    double us = 0;
    if ((rc = pcg_time<T>(d, rhs, iters, &us, err))) break;
    d->tune_candidates++;
    if (c + 1 == cand.size()) rule_us = us;
    if (us < best_us) {
      best_us = us;
      fastest = cand[c];
    }
  }
  // the rule stays unless a candidate is faster by more than the timing noise (1%)
  if (best_us < 0.99 * rule_us) {
    best = fastest;
  } else {
    best_us = rule_us;
  }
  // then the Psi rows on their own partition, for a few per-row overheads
  for (int psi : {16, 64, 256}) {
    if (rc) break;
    PcgSched c = best;
    c.psi = psi;
    std::string e2;
    const int prc = pcg_plan(d, c, e2);
    if (prc) {
      err = e2;
      rc = prc;
      break;
    }
    double us = 0;
    if ((rc = pcg_time<T>(d, rhs, iters, &us, err))) break;
    d->tune_candidates++;
    if (us < 0.99 * best_us) {
      best_us = us;
      best = c;
    }
  }
  // then per-segment weights of the partitions (fewer, larger segments per CTA: each
  // segment stages its vector before its rows), and for the nested-dissection coarse
  // solve the per-node counters instead of grid barriers between its levels
  std::vector<std::pair<int, int>> extra;
  for (int seg : {2048, 8192, 32768}) extra.push_back({seg, -1});
  if (d->coarse_nd) extra.push_back({-1, 1});
  for (auto [seg, flow] : extra) {
    if (rc) break;
    PcgSched c = best;
    if (seg >= 0) c.seg = seg;
    if (flow >= 0) c.flow = flow;
    std::string e2;
    const int prc = pcg_plan(d, c, e2);
    if (prc) {
      err = e2;
      rc = prc;
      break;
    }
    double us = 0;
    if ((rc = pcg_time<T>(d, rhs, iters, &us, err))) break;
    d->tune_candidates++;
    if (us < 0.99 * best_us) {
      best_us = us;
      best = c;
    }
  }
  cudaStreamSynchronize(d->stream);
  cudaFree(rhs);
  d->allocs.erase(std::find(d->allocs.begin(), d->allocs.end(), (void *)rhs));
  d->bytes -= d->NK * 8;
  if (rc) return rc;
  if ((rc = pcg_plan(d, best, err))) return rc;
  // the tuning solves leave the iteration vectors non-zero: clear the ones a solve
  // reads before writing
  CK(cudaMemsetAsync(d->p, 0, d->M * sizeof(double), d->stream));
  CK(cudaMemsetAsync(d->p1, 0, d->M * sizeof(double), d->stream));
  CK(cudaStreamSynchronize(d->stream));
  d->tune_us[0] = rule_us;
  d->tune_us[1] = best_us;
  d->sched_source = 1;
  if (cache && *cache && tune_cache_store(cache, key, best)) d->sched_source = 2;
  d->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return IETI_OK;
}

// The balanced preconditioner's deflation space: one column per pair of patches
// (s < t) joined by multipliers, the indicator of that pair's multipliers.  F U by k
// applications of the dual operator (the setup's operators, the path's precision),
// E = U^T F U summed on the host in FP64, E^{-1} by a host Cholesky (k is the number of
// patch pairs: hundreds to a few thousand).
template <class T>
static int deflation_setup(DeviceState *d, const HostSetup &hs, std::string &err) {
  const int64_t m = d->M;
  if (m == 0) return IETI_OK;
  std::vector<std::pair<int32_t, int32_t>> pairs;
  pairs.reserve(hs.lam.size());
  for (const Multiplier &L : hs.lam) pairs.emplace_back(L.s, L.t);
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  const int k = (int)pairs.size();
  if ((double)k * (double)m * 8.0 > 8e9 || k > 4096) {  // F U on the device, E^{-1} by a host Cholesky
    err = "balanced preconditioner: the patch-pair space is too large (" + std::to_string(k) + " pairs x " +
          std::to_string(m) + " multipliers)";
    return IETI_ERR_TOO_LARGE;
  }
  std::vector<int32_t> pair_of(m), ptr(k + 1, 0), lam_of(m);
  for (int64_t l = 0; l < m; ++l) {
    const auto it = std::lower_bound(pairs.begin(), pairs.end(), std::make_pair(hs.lam[l].s, hs.lam[l].t));
    pair_of[l] = (int32_t)(it - pairs.begin());
    ptr[pair_of[l] + 1]++;
  }
  for (int j = 0; j < k; ++j) ptr[j + 1] += ptr[j];
  {
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t l = 0; l < m; ++l) lam_of[fill[pair_of[l]]++] = (int32_t)l;
  }
  int rc;
  if ((rc = upload(d, &d->defl_pair, pair_of, err)) || (rc = upload(d, &d->defl_ptr, ptr, err)) ||
      (rc = upload(d, &d->defl_lam, lam_of, err)) || (rc = dalloc(d, &d->defl_FUt, (size_t)k * m, err)) ||
      (rc = dalloc(d, &d->defl_Einv, (size_t)k * k, err)) || (rc = dalloc(d, &d->defl_ur, (size_t)k, err)) ||
      (rc = dalloc(d, &d->defl_c, (size_t)k, err)) || (rc = dalloc(d, &d->defl_fw, (size_t)k, err)) ||
      (rc = dalloc(d, &d->defl_rh, (size_t)m, err)) || (rc = dalloc(d, &d->defl_w, (size_t)m, err)))
    return rc;
  cudaStream_t st = d->stream;
  for (int j = 0; j < k; ++j) {
    k_pair_indicator<<<grid_for(m, 256), 256, 0, st>>>(m, d->defl_pair, j, d->defl_w);
    apply_F<T>(d, d->defl_w, d->defl_FUt + (int64_t)j * m, d->defl_w, d->part);
  }
  d->launches_setup += 3 * (int64_t)k;
  CK(cudaGetLastError());
  std::vector<double> FUt((size_t)k * m), E((size_t)k * k, 0.0);
  CK(cudaMemcpyAsync(FUt.data(), d->defl_FUt, FUt.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int j = 0; j < k; ++j)
    for (int64_t l = 0; l < m; ++l) E[(size_t)pair_of[l] * k + j] += FUt[(size_t)j * m + l];
  for (int i = 0; i < k; ++i)  // F is symmetric: average the two rounding orders
    for (int j = 0; j < i; ++j) {
      const double v = 0.5 * (E[(size_t)i * k + j] + E[(size_t)j * k + i]);
      E[(size_t)i * k + j] = E[(size_t)j * k + i] = v;
    }
  // Cholesky E = L L^T (lower, in place), then E^{-1} = L^{-T} L^{-1} column by column
  for (int j = 0; j < k; ++j) {
    double dj = E[(size_t)j * k + j];
    for (int q = 0; q < j; ++q) dj -= E[(size_t)j * k + q] * E[(size_t)j * k + q];
    if (!(dj > 0.0)) {
      err = "balanced preconditioner: U^T F U is not positive definite (pair " + std::to_string(j) + ")";
      return IETI_ERR_NOT_SPD;
    }
    const double ljj = std::sqrt(dj);
    E[(size_t)j * k + j] = ljj;
    for (int i = j + 1; i < k; ++i) {
      double v = E[(size_t)i * k + j];
      for (int q = 0; q < j; ++q) v -= E[(size_t)i * k + q] * E[(size_t)j * k + q];
      E[(size_t)i * k + j] = v / ljj;
    }
  }
  std::vector<double> Einv((size_t)k * k), col(k);
  for (int c = 0; c < k; ++c) {
    for (int i = 0; i < k; ++i) {   // L y = e_c
      double v = i == c ? 1.0 : 0.0;
      for (int q = 0; q < i; ++q) v -= E[(size_t)i * k + q] * col[q];
      col[i] = v / E[(size_t)i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {  // L^T x = y
      double v = col[i];
      for (int q = i + 1; q < k; ++q) v -= E[(size_t)q * k + i] * col[q];
      col[i] = v / E[(size_t)i * k + i];
    }
    for (int i = 0; i < k; ++i) Einv[(size_t)i * k + c] = col[i];
  }
  CK(cudaMemcpyAsync(d->defl_Einv, Einv.data(), Einv.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  d->defl_k = k;
  return IETI_OK;
}

int device_setup(const HostSetup &hs, const CoarseTree *tree, const ieti_options &opt_in, DeviceState **out,
                 std::string &err) {
  auto t0 = std::chrono::steady_clock::now();
  // the balanced preconditioner runs in the host-loop PCG (its projections are extra
  // passes between the library's kernels)
  ieti_options opt = opt_in;
  if (opt.deflation) opt.pcg_mode = 1;
  DeviceState *d = new DeviceState();
  *out = nullptr;
  d->opt = opt;
  d->device = opt.device;
  d->mixed = opt.precision == IETI_PREC_MIXED;
  d->factor = d->mixed ? opt.factor : IETI_FACTOR_FP64;
  d->nonlinear = hs.nonlinear;
  d->law = NlLaw{hs.law[0], hs.law[1], hs.law[2], hs.law[3]};
  d->dt = hs.dt;
  auto fail = [&](int rc) {
    device_destroy(d);
    return rc;
  };
  CK(cudaSetDevice(d->device));
  d->stream = (cudaStream_t)opt.cuda_stream;
  // coarse solve: dense S_c^{-1} rows, or the nested-dissection factor; auto takes the
  // factor once the dense inverse passes 64 MB (its bytes per iteration grow as nc^2)
  {
    const double nc0 = (double)hs.n_coarse;
    bool nd = opt.coarse == IETI_COARSE_ND;
    if (opt.coarse == IETI_COARSE_AUTO)
      nd = tree && tree->n_nodes > 0 && opt.pcg_mode == 0 && 8.0 * nc0 * nc0 > 64e6;
    if (nd && (opt.pcg_mode != 0 || !tree)) {
      err = opt.deflation ? "the nested-dissection coarse solve needs the persistent PCG (deflation runs the "
                            "host-loop PCG)"
                          : "the nested-dissection coarse solve needs pcg_mode 0";
      return fail(IETI_ERR_INVALID_ARG);
    }
    d->coarse_nd = nd && hs.n_coarse > 0 && tree->n_nodes > 0;
    d->nd_tree = d->coarse_nd ? tree : nullptr;
  }
  CK(cudaEventCreate(&d->ev0));
  CK(cudaEventCreate(&d->ev1));
  const int np_ = hs.n_patches();
  d->np_ = np_;
  d->n_edges = hs.n_edges;
  // ---------------- sizes and offsets
  std::vector<int32_t> hni(np_), hnb(np_), hnp(np_), hn(np_), hnn(np_), hrowpatch, hrowlocal, hldb(np_), hldp(np_);
  std::vector<int64_t> hkofs(np_ + 1, 0), hdoff(np_ + 1, 0), hig(np_ + 1, 0), hgt(np_ + 1, 0), hh(np_ + 1, 0),
      hq(np_ + 1, 0), hp(np_ + 1, 0), hbofs(np_ + 1, 0), hpofs(np_ + 1, 0);
  std::vector<int32_t> hldi(np_), hldg(np_);
  // leading dimension of an operator block with n columns: whole 16-byte units, an
  // odd number of them, so that lanes reading different rows at the same column hit
  // distinct shared-memory banks (the row kernels of the dual-primal sweep)
  const int esz_op = d->mixed ? 4 : 8;
  auto op_ld = [&](int n) {
    if (n <= 0) return 0;
    int l = (n + 3) / 4 * 4;
    if ((l * esz_op / 16) % 2 == 0) l += 16 / esz_op;
    return l;
  };
  for (int s = 0; s < np_; ++s) {
    const Patch &pt = hs.patches[s];
    hni[s] = pt.ni;
    hnb[s] = pt.nb;
    hnp[s] = pt.np;
    hn[s] = pt.ni + pt.nb + pt.np;
    hnn[s] = (hn[s] + pt.nb + pt.ni + 3) / 4 * 4;  // augmented [i b p | b' | i'], 16-byte rows (zero padded)
    hkofs[s + 1] = hkofs[s] + hn[s];
    hdoff[s + 1] = hdoff[s] + (int64_t)hnn[s] * hnn[s];
    hldi[s] = op_ld(pt.ni);
    hldg[s] = op_ld(pt.nb + pt.np);
    hig[s + 1] = hig[s] + (int64_t)hn[s] * hldi[s];
    hgt[s + 1] = hgt[s] + (int64_t)pt.ni * hldg[s];
    int ldb_s = op_ld(pt.nb), ldp_s = op_ld(pt.np);
    hldb[s] = ldb_s;
    hldp[s] = ldp_s;
    hh[s + 1] = hh[s] + (int64_t)(pt.nb + pt.np) * ldb_s;
    hq[s + 1] = hq[s] + (int64_t)pt.nb * ldp_s;
    hp[s + 1] = hp[s] + (int64_t)pt.nb * ldb_s;
    hbofs[s + 1] = hbofs[s] + pt.nb;
    hpofs[s + 1] = hpofs[s] + pt.np;
    d->max_ni = std::max(d->max_ni, pt.ni);
  }
  d->h_ni = hni;
  d->h_nb = hnb;
  d->h_np = hnp;
  d->NK = hkofs[np_];
  d->NBt = hbofs[np_];
  d->NPt = hpofs[np_];
  d->M = (int64_t)hs.lam.size();
  d->NC = hs.n_coarse;
  d->NF = (int64_t)hs.free_edges.size();
  // ---------------- kept space arrays and CSR (columns as absolute kept indices)
  std::vector<int64_t> kglob(d->NK), wptr(1, 0), mptr(1, 0), b_kept, p_kept;
  std::vector<double> kw(d->NK), wval, mval;
  std::vector<uint8_t> kown(d->NK, 0);
  std::vector<int32_t> wcol, mcol;
  std::vector<uint8_t> seen(hs.n_edges, 0);
  for (int s = 0; s < np_; ++s) {
    const Patch &pt = hs.patches[s];
    for (int k = 0; k < hn[s]; ++k) {
      int64_t g = pt.kept_glob[k];
      kglob[hkofs[s] + k] = g;
      kw[hkofs[s] + k] = pt.load_w[k];
      if (!seen[g]) {
        seen[g] = 1;
        kown[hkofs[s] + k] = 1;  // lowest patch id holding the DOF owns it
      }
      hrowpatch.push_back(s);
      hrowlocal.push_back(k);
      for (int t = pt.Wk.ptr[k]; t < pt.Wk.ptr[k + 1]; ++t) {
        wcol.push_back((int32_t)(hkofs[s] + pt.Wk.col[t]));
        wval.push_back(pt.Wk.val[t]);
      }
      wptr.push_back((int64_t)wcol.size());
      for (int t = pt.Mk.ptr[k]; t < pt.Mk.ptr[k + 1]; ++t) {
        mcol.push_back((int32_t)(hkofs[s] + pt.Mk.col[t]));
        mval.push_back(pt.Mk.val[t]);
      }
      mptr.push_back((int64_t)mcol.size());
    }
    for (int k = 0; k < pt.nb; ++k) b_kept.push_back(hkofs[s] + pt.ni + k);
    for (int k = 0; k < pt.np; ++k) p_kept.push_back(hkofs[s] + pt.ni + pt.nb + k);
  }
  if (d->NK >= (int64_t)INT32_MAX) {
    err = "kept space exceeds 2^31 entries";
    return fail(IETI_ERR_TOO_LARGE);
  }
  // ---------------- multipliers: B^T gather lists, jump pairs, scaling weights
  std::vector<double> rho(d->NBt, 1.0);
  if (opt.precond == IETI_PRECOND_DIRICHLET_STIFF)
    for (int s = 0; s < np_; ++s) {
      const Patch &pt = hs.patches[s];
      for (int k = 0; k < pt.nb; ++k) {
        int row = pt.ni + k;
        for (int t = pt.Wk.ptr[row]; t < pt.Wk.ptr[row + 1]; ++t)
          if (pt.Wk.col[t] == row) rho[hbofs[s] + k] = pt.Wk.val[t];
      }
    }
  std::vector<double> rho_sum(hs.n_edges, 0.0);
  for (int s = 0; s < np_; ++s)
    for (int k = 0; k < hs.patches[s].nb; ++k) rho_sum[hs.patches[s].kept_glob[hs.patches[s].ni + k]] += rho[hbofs[s] + k];
  int64_t m = d->M;
  std::vector<int32_t> qp(m), qm(m);
  std::vector<double> wp(m), wm(m);
  std::vector<std::vector<std::pair<int32_t, std::pair<double, double>>>> lists(d->NBt);
  for (int64_t l = 0; l < m; ++l) {
    const Multiplier &L = hs.lam[l];
    int64_t a = hbofs[L.s] + L.pos_s, b = hbofs[L.t] + L.pos_t;
    qp[l] = (int32_t)a;
    qm[l] = (int32_t)b;
    double rs = rho_sum[L.edge];
    wp[l] = rho[b] / rs;  // copy in s scaled by delta_t
    wm[l] = rho[a] / rs;
    lists[a].push_back({(int32_t)l, {1.0, wp[l]}});
    lists[b].push_back({(int32_t)l, {-1.0, -wm[l]}});
  }
  std::vector<int32_t> bt_ptr(1, 0), bt_lam;
  std::vector<double> bt_sgn, bt_wd;
  for (int64_t q = 0; q < d->NBt; ++q) {
    for (auto &e : lists[q]) {
      bt_lam.push_back(e.first);
      bt_sgn.push_back(e.second.first);
      bt_wd.push_back(e.second.second);
    }
    bt_ptr.push_back((int32_t)bt_lam.size());
  }
  // ---------------- coarse maps
  std::vector<int32_t> pc(d->NPt);
  std::vector<std::vector<int32_t>> copies(d->NC);
  for (int s = 0; s < np_; ++s) {
    const Patch &pt = hs.patches[s];
    for (int k = 0; k < pt.np; ++k) {
      int64_t c = hs.coarse_of_edge[pt.kept_glob[pt.ni + pt.nb + k]];
      if (d->coarse_nd) c = tree->perm[c];  // elimination order of the nested dissection
      pc[hpofs[s] + k] = (int32_t)c;
      copies[c].push_back((int32_t)(hpofs[s] + k));
    }
  }
  std::vector<int32_t> cptr(1, 0), cpos;
  for (int64_t c = 0; c < d->NC; ++c) {
    for (int32_t x : copies[c]) cpos.push_back(x);
    cptr.push_back((int32_t)cpos.size());
  }
  // free global DOFs -> kept copies (assembled residual norm)
  std::vector<std::vector<int64_t>> fcop(hs.n_edges);
  for (int64_t k = 0; k < d->NK; ++k) fcop[kglob[k]].push_back(k);
  std::vector<int64_t> fptr(1, 0), fpos, fglob(hs.free_edges);
  for (int64_t g : hs.free_edges) {
    for (int64_t k : fcop[g]) fpos.push_back(k);
    fptr.push_back((int64_t)fpos.size());
  }
  // ---------------- upload index data
  int rc;
  std::vector<int64_t> hkofs_v(hkofs.begin(), hkofs.end() - 1),
      hig_v(hig.begin(), hig.end() - 1), hgt_v(hgt.begin(), hgt.end() - 1), hh_v(hh.begin(), hh.end() - 1),
      hq_v(hq.begin(), hq.end() - 1), hp_v(hp.begin(), hp.end() - 1);
  int32_t *dnn = nullptr, *dn = nullptr, *drowpatch = nullptr, *drowlocal = nullptr;
  if ((rc = upload(d, &d->ni, hni, err)) || (rc = upload(d, &d->nb, hnb, err)) || (rc = upload(d, &d->npp, hnp, err)) ||
      (rc = upload(d, &d->kofs, hkofs_v, err)) ||
      (rc = upload(d, &d->igoff, hig_v, err)) || (rc = upload(d, &d->gtoff, hgt_v, err)) ||
      (rc = upload(d, &d->hoff, hh_v, err)) ||
      (rc = upload(d, &d->qoff, hq_v, err)) || (rc = upload(d, &d->poff, hp_v, err)) ||
      (rc = upload(d, &dnn, hnn, err)) || (rc = upload(d, &dn, hn, err)) ||
      (rc = upload(d, &drowpatch, hrowpatch, err)) ||
      (rc = upload(d, &drowlocal, hrowlocal, err)) || (rc = upload(d, &d->kglob, kglob, err)) ||
      (rc = upload(d, &d->kw, kw, err)) || (rc = upload(d, &d->kown, kown, err)) ||
      (rc = upload(d, &d->wptr, wptr, err)) || (rc = upload(d, &d->wcol, wcol, err)) ||
      (rc = upload(d, &d->wval, wval, err)) || (rc = upload(d, &d->mptr, mptr, err)) ||
      (rc = upload(d, &d->mcol, mcol, err)) || (rc = upload(d, &d->mval, mval, err)) ||
      (rc = upload(d, &d->b_kept, b_kept, err)) || (rc = upload(d, &d->p_kept, p_kept, err)) ||
      (rc = upload(d, &d->bt_ptr, bt_ptr, err)) || (rc = upload(d, &d->bt_lam, bt_lam, err)) ||
      (rc = upload(d, &d->bt_sgn, bt_sgn, err)) || (rc = upload(d, &d->bt_wd, bt_wd, err)) ||
      (rc = upload(d, &d->lam_qp, qp, err)) || (rc = upload(d, &d->lam_qm, qm, err)) ||
      (rc = upload(d, &d->lam_wp, wp, err)) || (rc = upload(d, &d->lam_wm, wm, err)) ||
      (rc = upload(d, &d->pc, pc, err)) || (rc = upload(d, &d->cptr, cptr, err)) ||
      (rc = upload(d, &d->cpos, cpos, err)) || (rc = upload(d, &d->fptr, fptr, err)) ||
      (rc = upload(d, &d->fpos, fpos, err)) || (rc = upload(d, &d->fglob, fglob, err)))
    return fail(rc);
  {
    std::vector<int64_t> hb(hbofs.begin(), hbofs.end() - 1), hpo(hpofs.begin(), hpofs.end() - 1);
    std::vector<int32_t> bp_(d->NBt);
    for (int s = 0; s < np_; ++s)
      for (int64_t k = hbofs[s]; k < hbofs[s + 1]; ++k) bp_[k] = s;
    if ((rc = upload(d, &d->ldb, hldb, err)) || (rc = upload(d, &d->ldp, hldp, err)) ||
        (rc = upload(d, &d->ldi, hldi, err)) || (rc = upload(d, &d->ldg, hldg, err)) ||
        (rc = upload(d, &d->bofs_d, hb, err)) || (rc = upload(d, &d->pofs_d, hpo, err)) ||
        (rc = upload(d, &d->bpatch, bp_, err)))
      return fail(rc);
  }
  // ---------------- GEMV descriptors
  {
    std::vector<int64_t> ao, xo, yi;
    std::vector<int32_t> nc;
    auto clear = [&]() { ao.clear(); xo.clear(); yi.clear(); nc.clear(); };
    // W_ii^{-1} rows: z_i = W_ii^{-1} f_i  (kept space)
    for (int s = 0; s < np_; ++s)
      for (int r = 0; r < hni[s]; ++r) {
        ao.push_back(hig[s] + (int64_t)r * hldi[s]);
        xo.push_back(hkofs[s]);
        yi.push_back(hkofs[s] + r);
        nc.push_back(hni[s]);
      }
    if ((rc = upload_desc(d, d->dIGi, ao, xo, yi, nc, err))) return fail(rc);
    clear();
    // G rows: g_[bp] = f_[bp] - G f_i
    for (int s = 0; s < np_; ++s)
      for (int r = hni[s]; r < hn[s]; ++r) {
        ao.push_back(hig[s] + (int64_t)r * hldi[s]);
        xo.push_back(hkofs[s]);
        yi.push_back(hkofs[s] + r);
        nc.push_back(hni[s]);
      }
    if ((rc = upload_desc(d, d->dIGg, ao, xo, yi, nc, err))) return fail(rc);
    clear();
    // G^T rows: a_i = z_i - G^T a_[bp]
    for (int s = 0; s < np_; ++s)
      for (int t = 0; t < hni[s]; ++t) {
        ao.push_back(hgt[s] + (int64_t)t * hldg[s]);
        xo.push_back(hkofs[s] + hni[s]);
        yi.push_back(hkofs[s] + t);
        nc.push_back(hnb[s] + hnp[s]);
      }
    if ((rc = upload_desc(d, d->dGT, ao, xo, yi, nc, err))) return fail(rc);
    clear();
    // H rows: [F u ; Psi^T u] -> bp (B-space then Pi-space)
    for (int s = 0; s < np_; ++s)
      for (int r = 0; r < hnb[s] + hnp[s]; ++r) {
        ao.push_back(hh[s] + (int64_t)r * hldb[s]);
        xo.push_back(hbofs[s]);
        yi.push_back(r < hnb[s] ? hbofs[s] + r : d->NBt + hpofs[s] + (r - hnb[s]));
        nc.push_back(hnb[s]);
      }
    if ((rc = upload_desc(d, d->dH, ao, xo, yi, nc, err))) return fail(rc);
    clear();
    // Psi rows: bp_b -= Psi qloc
    for (int s = 0; s < np_; ++s)
      for (int r = 0; r < hnb[s]; ++r) {
        ao.push_back(hq[s] + (int64_t)r * hldp[s]);
        xo.push_back(hpofs[s]);
        yi.push_back(hbofs[s] + r);
        nc.push_back(hnp[s]);
      }
    if ((rc = upload_desc(d, d->dQ, ao, xo, yi, nc, err))) return fail(rc);
    clear();
    // P rows (Dirichlet preconditioner S_bb)
    for (int s = 0; s < np_; ++s)
      for (int r = 0; r < hnb[s]; ++r) {
        ao.push_back(hp[s] + (int64_t)r * hldb[s]);
        xo.push_back(hbofs[s]);
        yi.push_back(hbofs[s] + r);
        nc.push_back(hnb[s]);
      }
    if ((rc = upload_desc(d, d->dP, ao, xo, yi, nc, err))) return fail(rc);
    clear();
    d->ldc = (int)((d->NC + 3) / 4 * 4);
    for (int64_t r = 0; r < d->NC; ++r) {
      ao.push_back(r * d->ldc);
      xo.push_back(0);
      yi.push_back(r);
      nc.push_back((int32_t)d->NC);
    }
    if ((rc = upload_desc(d, d->dS, ao, xo, yi, nc, err))) return fail(rc);
  }
  if (d->coarse_nd && (rc = coarse_nd_tables(d, *tree, err))) return fail(rc);
  // ---------------- work vectors
  if ((rc = dalloc(d, &d->a, hs.n_edges, err)) || (rc = dalloc(d, &d->j, hs.n_edges, err)) ||
      (opt.predictor && ((rc = dalloc(d, &d->a_prev, hs.n_edges, err)) ||
                         (rc = dalloc(d, &d->a_old, hs.n_edges, err)))) ||
      (opt.predictor == 2 && (rc = dalloc(d, &d->a_prev2, hs.n_edges, err))) ||
      (rc = dalloc(d, &d->rglob, hs.n_edges, err)) ||
      (rc = dalloc(d, &d->kf, d->NK, err)) || (rc = dalloc(d, &d->kx, d->NK, err)) ||
      (rc = dalloc(d, &d->kr, d->NK, err)) || (rc = dalloc(d, &d->kz, d->NK, err)) ||
      (rc = dalloc(d, &d->ka, d->NK, err)) || (rc = dalloc(d, &d->kt, d->NK, err)) ||
      (rc = dalloc(d, &d->kg, d->NK, err)) ||
      (rc = dalloc(d, &d->bp, d->NBt + d->NPt, err)) ||
      (rc = dalloc(d, &d->ub, d->NBt, err)) || (rc = dalloc(d, &d->gb, d->NBt, err)) ||
      (rc = dalloc(d, &d->gp, d->NPt, err)) || (rc = dalloc(d, &d->cc, d->NC, err)) ||
      (rc = dalloc(d, &d->q, d->NC, err)) || (rc = dalloc(d, &d->qloc, d->NPt, err)) ||
      (rc = dalloc(d, &d->lam, m, err)) || (rc = dalloc(d, &d->r, m, err)) || (rc = dalloc(d, &d->z, m, err)) ||
      (rc = dalloc(d, &d->p, m, err)) || (rc = dalloc(d, &d->Fp, m, err)) || (rc = dalloc(d, &d->dvec, m, err)) ||
      (rc = dalloc(d, &d->part, RED_BLOCKS, err)) || (rc = dalloc(d, &d->sc, 16, err)))
    return fail(rc);
  CK(cudaMallocHost((void **)&d->h_sc, 16 * sizeof(double)));
  CK(cudaMemsetAsync(d->a, 0, hs.n_edges * sizeof(double), d->stream));
  CK(cudaMemsetAsync(d->j, 0, hs.n_edges * sizeof(double), d->stream));
  CK(cudaMemsetAsync(d->rglob, 0, hs.n_edges * sizeof(double), d->stream));
  // ---------------- dense augmented blocks, partial Cholesky (FP64, or FP32 with
  // SIMT or tensor-core trailing updates), in batches of patches whose blocks fit one
  // arena (all patches at once when they fit in 64 GB and 40% of the free memory)
  const bool f32 = d->factor != IETI_FACTOR_FP64;
  const size_t dsz = f32 ? sizeof(float) : sizeof(double);
  size_t esz = d->mixed ? sizeof(float) : sizeof(double);
  std::vector<int> bstart{0};
  int64_t arena_elems = 0;
  {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const double cap = (opt.factor_arena_mb > 0 ? (double)opt.factor_arena_mb * 1048576.0
                                                 : std::min(64e9, 0.4 * (double)free_b)) / (double)dsz;
    int64_t acc = 0;
    for (int s = 0; s < np_; ++s) {
      const int64_t e = (int64_t)hnn[s] * hnn[s];
      if (acc > 0 && (double)(acc + e) > cap) {
        bstart.push_back(s);
        acc = 0;
      }
      acc += e;
      arena_elems = std::max(arena_elems, acc);
    }
    bstart.push_back(np_);
  }
  const int n_batches = (int)bstart.size() - 1;
  d->factor_batches = n_batches;
  double *D = nullptr;  // FP64 arena
  float *Df = nullptr;  // FP32 arena
  if (f32) {
    if ((rc = dalloc(d, &Df, arena_elems, err))) return fail(rc);
  } else if ((rc = dalloc(d, &D, arena_elems, err))) {
    return fail(rc);
  }
  void *Dv = f32 ? (void *)Df : (void *)D;
  // offsets of the blocks inside the arena, relative to their batch's first block
  std::vector<int64_t> hboff(np_);
  for (int b = 0; b < n_batches; ++b)
    for (int s = bstart[b]; s < bstart[b + 1]; ++s) hboff[s] = hdoff[s] - hdoff[bstart[b]];
  int64_t *dboff = nullptr;
  if ((rc = upload(d, &dboff, hboff, err))) return fail(rc);
  if (d->nonlinear && !hs.nl.patches.empty()) {
    // patches holding nonlinear elements: keep their blocks without the law (base of
    // every refactorization) and the quadrature tables of their nonlinear elements
    const NlTables &T = hs.nl;
    const int nb = (int)T.patches.size();
    d->nl_np = nb;
    d->nl_ne = (int64_t)T.nloc.size();
    d->nl_arena = 0;
    for (int b = 0; b < nb; ++b) {
      int sg = T.patches[b];
      d->nlh_ids.push_back(sg);
      d->nlh_nn.push_back(hnn[sg]);
      d->nlh_n.push_back(hn[sg]);
      d->nlh_ni.push_back(hni[sg]);
      d->nlh_nb.push_back(hnb[sg]);
      d->nlh_np.push_back(hnp[sg]);
      d->nlh_doff.push_back(d->nl_arena);
      d->nlh_pofs.push_back(hpofs[sg]);
      d->nl_arena += (int64_t)hnn[sg] * hnn[sg];
    }
    for (int e = 0; e < (int)d->nl_ne; ++e) {
      d->nl_max_nloc = std::max(d->nl_max_nloc, T.nloc[e]);
      d->nl_max_nq = std::max(d->nl_max_nq, T.nq[e]);
    }
    if (NL_QC * d->nl_max_nloc * (int)sizeof(float4) > 48 * 1024 ||
        (d->nl_max_nloc + 4 * d->nl_max_nq) * (int)sizeof(double) > 48 * 1024) {
      err = "nonlinear elements too large for the element kernels' shared memory";
      return fail(IETI_ERR_TOO_LARGE);
    }
    CK(cudaMalloc(&d->nl_base, (size_t)d->nl_arena * dsz));
    d->allocs.push_back(d->nl_base);
    CK(cudaMalloc(&d->nl_work, (size_t)d->nl_arena * dsz));
    d->allocs.push_back(d->nl_work);
    d->bytes += 2 * d->nl_arena * (int64_t)dsz;
    std::vector<int64_t> kofs_b, hoff_b, qoff_b, poff_b, igoff_b, gtoff_b;
    std::vector<int32_t> ldb_b, ldp_b, ldi_b, ldg_b;
    for (int b = 0; b < nb; ++b) {
      int sg = T.patches[b];
      kofs_b.push_back(hkofs[sg]);
      hoff_b.push_back(hh[sg]);
      qoff_b.push_back(hq[sg]);
      poff_b.push_back(hp[sg]);
      igoff_b.push_back(hig[sg]);
      gtoff_b.push_back(hgt[sg]);
      ldb_b.push_back(hldb[sg]);
      ldp_b.push_back(hldp[sg]);
      ldi_b.push_back(hldi[sg]);
      ldg_b.push_back(hldg[sg]);
    }
    std::vector<int32_t> zeros(nb, 0);
    std::vector<float4> tq0(std::max<size_t>(T.cq.size(), 1));
    if ((rc = upload(d, &d->nlb_doff, d->nlh_doff, err)) || (rc = upload(d, &d->nlb_kofs, kofs_b, err)) ||
        (rc = upload(d, &d->nlb_hoff, hoff_b, err)) || (rc = upload(d, &d->nlb_qoff, qoff_b, err)) ||
        (rc = upload(d, &d->nlb_poff, poff_b, err)) || (rc = upload(d, &d->nlb_igoff, igoff_b, err)) ||
        (rc = upload(d, &d->nlb_gtoff, gtoff_b, err)) || (rc = upload(d, &d->nlb_nn, d->nlh_nn, err)) ||
        (rc = upload(d, &d->nlb_n, d->nlh_n, err)) || (rc = upload(d, &d->nlb_ni, d->nlh_ni, err)) ||
        (rc = upload(d, &d->nlb_nb, d->nlh_nb, err)) || (rc = upload(d, &d->nlb_np, d->nlh_np, err)) ||
        (rc = upload(d, &d->nlb_ldb, ldb_b, err)) || (rc = upload(d, &d->nlb_ldp, ldp_b, err)) ||
        (rc = upload(d, &d->nlb_ldi, ldi_b, err)) || (rc = upload(d, &d->nlb_ldg, ldg_b, err)) ||
        (rc = upload(d, &d->nlb_kb, zeros, err)) || (rc = upload(d, &d->nlb_ke, zeros, err)) ||
        (rc = upload(d, &d->nlb_na, zeros, err)) || (rc = upload(d, &d->nlb_st, zeros, err)) ||
        (rc = upload(d, &d->nlb_sklo, zeros, err)) || (rc = upload(d, &d->nlb_skhi, zeros, err)) ||
        (rc = upload(d, &d->nlb_rlim, zeros, err)) || (rc = upload(d, &d->nlb_clim, zeros, err)) ||
        (rc = upload(d, &d->nl_G, T.G, err)) || (rc = upload(d, &d->nl_cq, T.cq, err)) ||
        (rc = upload(d, &d->nl_kept, T.kept, err)) || (rc = upload(d, &d->nl_glob, T.glob, err)) ||
        (rc = upload(d, &d->nl_goff, T.g_off, err)) || (rc = upload(d, &d->nl_qoff, T.q_off, err)) ||
        (rc = upload(d, &d->nl_doff, T.d_off, err)) || (rc = upload(d, &d->nl_nloc, T.nloc, err)) ||
        (rc = upload(d, &d->nl_nq, T.nq, err)) || (rc = upload(d, &d->nl_bpos, T.el_batch, err)) ||
        (rc = upload(d, &d->nl_tq, tq0, err)))
      return fail(rc);
  }
  // per-patch factorization controls (device copies; the kernels see a batch through
  // pointers offset to its first patch)
  std::vector<int32_t> hkb(np_), hke(np_), hna(np_);
  int32_t *dkb = nullptr, *dke = nullptr, *dna = nullptr, *dstat = nullptr;
  int32_t *dsklo = nullptr, *dskhi = nullptr, *drlim = nullptr, *dclim = nullptr;
  if ((rc = dalloc(d, &dkb, np_, err)) || (rc = dalloc(d, &dke, np_, err)) || (rc = dalloc(d, &dna, np_, err)) ||
      (rc = dalloc(d, &dstat, np_, err)) || (rc = dalloc(d, &dsklo, np_, err)) || (rc = dalloc(d, &dskhi, np_, err)) ||
      (rc = dalloc(d, &drlim, np_, err)) || (rc = dalloc(d, &dclim, np_, err)))
    return fail(rc);
  CK(cudaMemsetAsync(dstat, 0, np_ * sizeof(int32_t), d->stream));
  std::vector<int32_t> hsklo(np_), hskhi(np_), hrlim(np_), hclim(np_);
  auto put = [&](int32_t *dst, const std::vector<int32_t> &h) -> int {
    CK(cudaMemcpyAsync(dst, h.data(), np_ * 4, cudaMemcpyHostToDevice, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return IETI_OK;
  };
  int maxnb = *std::max_element(hnb.begin(), hnb.end());
  int maxnp = *std::max_element(hnp.begin(), hnp.end());
  int64_t maxP = (int64_t)maxnb * maxnb;
  int64_t maxH = 0, maxIG = 0;
  for (int s = 0; s < np_; ++s) {
    maxH = std::max(maxH, (int64_t)(hnb[s] + hnp[s]) * hnb[s]);
    maxIG = std::max(maxIG, (int64_t)hn[s] * hni[s]);
  }
  auto alloc_op = [&](void **ptr, int64_t n) -> int {
    cudaError_t e = cudaMalloc(ptr, std::max<int64_t>(n, 1) * esz);
    if (e != cudaSuccess) {
      err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
      return IETI_ERR_OOM;
    }
    d->allocs.push_back(*ptr);
    d->bytes += std::max<int64_t>(n, 1) * esz;
    return IETI_OK;
  };
  {
    // H, Q, P and the coarse operators are re-read every PCG iteration: one arena
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t bH = al(std::max<int64_t>(hh[np_], 1) * esz), bQ = al(std::max<int64_t>(hq[np_], 1) * esz),
           bP = al(std::max<int64_t>(hp[np_], 1) * esz),
           bS = al(std::max<int64_t>(d->coarse_nd ? d->nd_z_elems + d->nd_lt_elems : d->NC * d->ldc, 1) * 8);
    d->iter_bytes = bH + bQ + bP + bS;
    cudaError_t e = cudaMalloc((void **)&d->iter_arena, d->iter_bytes);
    if (e != cudaSuccess) {
      err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
      return fail(IETI_ERR_OOM);
    }
    d->allocs.push_back(d->iter_arena);
    d->bytes += d->iter_bytes;
    d->H = d->iter_arena;
    d->Q = d->iter_arena + bH;
    d->P = d->iter_arena + bH + bQ;
    d->Scoarse_slot = (double *)(d->iter_arena + bH + bQ + bP);
    if (d->coarse_nd) {
      d->nd_Z = d->Scoarse_slot;
      d->nd_Lt = d->nd_Z + d->nd_z_elems;
      CK(cudaMemsetAsync(d->Scoarse_slot, 0, bS, d->stream));  // row padding stays zero
    }
  }
  if ((rc = alloc_op(&d->IG, hig[np_])) || (rc = alloc_op(&d->GT, hgt[np_]))) return fail(rc);
  CK(cudaMemsetAsync(d->IG, 0, std::max<int64_t>(hig[np_], 1) * esz, d->stream));
  CK(cudaMemsetAsync(d->GT, 0, std::max<int64_t>(hgt[np_], 1) * esz, d->stream));
  CK(cudaMemsetAsync(d->P, 0, std::max<int64_t>(hp[np_], 1) * esz, d->stream));
  CK(cudaMemsetAsync(d->H, 0, std::max<int64_t>(hh[np_], 1) * esz, d->stream));
  CK(cudaMemsetAsync(d->Q, 0, std::max<int64_t>(hq[np_], 1) * esz, d->stream));
  // coarse accumulators: S_c (nested dissection) or [[S_c, I], [I, 0]] (dense inverse),
  // and for Newton the linear patches' part of S_c
  const int64_t nc = d->NC, ldS = d->coarse_nd ? nc : 2 * nc;
  double *Sc = nullptr;
  std::vector<uint8_t> is_nl(np_, 0);
  for (int sg : hs.nl.patches) is_nl[sg] = 1;
  if (nc > 0) {
    if ((rc = dalloc(d, &Sc, (size_t)(ldS * ldS), err))) return fail(rc);
    CK(cudaMemsetAsync(Sc, 0, (size_t)(ldS * ldS) * sizeof(double), d->stream));
    if (d->nl_np > 0) {
      if ((rc = dalloc(d, &d->sc_lin, (size_t)(nc * nc), err))) return fail(rc);
      CK(cudaMemsetAsync(d->sc_lin, 0, (size_t)(nc * nc) * sizeof(double), d->stream));
    }
  }
  d->t_factor_ms = 0;
  for (int bt = 0; bt < n_batches; ++bt) {
    const int s0 = bstart[bt], s1 = bstart[bt + 1], nbt = s1 - s0;
    const int64_t a0 = hdoff[s0], belems = hdoff[s1] - a0;
    CK(cudaMemsetAsync(Dv, 0, (size_t)belems * dsz, d->stream));
    {
      const int64_t r0 = hkofs[s0], nrows = hkofs[s1] - r0;
      unsigned g0 = grid_for(nrows * 32, 256);
      if (f32)
        k_csr_to_dense<float><<<g0, 256, 0, d->stream>>>(nrows, drowpatch + r0, drowlocal + r0, d->wptr + r0,
                                                         d->wcol, d->wval, d->kofs, dboff, dnn, Df);
      else
        k_csr_to_dense<double><<<g0, 256, 0, d->stream>>>(nrows, drowpatch + r0, drowlocal + r0, d->wptr + r0,
                                                          d->wcol, d->wval, d->kofs, dboff, dnn, D);
      int maxaug = 0;
      for (int s = s0; s < s1; ++s) maxaug = std::max({maxaug, hnb[s], hni[s]});
      if (maxaug > 0) {
        dim3 g(grid_for(maxaug, 128), nbt);
        if (f32)
          k_augment<float><<<g, 128, 0, d->stream>>>(nbt, d->ni + s0, d->nb + s0, dn + s0, dnn + s0, dboff + s0, Df);
        else
          k_augment<double><<<g, 128, 0, d->stream>>>(nbt, d->ni + s0, d->nb + s0, dn + s0, dnn + s0, dboff + s0, D);
      }
      d->launches_setup += 2;
    }
    CK(cudaGetLastError());
    // the nonlinear patches' blocks without the law: base of every refactorization
    for (int b = 0; b < d->nl_np; ++b) {
      const int sg = d->nlh_ids[b];
      if (sg < s0 || sg >= s1) continue;
      CK(cudaMemcpyAsync((char *)d->nl_base + d->nlh_doff[b] * dsz, (char *)Dv + hboff[sg] * dsz,
                         (size_t)hnn[sg] * hnn[sg] * dsz, cudaMemcpyDeviceToDevice, d->stream));
    }
    TcHost th;
    th.off.assign(hboff.begin() + s0, hboff.begin() + s1);
    th.ld.assign(hnn.begin() + s0, hnn.begin() + s1);
    AugLimits lim{dsklo + s0, dskhi + s0, drlim + s0, dclim + s0};
    auto slice = [&](const std::vector<int32_t> &v) { return std::vector<int32_t>(v.begin() + s0, v.begin() + s1); };
    // one partial-Cholesky phase over the batch in the chosen factor precision
    auto factor_phase = [&]() -> int {
      const std::vector<int32_t> kb = slice(hkb), ke = slice(hke), na = slice(hna);
      th.sk_lo = slice(hsklo);
      th.sk_hi = slice(hskhi);
      th.rlim = slice(hrlim);
      th.clim = slice(hclim);
      d->factor_flops += partial_chol_flops(th, kb, ke, na);
      if (d->factor == IETI_FACTOR_FP64)
        return potrf_partial<double>(d, D, dboff + s0, dnn + s0, kb, ke, na, dkb + s0, dke + s0, dna + s0,
                                     dstat + s0, lim, err);
      return potrf_partial_f32(d, d->factor, Df, dboff + s0, dnn + s0, th, kb, ke, na, dkb + s0, dke + s0,
                               dna + s0, dstat + s0, lim, err);
    };
    // phase A: interior pivots -> trailing [b p b'] = Schur complement; copy S_bb
    for (int s = s0; s < s1; ++s) {
      hkb[s] = 0;
      hke[s] = hni[s];
      hna[s] = hnn[s];
      hsklo[s] = hn[s];              // b' rows: zero in the interior columns
      hskhi[s] = hn[s] + hnb[s];
      hrlim[s] = INT32_MAX;          // i' rows: full updates (W_ii^{-1} and G^T come out of them)
      hclim[s] = 0;
    }
    if ((rc = put(dkb, hkb)) || (rc = put(dke, hke)) || (rc = put(dna, hna)) || (rc = put(dsklo, hsklo)) ||
        (rc = put(dskhi, hskhi)) || (rc = put(drlim, hrlim)) || (rc = put(dclim, hclim)))
      return fail(rc);
    CK(cudaEventRecord(d->ev0, d->stream));
    if ((rc = factor_phase())) return fail(rc);
    if (maxP > 0) {
      dim3 g(grid_for(maxP, 256), nbt);
      if (f32)
        k_extract_P<float, float><<<g, 256, 0, d->stream>>>(Df, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                            d->ldb + s0, d->poff + s0, (float *)d->P);
      else if (d->mixed)
        k_extract_P<double, float><<<g, 256, 0, d->stream>>>(D, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                             d->ldb + s0, d->poff + s0, (float *)d->P);
      else
        k_extract_P<double, double><<<g, 256, 0, d->stream>>>(D, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                              d->ldb + s0, d->poff + s0, (double *)d->P);
      d->launches_setup++;
    }
    // phase B: interface pivots -> trailing [p b'] = [[C_s, -Psi^T], [-Psi, -F_s]]
    for (int s = s0; s < s1; ++s) {
      hkb[s] = hni[s];
      hke[s] = hni[s] + hnb[s];
      hna[s] = hn[s] + hnb[s];       // the i' rows are done
      hsklo[s] = hskhi[s] = 0;
      hrlim[s] = INT32_MAX;
      hclim[s] = 0;
    }
    if ((rc = put(dkb, hkb)) || (rc = put(dke, hke)) || (rc = put(dna, hna)) || (rc = put(dsklo, hsklo)) ||
        (rc = put(dskhi, hskhi)) || (rc = put(drlim, hrlim)) || (rc = put(dclim, hclim)))
      return fail(rc);
    if ((rc = factor_phase())) return fail(rc);
    CK(cudaEventRecord(d->ev1, d->stream));
    {
      std::vector<int32_t> hstat(nbt);
      CK(cudaMemcpyAsync(hstat.data(), dstat + s0, nbt * 4, cudaMemcpyDeviceToHost, d->stream));
      CK(cudaStreamSynchronize(d->stream));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, d->ev0, d->ev1));
      d->t_factor_ms += ms;
      for (int s = s0; s < s1; ++s)
        if (hstat[s - s0]) {
          err = "local block of patch " + std::to_string(s) + " is not positive definite (pivot " +
                std::to_string(hstat[s - s0] - 1) + ")";
          return fail(IETI_ERR_NOT_SPD);
        }
    }
    if (maxH > 0) {
      dim3 g((unsigned)std::min<int64_t>(grid_for(maxH, 256), 4096), nbt);
      if (f32)
        k_extract_ops<float, float><<<g, 256, 0, d->stream>>>(Df, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                              d->npp + s0, d->ldb + s0, d->ldp + s0, d->hoff + s0,
                                                              d->qoff + s0, (float *)d->H, (float *)d->Q);
      else if (d->mixed)
        k_extract_ops<double, float><<<g, 256, 0, d->stream>>>(D, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                               d->npp + s0, d->ldb + s0, d->ldp + s0, d->hoff + s0,
                                                               d->qoff + s0, (float *)d->H, (float *)d->Q);
      else
        k_extract_ops<double, double><<<g, 256, 0, d->stream>>>(D, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                                d->npp + s0, d->ldb + s0, d->ldp + s0, d->hoff + s0,
                                                                d->qoff + s0, (double *)d->H, (double *)d->Q);
      d->launches_setup++;
    }
    if (maxIG > 0) {
      dim3 g((unsigned)std::min<int64_t>(grid_for(maxIG, 256), 4096), nbt);
      if (f32)
        k_extract_IG<float, float><<<g, 256, 0, d->stream>>>(Df, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                             d->npp + s0, d->ldi + s0, d->ldg + s0, d->igoff + s0,
                                                             d->gtoff + s0, (float *)d->IG, (float *)d->GT);
      else if (d->mixed)
        k_extract_IG<double, float><<<g, 256, 0, d->stream>>>(D, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                              d->npp + s0, d->ldi + s0, d->ldg + s0, d->igoff + s0,
                                                              d->gtoff + s0, (float *)d->IG, (float *)d->GT);
      else
        k_extract_IG<double, double><<<g, 256, 0, d->stream>>>(D, dboff + s0, dnn + s0, d->ni + s0, d->nb + s0,
                                                               d->npp + s0, d->ldi + s0, d->ldg + s0, d->igoff + s0,
                                                               d->gtoff + s0, (double *)d->IG, (double *)d->GT);
      d->launches_setup++;
    }
    // coarse contributions C_s of the batch (one launch per patch, in patch order)
    for (int s = s0; s < s1 && nc > 0; ++s) {
      if (hnp[s] == 0) continue;
      const int64_t cnt = (int64_t)hnp[s] * hnp[s];
      for (int lin = 0; lin < (d->nl_np > 0 && !is_nl[s] ? 2 : 1); ++lin) {
        double *dst = lin ? d->sc_lin : Sc;
        const int64_t ldd = lin ? nc : ldS;
        if (f32)
          k_coarse_add<float><<<grid_for(cnt, 256), 256, 0, d->stream>>>(Df, hboff[s], hnn[s], hni[s], hnb[s],
                                                                         hnp[s], d->pc + hpofs[s], dst, ldd);
        else
          k_coarse_add<double><<<grid_for(cnt, 256), 256, 0, d->stream>>>(D, hboff[s], hnn[s], hni[s], hnb[s],
                                                                          hnp[s], d->pc + hpofs[s], dst, ldd);
        d->launches_setup++;
      }
    }
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(d->stream));
  cudaFree(Dv);
  d->allocs.erase(std::find(d->allocs.begin(), d->allocs.end(), Dv));
  d->bytes -= arena_elems * (int64_t)dsz;
  // ---------------- coarse: S_c = sum_s A_s^T C_s A_s, factored along the nested
  // dissection, or inverted through [[S_c, I], [I, 0]]
  if (nc > 0 && d->coarse_nd) {
    auto tc0 = std::chrono::steady_clock::now();
    rc = coarse_nd_factor(d, *tree, Sc, err);
    if (rc == IETI_OK && d->mixed) {
      // the mixed path streams the blocks as (hi, lo) FP32 pairs (in place: same 8 bytes)
      const int64_t n = d->nd_z_elems + d->nd_lt_elems;
      k_split_pairs<<<grid_for(n, 256), 256, 0, d->stream>>>(n, d->nd_Z, (float2 *)d->nd_Z);
      d->launches_setup++;
    }
    cudaStreamSynchronize(d->stream);
    if (d->nl_np > 0) {
      d->sc_aug = Sc;  // the assembled S_c of every Newton refactorization
    } else {
      cudaFree(Sc);
      d->allocs.erase(std::find(d->allocs.begin(), d->allocs.end(), (void *)Sc));
      d->bytes -= (int64_t)(ldS * ldS) * 8;
    }
    if (rc) return fail(rc);
    d->t_coarse_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc0).count();
  } else if (nc > 0) {
    k_coarse_identity<<<grid_for(nc, 256), 256, 0, d->stream>>>((int)nc, Sc, ldS);
    if ((rc = coarse_factor(d, Sc, err))) return fail(rc);
    CK(cudaStreamSynchronize(d->stream));
    if (d->nl_np > 0) {
      d->sc_aug = Sc;  // reused by the full refactorizations
      if ((rc = coarse_block_setup(d, pc, err))) return fail(rc);
    } else {
      cudaFree(Sc);
      d->allocs.erase(std::find(d->allocs.begin(), d->allocs.end(), (void *)Sc));
      d->bytes -= (int64_t)(ldS * ldS) * 8;
    }
  }
  CK(cudaStreamSynchronize(d->stream));
  CK(cudaGetLastError());
  // algorithmic bytes of one PCG iteration: H and Psi once each (F apply), P once
  // (preconditioner), S_c^{-1} once, plus the lambda / B-space vectors
  d->bytes_iter = (int64_t)esz * (hh[np_] + hq[np_] + hp[np_]) +
                  (d->coarse_nd ? (int64_t)d->nd_bytes : 8 * d->NC * d->NC) +
                  8 * (12 * d->M + 6 * d->NBt + 4 * d->NPt);
  {
    // ---- persistent PCG plan: one CTA per SM, three TMA stages of at most 64 KB (the
    // rule), or the autotuner's choice at the end of setup
    for (int s = 0; s < np_; ++s) d->ldmax = std::max({d->ldmax, hldb[s], hldp[s], hldi[s], hldg[s]});
    d->plan_ld[0] = hldb;  // H rows: [F_s; Psi_s^T]
    d->plan_rows[0].resize(np_);
    for (int s = 0; s < np_; ++s) d->plan_rows[0][s] = hnb[s] + hnp[s];
    d->plan_rows[1] = hnb;  // interface rows (Psi and S_bb)
    d->plan_ld[1] = hldb;
    d->plan_rows[2] = hn;   // IG rows
    d->plan_ld[2] = hldi;
    d->plan_rows[3] = hni;  // GT rows
    d->plan_ld[3] = hldg;
    d->plan_rows[4] = hnb;  // interface rows for Psi (own partition when the autotuner picks one)
    d->plan_ld[4] = hldp;
    int coop = 0;
    CK(cudaDeviceGetAttribute(&d->n_sm, cudaDevAttrMultiProcessorCount, d->device));
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, d->device));
    if (!coop) {
      err = "device cannot run the cooperative PCG kernel";
      return fail(IETI_ERR_CUDA);
    }
    PcgSched rule;
    if ((rc = pcg_rule(d, &rule, err)) || (rc = pcg_plan(d, rule, err))) return fail(rc);
    // fixed-width gather lists (an edge DOF is shared by at most 4 patches)
    std::vector<int32_t> ell_l(d->NBt * BT_W, -1), cpp(d->NC * CP_W, -1);
    std::vector<double> ell_s(d->NBt * BT_W, 0.0), ell_w(d->NBt * BT_W, 0.0);
    for (int64_t q = 0; q < d->NBt; ++q) {
      if (bt_ptr[q + 1] - bt_ptr[q] > BT_W) {
        err = "an interface copy has more than 3 multipliers";
        return fail(IETI_ERR_INVALID_ARG);
      }
      for (int t = bt_ptr[q]; t < bt_ptr[q + 1]; ++t) {
        ell_l[q * BT_W + (t - bt_ptr[q])] = bt_lam[t];
        ell_s[q * BT_W + (t - bt_ptr[q])] = bt_sgn[t];
        ell_w[q * BT_W + (t - bt_ptr[q])] = bt_wd[t];
      }
    }
    for (int64_t c = 0; c < d->NC; ++c) {
      if (cptr[c + 1] - cptr[c] > CP_W) {
        err = "a primal DOF has more than 4 copies";
        return fail(IETI_ERR_INVALID_ARG);
      }
      for (int t = cptr[c]; t < cptr[c + 1]; ++t) cpp[c * CP_W + (t - cptr[c])] = cpos[t];
    }
    if ((rc = upload(d, &d->ell_lam, ell_l, err)) || (rc = upload(d, &d->ell_sgn, ell_s, err)) ||
        (rc = upload(d, &d->ell_wd, ell_w, err)) || (rc = upload(d, &d->cp_pos, cpp, err)))
      return fail(rc);
    {
      // interface-copy neighbour lists of the two products through the multipliers the
      // preconditioner needs every iteration: entry 0 is the copy itself, entries 1..3
      // the other copies of its edge DOF (one multiplier joins the copy to each)
      //   (B_D^T B v)_q = sum_t wd_qt (v[qp(l_t)] - v[qm(l_t)])          -> coefficients ca
      //   (B^T B_D v)_q = sum_t sgn_qt (wp_l v[qp(l_t)] - wm_l v[qm(l_t)]) -> coefficients cb
      const bool scaled = opt.precond == IETI_PRECOND_DIRICHLET_MULT || opt.precond == IETI_PRECOND_DIRICHLET_STIFF;
      std::vector<int32_t> nidx(d->NBt * NB_W, -1);
      std::vector<double> nca(d->NBt * NB_W, 0.0), ncb(d->NBt * NB_W, 0.0);
      for (int64_t q = 0; q < d->NBt; ++q) {
        nidx[q * NB_W] = (int32_t)q;
        int e = 1;
        for (int t = bt_ptr[q]; t < bt_ptr[q + 1]; ++t) {
          const int32_t l = bt_lam[t];
          const bool plus = qp[l] == (int32_t)q;
          const int32_t other = plus ? qm[l] : qp[l];
          const double wdq = scaled ? bt_wd[t] : bt_sgn[t], sg = bt_sgn[t];
          const double wpl = scaled ? wp[l] : 1.0, wml = scaled ? wm[l] : 1.0;
          // v[qp] carries +1 (ca) / +wp (cb), v[qm] carries -1 / -wm
          const double a_self = plus ? wdq : -wdq, a_other = -a_self;
          const double b_self = plus ? sg * wpl : -sg * wml, b_other = plus ? -sg * wml : sg * wpl;
          nca[q * NB_W] += a_self;
          ncb[q * NB_W] += b_self;
          nidx[q * NB_W + e] = other;
          nca[q * NB_W + e] = a_other;
          ncb[q * NB_W + e] = b_other;
          ++e;
        }
      }
      if ((rc = upload(d, &d->nb_idx, nidx, err)) || (rc = upload(d, &d->nb_ca, nca, err)) ||
          (rc = upload(d, &d->nb_cb, ncb, err)) || (rc = dalloc(d, &d->yv0, d->NBt, err)) ||
          (rc = dalloc(d, &d->yv1, d->NBt, err)))
        return fail(rc);
    }
    if ((rc = dalloc(d, &d->p1, m, err)) || (rc = dalloc(d, &d->r1, m, err)) || (rc = dalloc(d, &d->zb, d->NBt, err)) ||
        (rc = dalloc(d, &d->zf, d->NBt, err)) || (rc = dalloc(d, &d->ubp, d->NBt, err)) ||
        (rc = dalloc(d, &d->ub1, d->NBt, err)) || (rc = dalloc(d, &d->uz, d->NBt, err)) ||
        (rc = dalloc(d, &d->tpi, d->NPt, err)) || (rc = dalloc(d, &d->zp, d->NBt, err)) ||
        (rc = dalloc(d, &d->ccg, d->NC, err)) || (rc = dalloc(d, &d->ppart, 4 * (size_t)PCG_MAX_CPS * d->n_sm, err)) ||
        (rc = dalloc(d, &d->bar, 4, err)) || (rc = dalloc(d, &d->pcg_its, 1, err)) ||
        (rc = dalloc(d, &d->pcg_rr, 1, err)) || (rc = dalloc(d, &d->pcg_dd, 1, err)) ||
        (rc = dalloc(d, &d->trace, TRACE_IT * TRACE_SLOTS, err)))
      return fail(rc);
    CK(cudaMemsetAsync(d->p, 0, m * sizeof(double), d->stream));
    CK(cudaMemsetAsync(d->p1, 0, m * sizeof(double), d->stream));
    if (opt.l2_persist == 2) {
      // keep about 60% of the L2 for the per-iteration operators, the rest for the
      // vectors and the per-sweep streams
      int l2 = 0;
      CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, d->device));
      if (l2 > 0 && d->iter_bytes > 0)
        d->l2_keep_frac = (float)std::min(1.0, 0.6 * (double)l2 / (double)d->iter_bytes);
    } else if (opt.l2_persist == 1) {
      int max_persist = 0, max_window = 0;
      CK(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, d->device));
      CK(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, d->device));
      if (max_persist > 0 && max_window > 0) {
        CK(cudaDeviceGetLimit(&d->l2_prev_limit, cudaLimitPersistingL2CacheSize));
        size_t want = std::min((size_t)max_persist, d->iter_bytes);
        CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, std::max(want, d->l2_prev_limit)));
        d->l2_set = true;
        d->l2_window = std::min((size_t)max_window, d->iter_bytes);
        d->l2_hit_ratio = (float)std::min(1.0, (double)want / (double)d->l2_window);
      }
    }
    int64_t sH = 0, sQ = 0, sP = 0;
    for (int s = 0; s < np_; ++s) {
      sH += (int64_t)(hnb[s] + hnp[s]) * hnb[s];
      sQ += (int64_t)hnb[s] * hnp[s];
      sP += (int64_t)hnb[s] * hnb[s];
    }
    d->bytes_iter_alg = (double)esz * (sH + sQ + sP) + (d->coarse_nd ? d->nd_bytes : 8.0 * (double)d->NC * d->NC) +
                        8.0 * (14.0 * d->M + 8.0 * d->NBt + 2.0 * d->NPt + 2.0 * d->NC);
  }
  {
    // algorithmic bytes of one launch: every operator entry once, input vectors once per patch, outputs once
    double e = (double)esz;
    d->gemv_bytes[IETI_K_GEMV_H] = e * hh[np_] + 8.0 * (d->NBt + d->NBt + d->NPt);
    d->gemv_bytes[IETI_K_GEMV_Q] = e * hq[np_] + 8.0 * (d->NPt + 2 * d->NBt);
    d->gemv_bytes[IETI_K_GEMV_P] = e * hp[np_] + 8.0 * (2 * d->NBt);
    d->gemv_bytes[IETI_K_GEMV_S] = 8.0 * (double)d->NC * d->NC + 16.0 * d->NC;
    int64_t sy = 0, sl = 0;
    for (int s = 0; s < np_; ++s) {
      sy += (int64_t)(hnb[s] + hnp[s]) * hni[s];
      sl += (int64_t)hni[s] * hni[s];
    }
    d->gemv_bytes[IETI_K_GEMV_Y] = e * sy + 8.0 * (2 * (double)d->NK);
    d->gemv_bytes[IETI_K_TRI] = e * sl + 8.0 * 2 * (double)d->NK;
    d->bytes_sweep_alg = e * (2.0 * sy + sl) + 8.0 * 6 * (double)d->NK;
    d->gemv_bytes[IETI_K_SPMV] = 12.0 * (double)wval.size() + 8.0 * 3 * (double)d->NK;
  }
  if (d->nl_np > 0) {
    // operators of the nonlinear patches at the initial state a = 0 (the tangent there)
    if ((rc = nl_refactor_any(d, err))) return fail(rc);
    CK(cudaStreamSynchronize(d->stream));
    d->refactors = 0;
  }
  if (opt.deflation && (rc = d->mixed ? deflation_setup<float>(d, hs, err) : deflation_setup<double>(d, hs, err)))
    return fail(rc);
  if (opt.autotune && opt.pcg_mode == 0) {
    rc = d->mixed ? pcg_autotune<float>(d, err) : pcg_autotune<double>(d, err);
    if (rc) return fail(rc);
  }
  if (opt.graph && opt.pcg_mode == 0 && d->nl_np == 0 && !opt.profile && d->l2_window == 0) {
    // the sweep loop of every step as one CUDA graph; without it (a graph call that
    // fails here) the host loop runs the same sweeps
    if ((rc = dalloc(d, &d->ctl, 1, err))) return fail(rc);
    CK(cudaMallocHost((void **)&d->h_ctl, sizeof(StepCtl)));
    std::string gerr;
    if ((d->mixed ? graph_build<float>(d, gerr) : graph_build<double>(d, gerr)) != IETI_OK) graph_release(d);
  }
  d->opt.tune_cache = nullptr;  // caller-owned, read during setup only
  d->t_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  (void)maxnp;
  *out = d;
  return IETI_OK;
}

int device_step(DeviceState *d, const double *j, int j_mem, ieti_stats *st, std::string &err) {
  CK(cudaSetDevice(d->device));
  CK(cudaMemcpyAsync(d->j, j, d->n_edges * sizeof(double),
                     j_mem == IETI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, d->stream));
  CK(cudaEventRecord(d->ev0, d->stream));
  d->nlaunch = 0;
  int rc = d->mixed ? step_impl<float>(d, st, err) : step_impl<double>(d, st, err);
  CK(cudaEventRecord(d->ev1, d->stream));
  CK(cudaEventSynchronize(d->ev1));
  // the carve-out only serves the iterations inside a step: return its lines to
  // normal so that whatever runs between steps can evict them
  if (d->l2_window > 0) CK(cudaCtxResetPersistingL2Cache());
  if (d->l2_keep_frac > 0.f) {
    const int64_t lines = (int64_t)(d->iter_bytes / 128);
    k_l2_demote<<<grid_for(lines, 256), 256, 0, d->stream>>>(d->iter_arena, lines);
    CK(cudaGetLastError());
  }
  prof_collect(d);
  if (st) {
    float ms = 0;
    cudaEventElapsedTime(&ms, d->ev0, d->ev1);
    st->t_step_ms = ms;
    st->kernel_launches = d->nlaunch;
  }
  return rc;
}

int device_solution(DeviceState *d, double *a, int64_t len, int mem, std::string &err) {
  CK(cudaSetDevice(d->device));
  CK(cudaMemcpyAsync(a, d->a, len * sizeof(double),
                     mem == IETI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return IETI_OK;
}

int device_set_state(DeviceState *d, const double *a, int64_t len, int mem, std::string &err) {
  CK(cudaSetDevice(d->device));
  CK(cudaMemcpyAsync(d->a, a, len * sizeof(double),
                     mem == IETI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, d->stream));
  // eliminated entries are 0 by definition: rebuild them from the owner map
  CK(cudaMemsetAsync(d->kx, 0, d->NK * sizeof(double), d->stream));
  k_gather_kept<<<grid_for(d->NK, 256), 256, 0, d->stream>>>(d->NK, d->kglob, d->a, d->kx);
  CK(cudaMemsetAsync(d->a, 0, d->n_edges * sizeof(double), d->stream));
  k_owner_add<<<grid_for(d->NK, 256), 256, 0, d->stream>>>(d->NK, d->kglob, d->kown, d->kx, d->a);
  CK(cudaStreamSynchronize(d->stream));
  d->n_hist = 0;  // no history for the extrapolation of the next step
  return IETI_OK;
}

void device_info(const DeviceState *d, ieti_info *info) {
  info->n_lambda = d->M;
  info->n_coarse = d->NC;
  info->bytes_iter = (int64_t)d->bytes_iter_alg;
  info->bytes_device = d->bytes;
  info->t_setup_device_ms = d->t_setup_ms;
  info->kernel_launches_setup = d->launches_setup;
  info->l2_window_bytes = (int64_t)d->l2_window;
  info->l2_hit_ratio = d->l2_hit_ratio;
  info->iter_operator_bytes = (int64_t)d->iter_bytes;
  info->t_factor_ms = d->t_factor_ms;
  info->tc_ms = d->tc_ms;
  info->tc_flops = d->tc_flops;
  info->tc_useful_flops = d->tc_useful_flops;
  info->tc_launches = d->tc_launches;
  info->factor_flops = d->factor_flops;
  info->nl_patches = d->nl_np;
  info->nl_elements = d->nl_ne;
  info->refactors = d->refactors;
  info->nl_coarse_block = d->cN;
  for (int k = 0; k < 4; ++k) info->t_refactor_ms[k] = d->t_refactor_ms[k];
  info->step_graph = d->gexec != nullptr;
  info->pcg_grid = d->G;
  info->pcg_stages = d->n_stages;
  info->pcg_stage_bytes = (int32_t)d->stage_bytes;
  info->pcg_psi_partition = d->psi_overhead;
  info->pcg_sched_source = d->sched_source;
  info->tune_candidates = d->tune_candidates;
  info->tune_ms = d->tune_ms;
  info->tune_us_per_it[0] = d->tune_us[0];
  info->tune_us_per_it[1] = d->tune_us[1];
  info->coarse_mode = d->NC == 0 ? 0 : (d->coarse_nd ? IETI_COARSE_ND : IETI_COARSE_DENSE);
  info->coarse_nodes = d->nd_nodes;
  info->coarse_levels = d->coarse_nd ? d->nd_H + std::max(d->nd_D - 1, 0) : (d->NC > 0 ? 1 : 0);
  info->coarse_bytes = d->coarse_nd ? d->nd_bytes : 8.0 * (double)d->NC * d->NC;
  info->t_coarse_ms = d->t_coarse_ms;
  info->factor_batches = d->factor_batches;
  info->pcg_seg_weight = d->seg_overhead;
  info->coarse_flow = d->nd_flow;
  info->deflation_dim = d->defl_k;
}

void device_kernel_stats(DeviceState *d, ieti_kernel_stat *out, bool reset) {
  prof_collect(d);
  for (int c = 0; c < IETI_K_NCLASS; ++c) out[c] = d->kstat[c];
  if (reset)
    for (int c = 0; c < IETI_K_NCLASS; ++c) d->kstat[c] = ieti_kernel_stat{};
}

void device_coarse_level_times(DeviceState *d, double *us, int n, bool reset) {
  const int nl = std::min(TRACE_ND, d->coarse_nd ? d->nd_H + std::max(d->nd_D - 1, 0) : 0);
  for (int k = 0; k < n; ++k) {
    const int lv = k / 4, part = k % 4;
    us[k] = (lv < nl && d->trace_nd_n) ? d->trace_nd[lv][part] / d->trace_nd_n : 0.0;
  }
  if (reset) {
    for (auto &row : d->trace_nd)
      for (double &v : row) v = 0;
    d->trace_nd_n = 0;
  }
}

void device_pcg_trace(DeviceState *d, double *work_us, double *wait_us, double *sub_us, bool reset) {
  for (int ph = 0; ph < 6; ++ph) {
    work_us[ph] = d->trace_n ? d->trace_acc[ph] / d->trace_n : 0.0;
    wait_us[ph] = d->trace_n ? d->trace_wait[ph] / d->trace_n : 0.0;
  }
  if (sub_us)
    for (int k = 0; k < 4; ++k)
      for (int j = 0; j < 3; ++j) sub_us[3 * k + j] = d->trace_sub_n[k] ? d->trace_sub[k][j] / d->trace_sub_n[k] : 0.0;
  if (reset) {
    for (int ph = 0; ph < 8; ++ph) d->trace_acc[ph] = d->trace_wait[ph] = 0;
    for (int k = 0; k < 4; ++k) {
      d->trace_sub[k][0] = d->trace_sub[k][1] = d->trace_sub[k][2] = 0;
      d->trace_sub_n[k] = 0;
    }
    d->trace_n = 0;
  }
}

void device_destroy(DeviceState *d) {
  if (!d) return;
  graph_release(d);
  if (d->h_ctl) cudaFreeHost(d->h_ctl);
  if (d->l2_set) {
    if (d->device >= 0) cudaSetDevice(d->device);
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, d->l2_prev_limit);
  }
  for (cudaEvent_t e : d->ev_pool) cudaEventDestroy(e);
  if (d->device >= 0) cudaSetDevice(d->device);
  if (d->stream) cudaStreamSynchronize(d->stream);
  for (void *p : d->allocs) cudaFree(p);
  if (d->h_sc) cudaFreeHost(d->h_sc);
  if (d->ev0) cudaEventDestroy(d->ev0);
  if (d->ev1) cudaEventDestroy(d->ev1);
  delete d;
}

}  // namespace ieti

namespace ieti {

// standalone batched partial Cholesky on caller memory (descriptor scratch allocated here)
int device_potrf_batched(int batch, double *base, const int64_t *off, const int32_t *n, const int32_t *npiv,
                         int32_t *status, cudaStream_t st, std::string &err) {
  std::vector<int32_t> hkb(batch, 0), hke(npiv, npiv + batch), hna(n, n + batch), hz(batch, 0),
      hbig(batch, INT32_MAX);
  std::vector<int64_t> hoff(off, off + batch);
  std::vector<int32_t> hn(n, n + batch);
  // one device block holds every descriptor array and the status words
  size_t bytes = (size_t)batch * (sizeof(int64_t) + 8 * sizeof(int32_t));
  unsigned char *blk = nullptr;
  cudaError_t e = cudaMalloc((void **)&blk, bytes);
  if (e != cudaSuccess) {
    err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
    return IETI_ERR_OOM;
  }
  int64_t *doff = (int64_t *)blk;
  int32_t *dn = (int32_t *)(doff + batch), *dkb = dn + batch, *dke = dkb + batch, *dna = dke + batch,
          *dst = dna + batch, *dz = dst + batch, *dbig = dz + batch, *dz2 = dbig + batch;
  int rc = IETI_OK;
  auto cp = [&](void *dst_, const void *src, size_t nbytes) {
    if (rc == IETI_OK && cudaMemcpyAsync(dst_, src, nbytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      err = "cudaMemcpyAsync failed";
      rc = IETI_ERR_CUDA;
    }
  };
  cp(doff, hoff.data(), batch * 8);
  cp(dn, hn.data(), batch * 4);
  cp(dkb, hkb.data(), batch * 4);
  cp(dke, hke.data(), batch * 4);
  cp(dna, hna.data(), batch * 4);
  cp(dz, hz.data(), batch * 4);
  cp(dbig, hbig.data(), batch * 4);
  cp(dz2, hz.data(), batch * 4);
  if (rc == IETI_OK && cudaMemsetAsync(dst, 0, batch * 4, st) != cudaSuccess) rc = IETI_ERR_CUDA;
  if (rc == IETI_OK) {
    DeviceState tmp;
    tmp.stream = st;
    AugLimits lim{dz, dz2, dbig, dz};
    rc = potrf_partial<double>(&tmp, base, doff, dn, hkb, hke, hna, dkb, dke, dna, dst, lim, err);
  }
  if (rc == IETI_OK) {
    if (cudaMemcpyAsync(status, dst, batch * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      err = std::string("batched partial Cholesky failed: ") + cudaGetErrorString(cudaGetLastError());
      rc = IETI_ERR_CUDA;
    }
  }
  cudaStreamSynchronize(st);
  cudaFree(blk);
  return rc;
}

// standalone FP32 batched partial Cholesky (SIMT, or tensor-core trailing updates)
int device_potrf_batched_f32(int batch, float *base, const int64_t *off, const int32_t *n, const int32_t *ld,
                             const int32_t *npiv, int factor, int32_t *status, cudaStream_t st, std::string &err) {
  std::vector<int32_t> hkb(batch, 0), hke(npiv, npiv + batch), hna(n, n + batch);
  TcHost th;
  th.off.assign(off, off + batch);
  th.ld.assign(ld, ld + batch);
  th.sk_lo.assign(batch, 0);
  th.sk_hi.assign(batch, 0);
  th.rlim.assign(batch, INT32_MAX);
  th.clim.assign(batch, 0);
  size_t bytes = (size_t)batch * (sizeof(int64_t) + 9 * sizeof(int32_t));
  unsigned char *blk = nullptr;
  cudaError_t e = cudaMalloc((void **)&blk, bytes);
  if (e != cudaSuccess) {
    err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
    return IETI_ERR_OOM;
  }
  int64_t *doff = (int64_t *)blk;
  int32_t *dld = (int32_t *)(doff + batch), *dkb = dld + batch, *dke = dkb + batch, *dna = dke + batch,
          *dst = dna + batch, *dz = dst + batch, *dbig = dz + batch, *dz2 = dbig + batch;
  int rc = IETI_OK;
  auto cp = [&](void *dst_, const void *src, size_t nbytes) {
    if (rc == IETI_OK && cudaMemcpyAsync(dst_, src, nbytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      err = "cudaMemcpyAsync failed";
      rc = IETI_ERR_CUDA;
    }
  };
  cp(doff, th.off.data(), batch * 8);
  cp(dld, th.ld.data(), batch * 4);
  cp(dkb, hkb.data(), batch * 4);
  cp(dke, hke.data(), batch * 4);
  cp(dna, hna.data(), batch * 4);
  cp(dz, th.sk_lo.data(), batch * 4);
  cp(dbig, th.rlim.data(), batch * 4);
  cp(dz2, th.sk_hi.data(), batch * 4);
  if (rc == IETI_OK && cudaMemsetAsync(dst, 0, batch * 4, st) != cudaSuccess) rc = IETI_ERR_CUDA;
  if (rc == IETI_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = IETI_ERR_CUDA;
  if (rc == IETI_OK) {
    DeviceState tmp;
    tmp.stream = st;
    AugLimits lim{dz, dz2, dbig, dz};
    rc = potrf_partial_f32(&tmp, factor, base, doff, dld, th, hkb, hke, hna, dkb, dke, dna, dst, lim, err);
  }
  if (rc == IETI_OK) {
    if (cudaMemcpyAsync(status, dst, batch * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      err = std::string("batched partial Cholesky failed: ") + cudaGetErrorString(cudaGetLastError());
      rc = IETI_ERR_CUDA;
    }
  }
  cudaStreamSynchronize(st);
  cudaFree(blk);
  return rc;
}

}  // namespace ieti

namespace ieti {

// Scratch of ieti_potrf_batched_noalloc: per matrix one int64 offset and eight int32
// words (size, first pivot, pivot end, active rows, status, two zero words, one
// "no limit" word).  Held by every device that loads the library.
constexpr int NOALLOC_MAX = IETI_NOALLOC_MAX_BATCH;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_MAX * (8 + 8 * 4)];

// device address of the scratch array in the current device's context.  Looked up
// on every call (a host-side table lookup): a cached address would go stale when the
// primary context is destroyed and re-created (cudaDeviceReset).
static void *noalloc_scratch_address(std::string &err) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    err = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
    return nullptr;
  }
  return p;
}

int device_potrf_batched_noalloc(int batch, double *base, const int64_t *off, const int32_t *n,
                                 const int32_t *npiv, int32_t *status, cudaStream_t st, std::string &err) {
  if (batch > NOALLOC_MAX) {
    err = "ieti_potrf_batched_noalloc: batch " + std::to_string(batch) + " exceeds IETI_NOALLOC_MAX_BATCH (" +
          std::to_string(NOALLOC_MAX) + ")";
    return IETI_ERR_TOO_LARGE;
  }
  unsigned char *blk = (unsigned char *)noalloc_scratch_address(err);
  if (!blk) return IETI_ERR_CUDA;
  int64_t *doff = (int64_t *)blk;
  int32_t *dn = (int32_t *)(blk + 8 * NOALLOC_MAX);
  int32_t *dkb = dn + NOALLOC_MAX, *dke = dkb + NOALLOC_MAX, *dna = dke + NOALLOC_MAX, *dst = dna + NOALLOC_MAX,
          *dz = dst + NOALLOC_MAX, *dz2 = dz + NOALLOC_MAX, *dbig = dz2 + NOALLOC_MAX;
  // the previous call's contents remain: set every word this call reads
  if (cudaMemcpyAsync(doff, off, batch * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dn, n, batch * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dke, npiv, batch * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dna, n, batch * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(dkb, 0, batch * 4, st) != cudaSuccess || cudaMemsetAsync(dst, 0, batch * 4, st) != cudaSuccess ||
      cudaMemsetAsync(dz, 0, batch * 4, st) != cudaSuccess || cudaMemsetAsync(dz2, 0, batch * 4, st) != cudaSuccess ||
      cudaMemsetAsync(dbig, 0x7f, batch * 4, st) != cudaSuccess) {  // 0x7f7f7f7f: no row limit
    err = std::string("scratch upload failed: ") + cudaGetErrorString(cudaGetLastError());
    return IETI_ERR_CUDA;
  }
  // the same panel loop as ieti_potrf_batched (host copies of the sizes; a
  // DeviceState that owns no device memory carries the stream)
  std::vector<int32_t> hkb(batch, 0), hke(npiv, npiv + batch), hna(n, n + batch);
  DeviceState tmp;
  tmp.stream = st;
  AugLimits lim{dz, dz2, dbig, dz};
  int rc = potrf_partial<double>(&tmp, base, doff, dn, hkb, hke, hna, dkb, dke, dna, dst, lim, err);
  if (rc != IETI_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(status, dst, batch * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    err = std::string("batched partial Cholesky failed: ") + cudaGetErrorString(e);
    return IETI_ERR_CUDA;
  }
  return IETI_OK;
}

}  // namespace ieti
