// Nonlinear reluctivity nu(|B|) = nu0 (k1 exp(k2 |B|^2) + k3) in the conducting
// elements (the nonlinear material the paper names as an extension, Sec. 2):
// device evaluation of the Newton residual and of the tangent stiffness from the
// quadrature tables of the host setup (NlTables): at point q of element e,
// B_q = cq[q] sum_a x_a G[q][a],
// residual  N_a = sum_q nu(|B_q|^2) (B_q . G[q][a]) / cq[q]                 (FP64),
// tangent   K_t[a][b] = sum_q nu G[q][a].G[q][b] + 2 nu' (B_q.G[q][a])(B_q.G[q][b]) (FP32 accumulation).
#pragma once
#include <cstdint>

namespace ieti {

struct NlLaw {
  double nu0, k1, k2, k3;
};

__device__ __forceinline__ double warp_sum_nl(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA per nonlinear element.  mode bit 0: r[kept] -= dt N_a (the Newton residual
// of the assembled system); bit 1: tq[q] = (nu, sqrt(2 nu') B_q) for k_nl_tangent.
// Dynamic shared memory: (max nloc + 4 max nq) doubles.
__global__ void k_nl_eval(const double *G, const double *cq, const int32_t *kept, const int64_t *glob,
                          const int64_t *goff, const int64_t *qoff, const int64_t *doff, const int32_t *nloc,
                          const int32_t *nq, const int32_t *bpos, const int64_t *kofs_b, const double *a, NlLaw law,
                          double dt, double *r, float4 *tq, int mode) {
  extern __shared__ double nl_sm[];
  const int e = blockIdx.x;
  const int n = nloc[e], Q = nq[e];
  const double *Ge = G + goff[e];
  const double *ce = cq + qoff[e];
  const int32_t *ke = kept + doff[e];
  const int64_t *ge = glob + doff[e];
  double *al = nl_sm;          // coefficients of the element's functions
  double *Bq = al + n;         // B at the points (3 per point)
  double *nuq = Bq + 3 * Q;    // nu at the points
  for (int i = threadIdx.x; i < n; i += blockDim.x) al[i] = a[ge[i]];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = warp; q < Q; q += nw) {
    double b0 = 0, b1 = 0, b2 = 0;
    for (int i = lane; i < n; i += 32) {
      const double *g = Ge + ((int64_t)q * n + i) * 3;
      const double x = al[i];
      b0 += x * g[0];
      b1 += x * g[1];
      b2 += x * g[2];
    }
    b0 = warp_sum_nl(b0);
    b1 = warp_sum_nl(b1);
    b2 = warp_sum_nl(b2);
    if (lane == 0) {
      const double c = ce[q];
      b0 *= c;
      b1 *= c;
      b2 *= c;
      const double s = b0 * b0 + b1 * b1 + b2 * b2;
      const double E = exp(law.k2 * s);
      const double nu = law.nu0 * (law.k1 * E + law.k3);
      const double dnu = law.nu0 * law.k1 * law.k2 * E;
      Bq[3 * q] = b0;
      Bq[3 * q + 1] = b1;
      Bq[3 * q + 2] = b2;
      nuq[q] = nu;
      if (mode & 2) {
        const double f = sqrt(2.0 * dnu);
        tq[qoff[e] + q] = make_float4((float)nu, (float)(f * b0), (float)(f * b1), (float)(f * b2));
      }
    }
  }
  if (!(mode & 1)) return;
  __syncthreads();
  const int64_t kb = kofs_b[bpos[e]];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int k = ke[i];
    if (k < 0) continue;
    double acc = 0;
    for (int q = 0; q < Q; ++q) {
      const double *g = Ge + ((int64_t)q * n + i) * 3;
      acc += nuq[q] * (Bq[3 * q] * g[0] + Bq[3 * q + 1] * g[1] + Bq[3 * q + 2] * g[2]) / ce[q];
    }
    atomicAdd(&r[kb + k], -dt * acc);
  }
}

constexpr int NL_TB = 256;   // threads of k_nl_tangent
constexpr int NL_EPT = 16;   // lower-triangle entries per thread and pass
constexpr int NL_QC = 8;     // points staged per round

// dt K_t of every nonlinear element added to the lower triangle of its patch's
// dense augmented block (kept numbering = the first rows of the block).  One CTA per
// element; the n(n+1)/2 entries in passes of NL_TB * NL_EPT; the factors
// F[q][a] = (sqrt(nu) G[q][a], beta_q . G[q][a]) of NL_QC points at a time in
// shared memory.  Dynamic shared memory: NL_QC * max nloc float4.
template <class TD>
__global__ void __launch_bounds__(NL_TB) k_nl_tangent(const double *G, const int32_t *kept, const int64_t *goff,
                                                      const int64_t *qoff, const int64_t *doff,
                                                      const int32_t *nloc, const int32_t *nq, const int32_t *bpos,
                                                      const float4 *tq, const int64_t *Doff, const int32_t *ld,
                                                      double dt, TD *D) {
  extern __shared__ float4 nl_F[];
  const int e = blockIdx.x;
  const int n = nloc[e], Q = nq[e];
  const double *Ge = G + goff[e];
  const float4 *te = tq + qoff[e];
  const int32_t *ke = kept + doff[e];
  const int b_ = bpos[e];
  TD *Dp = D + Doff[b_];
  const int64_t ldp = ld[b_];
  const int P = n * (n + 1) / 2;
  for (int p0 = 0; p0 < P; p0 += NL_TB * NL_EPT) {
    int ea[NL_EPT], eb[NL_EPT];
    float acc[NL_EPT];
#pragma unroll
    for (int j = 0; j < NL_EPT; ++j) {
      const int t = p0 + threadIdx.x + j * NL_TB;
      int ra = 0, rb = -1;
      if (t < P) {
        ra = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while ((ra + 1) * (ra + 2) / 2 <= t) ++ra;
        while (ra * (ra + 1) / 2 > t) --ra;
        rb = t - ra * (ra + 1) / 2;
      }
      ea[j] = ra;
      eb[j] = rb;
      acc[j] = 0.f;
    }
    for (int q0 = 0; q0 < Q; q0 += NL_QC) {
      const int qc = min(NL_QC, Q - q0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < qc * n; idx += NL_TB) {
        const int qq = idx / n, i = idx % n;
        const double *g = Ge + ((int64_t)(q0 + qq) * n + i) * 3;
        const float4 t4 = te[q0 + qq];
        const float sn = sqrtf(t4.x);
        const float g0 = (float)g[0], g1 = (float)g[1], g2 = (float)g[2];
        nl_F[qq * n + i] = make_float4(sn * g0, sn * g1, sn * g2, t4.y * g0 + t4.z * g1 + t4.w * g2);
      }
      __syncthreads();
      for (int qq = 0; qq < qc; ++qq) {
        const float4 *Fq = nl_F + qq * n;
#pragma unroll
        for (int j = 0; j < NL_EPT; ++j) {
          if (eb[j] < 0) continue;
          const float4 u = Fq[ea[j]], v = Fq[eb[j]];
          acc[j] += u.x * v.x + u.y * v.y + u.z * v.z + u.w * v.w;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NL_EPT; ++j) {
      if (eb[j] < 0) continue;
      const int ka = ke[ea[j]], kb = ke[eb[j]];
      if (ka < 0 || kb < 0) continue;
      const int rr = max(ka, kb), cc = min(ka, kb);
      atomicAdd(&Dp[(int64_t)rr * ldp + cc], (TD)(dt * (double)acc[j]));
    }
  }
}

}  // namespace ieti
