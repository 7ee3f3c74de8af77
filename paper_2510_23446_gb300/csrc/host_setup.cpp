// Host setup: spline edge spaces and patch matrices (Sec. 2.2), the lattice of
// control-mesh edges, the hierarchical tree-cotree gauge and the e/p/r split
// (Sec. 3), multipliers B and the primal map N.  Exact integer / graph work plus
// FP64 quadrature; runs once per problem.
#include "host_setup.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <deque>
#include <functional>
#include <numeric>
#include <thread>

namespace ieti {

// ------------------------------------------------------------------ utilities
static void parallel_for(int n, int threads, const std::function<void(int)> &fn) {
  int T = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  if (T < 1) T = 1;
  T = std::min(T, n);
  if (T <= 1) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int> next{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t)
    pool.emplace_back([&]() {
      for (int i = next++; i < n; i = next++) fn(i);
    });
  for (auto &th : pool) th.join();
}

// Gauss-Legendre rule on [-1,1] by Newton iteration on P_q (three-term recurrence).
static void gauss_legendre(int q, std::vector<double> &x, std::vector<double> &w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    double z = std::cos(pi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= q; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    dp = q * (z * p1 - p0) / (z * z - 1.0);
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// The k+1 B-splines of degree k that are non-zero on the knot span [t[mu], t[mu+1])
// at x (Cox-de Boor triangle), written to out[0..k] for N_{mu-k .. mu, k}.
static void nonzero_basis(const std::vector<double> &t, int mu, int k, double x, double *out) {
  double left[16], right[16];
  out[0] = 1.0;
  for (int j = 1; j <= k; ++j) {
    left[j] = x - t[mu + 1 - j];
    right[j] = t[mu + j] - x;
    double carry = 0.0;
    for (int r = 0; r < j; ++r) {
      double tmp = out[r] / (right[r + 1] + left[j - r]);
      out[r] = carry + right[r + 1] * tmp;
      carry = left[j - r] * tmp;
    }
    out[j] = carry;
  }
}

// Per-direction data at the Gauss points of every element: H^1 values N, their
// derivatives, and the edge functions D_i = p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}.
struct DirData {
  int p = 0, ne = 0, q = 0;
  std::vector<double> w;          // [e][k]
  std::vector<double> N, dN;      // [e][k][a], a = 0..p       (function e + a)
  std::vector<double> D;          // [e][k][a], a = 0..p-1     (edge function e + a)
  double Nv(int e, int k, int a) const { return N[((size_t)e * q + k) * (p + 1) + a]; }
  double dNv(int e, int k, int a) const { return dN[((size_t)e * q + k) * (p + 1) + a]; }
  double Dv(int e, int k, int a) const { return D[((size_t)e * q + k) * p + a]; }
};

static DirData direction_data(const std::vector<double> &t, int p, int ne) {
  DirData dd;
  dd.p = p;
  dd.ne = ne;
  dd.q = p + 2;
  std::vector<double> gx, gw;
  gauss_legendre(dd.q, gx, gw);
  dd.w.resize((size_t)ne * dd.q);
  dd.N.resize((size_t)ne * dd.q * (p + 1));
  dd.dN.resize((size_t)ne * dd.q * (p + 1));
  dd.D.resize((size_t)ne * dd.q * p);
  double bp[16], bm[16];
  for (int e = 0; e < ne; ++e) {
    int mu = p + e;
    double lo = t[mu], hi = t[mu + 1];
    for (int k = 0; k < dd.q; ++k) {
      double x = lo + (hi - lo) * (gx[k] + 1.0) * 0.5;
      dd.w[(size_t)e * dd.q + k] = (hi - lo) * 0.5 * gw[k];
      nonzero_basis(t, mu, p, x, bp);
      nonzero_basis(t, mu, p - 1, x, bm);
      size_t o = ((size_t)e * dd.q + k);
      for (int a = 0; a < p; ++a) {
        int i = e + a;  // edge function index; uses N_{i+1,p-1} = bm[a]
        dd.D[o * p + a] = p / (t[i + p + 1] - t[i + 1]) * bm[a];
      }
      for (int a = 0; a <= p; ++a) {
        dd.N[o * (p + 1) + a] = bp[a];
        double d = 0.0;
        if (a >= 1) d += dd.D[o * p + a - 1];
        if (a < p) d -= dd.D[o * p + a];
        dd.dN[o * (p + 1) + a] = d;  // dN_i/dx = D_{i-1} - D_i
      }
    }
  }
  return dd;
}

// --------------------------------------------------------------- validation
int HostSetup::validate(const ieti_problem *pr, std::string &err) {
  if (!pr) { err = "problem is NULL"; return IETI_ERR_INVALID_ARG; }
  for (int d = 0; d < 3; ++d) {
    if (pr->n_patches[d] < 1 || pr->n_patches[d] > 4096) {
      err = "n_patches must be in [1, 4096]";
      return IETI_ERR_INVALID_ARG;
    }
    if (!pr->n_el[d] || !pr->degree[d] || !pr->knots[d]) {
      err = "n_el/degree/knots pointer is NULL";
      return IETI_ERR_INVALID_ARG;
    }
  }
  if (!pr->ctrl_pts || !pr->sigma_el || !pr->nu_el) { err = "ctrl/sigma/nu pointer is NULL"; return IETI_ERR_INVALID_ARG; }
  if (!(pr->dt > 0.0) || !std::isfinite(pr->dt)) { err = "dt must be positive"; return IETI_ERR_INVALID_ARG; }
  if (pr->primal_mode != 0) { err = "primal_mode must be 0"; return IETI_ERR_INVALID_ARG; }
  for (int d = 0; d < 3; ++d) {
    P[d] = pr->n_patches[d];
    n_el[d].assign(pr->n_el[d], pr->n_el[d] + P[d]);
    degree[d].assign(pr->degree[d], pr->degree[d] + P[d]);
    knots[d].assign(P[d], {});
    size_t off = 0;
    for (int a = 0; a < P[d]; ++a) {
      int ne = n_el[d][a], p = degree[d][a];
      if (ne < 1 || ne > 512 || p < 1 || p > 8) {
        err = "n_el must be in [1,512] and degree in [1,8]";
        return IETI_ERR_INVALID_ARG;
      }
      size_t m = (size_t)ne + 2 * p + 1;
      std::vector<double> t(pr->knots[d] + off, pr->knots[d] + off + m);
      off += m;
      for (int i = 0; i <= p; ++i)
        if (t[i] != 0.0 || t[m - 1 - i] != 1.0) {
          err = "knot vectors must be open on [0,1] (p+1 repeated end knots)";
          return IETI_ERR_INVALID_ARG;
        }
      for (size_t i = p; i + p + 1 < m; ++i)
        if (!(t[i + 1] > t[i]) || !std::isfinite(t[i + 1])) {
          err = "interior knots must be simple and increasing";
          return IETI_ERR_INVALID_ARG;
        }
      knots[d][a] = t;
    }
  }
  int np = n_patches();
  ctrl_off.assign(np + 1, 0);
  el_off.assign(np + 1, 0);
  for (int s = 0; s < np; ++s) {
    int a = s % P[0], b = (s / P[0]) % P[1], c = s / (P[0] * P[1]);
    int idx[3] = {a, b, c};
    int64_t nc = 3, ne = 1;
    for (int d = 0; d < 3; ++d) {
      nc *= n_el[d][idx[d]] + degree[d][idx[d]];
      ne *= n_el[d][idx[d]];
    }
    ctrl_off[s + 1] = ctrl_off[s] + nc;
    el_off[s + 1] = el_off[s] + ne;
  }
  ctrl.assign(pr->ctrl_pts, pr->ctrl_pts + ctrl_off[np]);
  sigma_el.assign(pr->sigma_el, pr->sigma_el + el_off[np]);
  nu_el.assign(pr->nu_el, pr->nu_el + el_off[np]);
  for (double x : ctrl)
    if (!std::isfinite(x)) { err = "non-finite control point"; return IETI_ERR_INVALID_ARG; }
  for (size_t i = 0; i < sigma_el.size(); ++i)
    if (!(sigma_el[i] >= 0.0) || !std::isfinite(sigma_el[i]) || !(nu_el[i] > 0.0) || !std::isfinite(nu_el[i])) {
      err = "sigma must be >= 0 and nu > 0 (finite) on every element";
      return IETI_ERR_INVALID_ARG;
    }
  dt = pr->dt;
  nonlinear = pr->reluctivity != nullptr;
  if (nonlinear) {
    for (int k = 0; k < 4; ++k) law[k] = pr->reluctivity[k];
    bool ok = law[0] > 0.0 && law[1] >= 0.0 && law[2] >= 0.0 && law[3] >= 0.0 && law[1] + law[3] > 0.0;
    for (int k = 0; k < 4; ++k) ok = ok && std::isfinite(law[k]);
    if (!ok) {
      err = "reluctivity law needs nu0 > 0, k1, k2, k3 >= 0 and k1 + k3 > 0";
      return IETI_ERR_INVALID_ARG;
    }
  }
  return IETI_OK;
}

// ------------------------------------------------------------------ lattice
int64_t HostSetup::edge_id(int d, int64_t I, int64_t J, int64_t K) const {
  if (d == 0) return edge_off[0] + I + (N[0] - 1) * (J + N[1] * K);
  if (d == 1) return edge_off[1] + I + N[0] * (J + (N[1] - 1) * K);
  return edge_off[2] + I + N[0] * (J + N[1] * K);
}

void HostSetup::edge_coords(int64_t g, int &d, int64_t &I, int64_t &J, int64_t &K) const {
  if (g < edge_off[1]) {
    d = 0;
    int64_t l = g;
    I = l % (N[0] - 1);
    l /= (N[0] - 1);
    J = l % N[1];
    K = l / N[1];
  } else if (g < edge_off[2]) {
    d = 1;
    int64_t l = g - edge_off[1];
    I = l % N[0];
    l /= N[0];
    J = l % (N[1] - 1);
    K = l / (N[1] - 1);
  } else {
    d = 2;
    int64_t l = g - edge_off[2];
    I = l % N[0];
    l /= N[0];
    J = l % N[1];
    K = l / N[1];
  }
}

bool HostSetup::boundary_node(int64_t n) const {
  int64_t I = n % N[0], J = (n / N[0]) % N[1], K = n / (N[0] * N[1]);
  return I == 0 || I == N[0] - 1 || J == 0 || J == N[1] - 1 || K == 0 || K == N[2] - 1;
}

int HostSetup::slab_start(int d, int64_t I) const {
  // largest slab a with off[d][a] <= I
  auto it = std::upper_bound(off[d].begin(), off[d].end(), I);
  return (int)(it - off[d].begin()) - 1;
}

void HostSetup::lattice() {
  for (int d = 0; d < 3; ++d) {
    off[d].assign(P[d], 0);
    for (int a = 1; a < P[d]; ++a) off[d][a] = off[d][a - 1] + n_el[d][a - 1] + degree[d][a - 1] - 1;
    N[d] = off[d][P[d] - 1] + n_el[d][P[d] - 1] + degree[d][P[d] - 1];
    is_sb[d].assign(N[d], 0);
    for (int a = 0; a < P[d]; ++a) is_sb[d][off[d][a]] = 1;
    is_sb[d][N[d] - 1] = 1;
  }
  E[0] = (N[0] - 1) * N[1] * N[2];
  E[1] = N[0] * (N[1] - 1) * N[2];
  E[2] = N[0] * N[1] * (N[2] - 1);
  edge_off[0] = 0;
  edge_off[1] = E[0];
  edge_off[2] = E[0] + E[1];
  n_edges = E[0] + E[1] + E[2];
  n_nodes = N[0] * N[1] * N[2];
  dirichlet.assign(n_edges, 0);
  kind.assign(n_edges, 0);
  n_share.assign(n_edges, 1);
  for (int64_t g = 0; g < n_edges; ++g) {
    int d;
    int64_t c[3];
    edge_coords(g, d, c[0], c[1], c[2]);
    int nsb = 0, nint = 0;
    bool bnd = false;
    for (int e = 0; e < 3; ++e) {
      if (e == d) continue;
      bool atb = c[e] == 0 || c[e] == N[e] - 1;
      bool atsb = is_sb[e][c[e]] != 0;
      bnd |= atb;
      nsb += atsb;
      nint += (atsb && !atb);
    }
    dirichlet[g] = bnd;
    kind[g] = (uint8_t)nsb;
    n_share[g] = (uint8_t)(1 << nint);
  }
  int np = n_patches();
  patches.assign(np, Patch{});
  for (int s = 0; s < np; ++s) {
    Patch &pt = patches[s];
    pt.a = s % P[0];
    pt.b = (s / P[0]) % P[1];
    pt.c = s / (P[0] * P[1]);
    int idx[3] = {pt.a, pt.b, pt.c};
    for (int d = 0; d < 3; ++d) {
      pt.p[d] = degree[d][idx[d]];
      pt.ne[d] = n_el[d][idx[d]];
      pt.n[d] = pt.ne[d] + pt.p[d];
    }
    pt.n_dofs = 0;
    for (int comp = 0; comp < 3; ++comp) {
      int m[3] = {pt.n[0], pt.n[1], pt.n[2]};
      m[comp] -= 1;
      for (int k = 0; k < m[2]; ++k)
        for (int j = 0; j < m[1]; ++j)
          for (int i = 0; i < m[0]; ++i)
            pt.l2g.push_back(edge_id(comp, off[0][pt.a] + i, off[1][pt.b] + j, off[2][pt.c] + k));
    }
    pt.n_dofs = (int)pt.l2g.size();
  }
}

// ---------------------------------------------------------------- assembly
// Support of a local edge DOF in element indices per direction (clipped).
static inline void dof_support(const Patch &pt, int comp, int i, int j, int k, int lo[3], int hi[3]) {
  int idx[3] = {i, j, k};
  for (int d = 0; d < 3; ++d) {
    int l = (d == comp) ? idx[d] + 1 - pt.p[d] : idx[d] - pt.p[d];
    int h = idx[d];
    lo[d] = std::max(l, 0);
    hi[d] = std::min(h, pt.ne[d] - 1);
  }
}

static inline void local_dims(const Patch &pt, int comp, int m[3]) {
  m[0] = pt.n[0]; m[1] = pt.n[1]; m[2] = pt.n[2];
  m[comp] -= 1;
}

static inline int comp_offset(const Patch &pt, int comp) {
  int n0 = pt.n[0], n1 = pt.n[1], n2 = pt.n[2];
  if (comp == 0) return 0;
  if (comp == 1) return (n0 - 1) * n1 * n2;
  return (n0 - 1) * n1 * n2 + n0 * (n1 - 1) * n2;
}

static void csr_pattern(const Patch &pt, Csr &A) {
  A.n = pt.n_dofs;
  A.ptr.assign(A.n + 1, 0);
  A.col.clear();
  int row = 0;
  for (int comp = 0; comp < 3; ++comp) {
    int m[3];
    local_dims(pt, comp, m);
    for (int k = 0; k < m[2]; ++k)
      for (int j = 0; j < m[1]; ++j)
        for (int i = 0; i < m[0]; ++i, ++row) {
          int lo[3], hi[3];
          dof_support(pt, comp, i, j, k, lo, hi);
          for (int c2 = 0; c2 < 3; ++c2) {
            int m2[3];
            local_dims(pt, c2, m2);
            int base = comp_offset(pt, c2);
            int idx0[3] = {i, j, k};
            int rlo[3], rhi[3];
            for (int d = 0; d < 3; ++d) {
              rlo[d] = std::max(0, idx0[d] - pt.p[d] - 1);
              rhi[d] = std::min(m2[d] - 1, idx0[d] + pt.p[d] + 1);
            }
            for (int kk = rlo[2]; kk <= rhi[2]; ++kk)
              for (int jj = rlo[1]; jj <= rhi[1]; ++jj)
                for (int ii = rlo[0]; ii <= rhi[0]; ++ii) {
                  int lo2[3], hi2[3];
                  dof_support(pt, c2, ii, jj, kk, lo2, hi2);
                  bool ov = true;
                  for (int d = 0; d < 3; ++d) ov &= (lo2[d] <= hi[d] && lo[d] <= hi2[d]);
                  if (ov) A.col.push_back(base + ii + m2[0] * (jj + m2[1] * kk));
                }
          }
          A.ptr[row + 1] = (int32_t)A.col.size();
        }
  }
  A.val.assign(A.col.size(), 0.0);
}

static inline int csr_find(const Csr &A, int r, int c) {
  const int32_t *b = A.col.data() + A.ptr[r];
  const int32_t *e = A.col.data() + A.ptr[r + 1];
  const int32_t *it = std::lower_bound(b, e, c);
  return (int)(it - A.col.data());
}

struct ElemBasis {
  // reference values w_hat and curls c_hat of the active functions at one point
  int nloc = 0;
  std::vector<int> lid;          // local DOF ids of the active functions
};

// Geometry of one point (GEOM visits): DF and DF^{-1}
struct PointRef {
  const double (*J)[3];
  const double (*inv)[3];
};

// Visit every quadrature point of every element of a patch with the geometry
// (x = F(xi), DF, det DF, weight) and the physical quantities of all active
// functions: U_a = DF c_hat_a (= det * curl w_a) and V_a = DF^{-T} w_hat_a (= w_a).
// GEOM: the callback gets the point's PointRef instead of the functions' values (none
// are formed).
template <bool GEOM = false, class Fn>
static void for_each_point(const HostSetup &hs, const Patch &pt, int s, const DirData dd[3], Fn &&fn) {
  const double *net = hs.ctrl.data() + hs.ctrl_off[s];
  int n0 = pt.n[0], n1 = pt.n[1];
  int p0 = pt.p[0], p1 = pt.p[1], p2 = pt.p[2];
  int nl0 = p0 * (p1 + 1) * (p2 + 1), nl1 = (p0 + 1) * p1 * (p2 + 1), nl2 = (p0 + 1) * (p1 + 1) * p2;
  int nloc = nl0 + nl1 + nl2;
  std::vector<int> lid(nloc);
  std::vector<double> wh(nloc * 3), ch(nloc * 3), U(nloc * 3), V(nloc * 3);
  for (int ez = 0; ez < pt.ne[2]; ++ez)
    for (int ey = 0; ey < pt.ne[1]; ++ey)
      for (int ex = 0; ex < pt.ne[0]; ++ex) {
        int el = ex + pt.ne[0] * (ey + pt.ne[1] * ez);
        // active function ids
        int t = 0;
        for (int comp = 0; comp < 3; ++comp) {
          int m[3];
          local_dims(pt, comp, m);
          int base = comp_offset(pt, comp);
          int na = (comp == 0) ? p0 : p0 + 1, nb = (comp == 1) ? p1 : p1 + 1, nc = (comp == 2) ? p2 : p2 + 1;
          for (int c = 0; c < nc; ++c)
            for (int b = 0; b < nb; ++b)
              for (int a = 0; a < na; ++a) lid[t++] = base + (ex + a) + m[0] * ((ey + b) + m[1] * (ez + c));
        }
        for (int kz = 0; kz < dd[2].q; ++kz)
          for (int ky = 0; ky < dd[1].q; ++ky)
            for (int kx = 0; kx < dd[0].q; ++kx) {
              double w = dd[0].w[(size_t)ex * dd[0].q + kx] * dd[1].w[(size_t)ey * dd[1].q + ky] *
                         dd[2].w[(size_t)ez * dd[2].q + kz];
              double F[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
              for (int c = 0; c <= p2; ++c)
                for (int b = 0; b <= p1; ++b)
                  for (int a = 0; a <= p0; ++a) {
                    const double *cp = net + 3 * ((size_t)(ex + a) + n0 * ((size_t)(ey + b) + n1 * (size_t)(ez + c)));
                    double Nx = dd[0].Nv(ex, kx, a), Ny = dd[1].Nv(ey, ky, b), Nz = dd[2].Nv(ez, kz, c);
                    double gx = dd[0].dNv(ex, kx, a) * Ny * Nz, gy = Nx * dd[1].dNv(ey, ky, b) * Nz,
                           gz = Nx * Ny * dd[2].dNv(ez, kz, c);
                    double nn = Nx * Ny * Nz;
                    for (int r = 0; r < 3; ++r) {
                      F[r] += cp[r] * nn;
                      J[r][0] += cp[r] * gx;
                      J[r][1] += cp[r] * gy;
                      J[r][2] += cp[r] * gz;
                    }
                  }
              double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
              // inverse (adjugate / det); DF^{-T} = (adj^T)/det
              double inv[3][3];
              inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
              inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
              inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
              inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
              inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
              inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
              inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
              inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
              inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
              // reference values and curls of the active functions
              t = 0;
              for (int comp = 0; comp < 3 && !GEOM; ++comp) {
                int na = (comp == 0) ? p0 : p0 + 1, nb = (comp == 1) ? p1 : p1 + 1, nc = (comp == 2) ? p2 : p2 + 1;
                for (int c = 0; c < nc; ++c)
                  for (int b = 0; b < nb; ++b)
                    for (int a = 0; a < na; ++a, ++t) {
                      double *wv = &wh[3 * t], *cv = &ch[3 * t];
                      if (comp == 0) {
                        double Dx = dd[0].Dv(ex, kx, a), Ny = dd[1].Nv(ey, ky, b), Nz = dd[2].Nv(ez, kz, c);
                        double dNy = dd[1].dNv(ey, ky, b), dNz = dd[2].dNv(ez, kz, c);
                        wv[0] = Dx * Ny * Nz; wv[1] = 0; wv[2] = 0;
                        cv[0] = 0; cv[1] = Dx * Ny * dNz; cv[2] = -Dx * dNy * Nz;
                      } else if (comp == 1) {
                        double Nx = dd[0].Nv(ex, kx, a), Dy = dd[1].Dv(ey, ky, b), Nz = dd[2].Nv(ez, kz, c);
                        double dNx = dd[0].dNv(ex, kx, a), dNz = dd[2].dNv(ez, kz, c);
                        wv[0] = 0; wv[1] = Nx * Dy * Nz; wv[2] = 0;
                        cv[0] = -Nx * Dy * dNz; cv[1] = 0; cv[2] = dNx * Dy * Nz;
                      } else {
                        double Nx = dd[0].Nv(ex, kx, a), Ny = dd[1].Nv(ey, ky, b), Dz = dd[2].Dv(ez, kz, c);
                        double dNx = dd[0].dNv(ex, kx, a), dNy = dd[1].dNv(ey, ky, b);
                        wv[0] = 0; wv[1] = 0; wv[2] = Nx * Ny * Dz;
                        cv[0] = Nx * dNy * Dz; cv[1] = -dNx * Ny * Dz; cv[2] = 0;
                      }
                      for (int r = 0; r < 3; ++r) {
                        U[3 * t + r] = J[r][0] * cv[0] + J[r][1] * cv[1] + J[r][2] * cv[2];
                        // (DF^{-T} w)_r = sum_j inv[j][r] w_j
                        V[3 * t + r] = inv[0][r] * wv[0] + inv[1][r] * wv[1] + inv[2][r] * wv[2];
                      }
                    }
              }
              if constexpr (GEOM) {
                const PointRef pr{J, inv};
                fn(el, nloc, lid.data(), F, det, w, pr);
              } else {
                fn(el, nloc, lid.data(), F, det, w, U.data(), V.data());
              }
            }
      }
}

// Element matrices by sum factorisation.  Every reference curl component and every
// reference value of an edge function is a product of 1-D factors (N, N' or D per
// direction), so a block sum over the element's points
//   E[a][b] += sign * sum_q X_a(qx) Y_a(qy) Z_a(qz) W(q) X_b(qx) Y_b(qy) Z_b(qz)
// is formed by contracting z, then y, then x (tensor-product quadrature).
struct Factor1D {
  const double *t[3];  // per direction: [function][point] values
  int n[3];            // functions per direction
};

static void sf_block(const Factor1D &A, const Factor1D &B, const int q[3], const double *W, double sign, int n,
                     int ra, int rb, double *E, std::vector<double> &t1, std::vector<double> &t2) {
  const int qx = q[0], qy = q[1], qz = q[2];
  const int az = A.n[2], bz = B.n[2], ay = A.n[1], by = B.n[1], ax = A.n[0], bx = B.n[0];
  // t1[(kx * qy + ky) * az * bz + cz * bz + cz'] = sum_kz Za[cz](kz) Zb[cz'](kz) W(kx, ky, kz)
  t1.assign((size_t)qx * qy * az * bz, 0.0);
  for (int kz = 0; kz < qz; ++kz)
    for (int ky = 0; ky < qy; ++ky)
      for (int kx = 0; kx < qx; ++kx) {
        const double w = W[kx + qx * (ky + qy * kz)];
        double *o = &t1[(size_t)(kx * qy + ky) * az * bz];
        for (int cz = 0; cz < az; ++cz) {
          const double zw = A.t[2][cz * qz + kz] * w;
          for (int dz = 0; dz < bz; ++dz) o[cz * bz + dz] += zw * B.t[2][dz * qz + kz];
        }
      }
  // t2[((kx * ay + cy) * by + dy) * az * bz + zz] = sum_ky Ya[cy](ky) Yb[dy](ky) t1[kx][ky][zz]
  const int zz = az * bz;
  t2.assign((size_t)qx * ay * by * zz, 0.0);
  for (int kx = 0; kx < qx; ++kx)
    for (int ky = 0; ky < qy; ++ky) {
      const double *src = &t1[(size_t)(kx * qy + ky) * zz];
      for (int cy = 0; cy < ay; ++cy) {
        const double ya = A.t[1][cy * qy + ky];
        for (int dy = 0; dy < by; ++dy) {
          const double yy = ya * B.t[1][dy * qy + ky];
          double *o = &t2[((size_t)(kx * ay + cy) * by + dy) * zz];
          for (int u = 0; u < zz; ++u) o[u] += yy * src[u];
        }
      }
    }
  // E[ra + (cx + ax (cy + ay cz))][rb + (dx + bx (dy + by dz))] += sign sum_kx Xa Xb t2
  for (int kx = 0; kx < qx; ++kx)
    for (int cx = 0; cx < ax; ++cx) {
      const double xa = sign * A.t[0][cx * qx + kx];
      for (int dx = 0; dx < bx; ++dx) {
        const double xx = xa * B.t[0][dx * qx + kx];
        for (int cy = 0; cy < ay; ++cy)
          for (int dy = 0; dy < by; ++dy) {
            const double *src = &t2[((size_t)(kx * ay + cy) * by + dy) * zz];
            for (int cz = 0; cz < az; ++cz) {
              double *row = E + (size_t)(ra + cx + ax * (cy + ay * cz)) * n + rb + dx;
              for (int dz = 0; dz < bz; ++dz) row[(size_t)bx * (dy + by * dz)] += xx * src[cz * bz + dz];
            }
          }
      }
    }
}

void HostSetup::assemble_patch(Patch &pt) const {
  int s = pt.a + P[0] * (pt.b + P[1] * pt.c);
  DirData dd[3];
  for (int d = 0; d < 3; ++d) {
    int slab = d == 0 ? pt.a : (d == 1 ? pt.b : pt.c);
    dd[d] = direction_data(knots[d][slab], pt.p[d], pt.ne[d]);
  }
  csr_pattern(pt, pt.K);
  pt.M = pt.K;
  const double *sig = sigma_el.data() + el_off[s];
  const double *nu = nu_el.data() + el_off[s];
  // K_e = sum over the element's points of (nu w / det) (DF c_hat_a) . (DF c_hat_b)
  //     = sum of c_hat_a^T G c_hat_b,  G = (nu w / det) DF^T DF, and
  // M_e = sum of (sigma w det) w_a . w_b = sum of w_hat_a^T H w_hat_b,
  //       H = (sigma w det) DF^{-1} DF^{-T}:
  // by sum factorisation over the 1-D factors of the reference curls and values
  const int q[3] = {dd[0].q, dd[1].q, dd[2].q};
  const int Q = q[0] * q[1] * q[2];
  const int p0 = pt.p[0], p1 = pt.p[1], p2 = pt.p[2];
  const int nl0 = p0 * (p1 + 1) * (p2 + 1), nl1 = (p0 + 1) * p1 * (p2 + 1), nl2 = (p0 + 1) * (p1 + 1) * p2;
  const int n = nl0 + nl1 + nl2;
  const int bs[3] = {0, nl0, nl0 + nl1};  // element-local function blocks by component
  // element-local function index of the first function of every (component, c, b)
  // group and the group's length (the a-run), in the order the element lists them
  std::vector<std::pair<int, int>> groups;
  {
    int t = 0;
    for (int comp = 0; comp < 3; ++comp) {
      const int na = (comp == 0) ? p0 : p0 + 1, nb = (comp == 1) ? p1 : p1 + 1, nc = (comp == 2) ? p2 : p2 + 1;
      for (int c = 0; c < nc; ++c)
        for (int b = 0; b < nb; ++b) {
          groups.push_back({t, na});
          t += na;
        }
    }
  }
  // 1-D tables of the current element, [function][point]: N, N' (p + 1 functions) and D
  // (p functions) per direction
  std::vector<double> tN[3], tdN[3], tD[3];
  for (int d = 0; d < 3; ++d) {
    tN[d].resize((size_t)(pt.p[d] + 1) * q[d]);
    tdN[d].resize((size_t)(pt.p[d] + 1) * q[d]);
    tD[d].resize((size_t)pt.p[d] * q[d]);
  }
  // factors of the reference curl component r of component c's functions, with signs:
  // c = 0: (D, N, N') r = 1, -(D, N', N) r = 2; c = 1: -(N, D, N') r = 0, (N', D, N) r = 2;
  // c = 2: (N, N', D) r = 0, -(N', N, D) r = 1.  Values of component c: D along c, N else.
  enum { TN = 0, TDN = 1, TD = 2 };
  static const int curl_tab[3][2][4] = {{{1, TD, TN, TDN}, {2, TD, TDN, TN}},
                                        {{0, TN, TD, TDN}, {2, TDN, TD, TN}},
                                        {{0, TN, TDN, TD}, {1, TDN, TN, TD}}};
  static const double curl_sign[3][2] = {{1.0, -1.0}, {-1.0, 1.0}, {1.0, -1.0}};
  auto table = [&](int d, int type) -> const double * {
    return type == TN ? tN[d].data() : (type == TDN ? tdN[d].data() : tD[d].data());
  };
  auto count = [&](int d, int type) { return type == TD ? pt.p[d] : pt.p[d] + 1; };
  auto factor = [&](int tx, int ty, int tz) {
    Factor1D f;
    const int ty3[3] = {tx, ty, tz};
    for (int d = 0; d < 3; ++d) {
      f.t[d] = table(d, ty3[d]);
      f.n[d] = count(d, ty3[d]);
    }
    return f;
  };
  std::vector<double> Gq((size_t)9 * Q), Hq((size_t)9 * Q), Ke, Me, t1, t2;
  std::vector<int> cur_lid;
  int cur_el = -1, qi = 0;
  bool any_m = false;
  auto flush = [&]() {
    if (cur_el < 0) return;
    const int e3[3] = {cur_el % pt.ne[0], (cur_el / pt.ne[0]) % pt.ne[1], cur_el / (pt.ne[0] * pt.ne[1])};
    for (int d = 0; d < 3; ++d)
      for (int k = 0; k < q[d]; ++k) {
        for (int a = 0; a <= pt.p[d]; ++a) {
          tN[d][(size_t)a * q[d] + k] = dd[d].Nv(e3[d], k, a);
          tdN[d][(size_t)a * q[d] + k] = dd[d].dNv(e3[d], k, a);
        }
        for (int a = 0; a < pt.p[d]; ++a) tD[d][(size_t)a * q[d] + k] = dd[d].Dv(e3[d], k, a);
      }
    Ke.assign((size_t)n * n, 0.0);
    for (int ca = 0; ca < 3; ++ca)
      for (int i = 0; i < 2; ++i) {
        const int *fa = curl_tab[ca][i];
        const Factor1D A = factor(fa[1], fa[2], fa[3]);
        for (int cb = 0; cb < 3; ++cb)
          for (int j = 0; j < 2; ++j) {
            const int *fb = curl_tab[cb][j];
            sf_block(A, factor(fb[1], fb[2], fb[3]), q, &Gq[(size_t)(fa[0] * 3 + fb[0]) * Q],
                     curl_sign[ca][i] * curl_sign[cb][j], n, bs[ca], bs[cb], Ke.data(), t1, t2);
          }
      }
    if (any_m) {
      Me.assign((size_t)n * n, 0.0);
      for (int ca = 0; ca < 3; ++ca)
        for (int cb = 0; cb < 3; ++cb)
          sf_block(factor(ca == 0 ? TD : TN, ca == 1 ? TD : TN, ca == 2 ? TD : TN),
                   factor(cb == 0 ? TD : TN, cb == 1 ? TD : TN, cb == 2 ? TD : TN), q,
                   &Hq[(size_t)(ca * 3 + cb) * Q], 1.0, n, bs[ca], bs[cb], Me.data(), t1, t2);
    }
    // the element's columns of one (component, c, b) group are consecutive DOF ids
    // whose CSR entries are consecutive in every row (a row's columns of one
    // component form a box of lattice indices): one search per row and group
    for (int a = 0; a < n; ++a)
      for (const auto &g : groups) {
        const int pos = csr_find(pt.K, cur_lid[a], cur_lid[g.first]);
        const double *kr = &Ke[(size_t)a * n + g.first];
        double *kv = &pt.K.val[pos];
        for (int u = 0; u < g.second; ++u) kv[u] += kr[u];
        if (any_m) {
          const double *mr = &Me[(size_t)a * n + g.first];
          double *mv = &pt.M.val[pos];
          for (int u = 0; u < g.second; ++u) mv[u] += mr[u];
        }
      }
  };
  for_each_point<true>(*this, pt, s, dd, [&](int el, int nloc, const int *lid, const double *, double det,
                                             double w, const PointRef &pr) {
    if (el != cur_el) {
      flush();
      cur_el = el;
      cur_lid.assign(lid, lid + nloc);
      qi = 0;
      any_m = false;
    }
    // the nonlinear law's stiffness is assembled on the device at every Newton iterate
    const double ck = nl_element(s, el) ? 0.0 : nu[el] * w / det;
    const double cm = sig[el] * w * det;
    if (cm != 0.0) any_m = true;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        Gq[(size_t)(r * 3 + c) * Q + qi] =
            ck * (pr.J[0][r] * pr.J[0][c] + pr.J[1][r] * pr.J[1][c] + pr.J[2][r] * pr.J[2][c]);
        Hq[(size_t)(r * 3 + c) * Q + qi] =
            cm * (pr.inv[r][0] * pr.inv[c][0] + pr.inv[r][1] * pr.inv[c][1] + pr.inv[r][2] * pr.inv[c][2]);
      }
    ++qi;
  });
  flush();
}

void HostSetup::assemble_all() {
  parallel_for(n_patches(), threads, [&](int s) { assemble_patch(patches[s]); });
}

void HostSetup::coil_load(const ieti_coil &coil, double *out) const {
  int np = n_patches();
  std::vector<std::vector<double>> loc(np);
  parallel_for(np, threads, [&](int s) {
    const Patch &pt = patches[s];
    DirData dd[3];
    for (int d = 0; d < 3; ++d) {
      int slab = d == 0 ? pt.a : (d == 1 ? pt.b : pt.c);
      dd[d] = direction_data(knots[d][slab], pt.p[d], pt.ne[d]);
    }
    loc[s].assign(pt.n_dofs, 0.0);
    for_each_point(*this, pt, s, dd, [&](int, int nloc, const int *lid, const double *F, double, double w,
                                         const double *U, const double *) {
      double r = std::sqrt((F[0] - coil.xc) * (F[0] - coil.xc) + (F[1] - coil.yc) * (F[1] - coil.yc));
      double Tz = 0.0;
      if (r <= coil.r_in) Tz = coil.J0 * (coil.r_out - coil.r_in);
      else if (r < coil.r_out) Tz = coil.J0 * (coil.r_out - r);
      if (!(std::fabs(F[2] - coil.zc) < coil.hz)) Tz = 0.0;
      if (Tz == 0.0) return;
      for (int a = 0; a < nloc; ++a) loc[s][lid[a]] += w * Tz * U[3 * a + 2];
    });
  });
  std::fill(out, out + n_edges, 0.0);
  for (int s = 0; s < np; ++s)
    for (int l = 0; l < patches[s].n_dofs; ++l) out[patches[s].l2g[l]] += loc[s][l];
}

// Quadrature points of the assembly: per patch its elements (x fastest) and per
// element its (p_d + 2)^3 Gauss points (x fastest), the order of for_each_point.
int64_t HostSetup::quad_point_count(std::vector<int64_t> *patch_off) const {
  int np = n_patches();
  if (patch_off) patch_off->assign(np + 1, 0);
  int64_t n = 0;
  for (int s = 0; s < np; ++s) {
    const Patch &pt = patches[s];
    n += (int64_t)pt.ne[0] * pt.ne[1] * pt.ne[2] * (pt.p[0] + 2) * (pt.p[1] + 2) * (pt.p[2] + 2);
    if (patch_off) (*patch_off)[s + 1] = n;
  }
  return n;
}

void HostSetup::quad_points(double *xyz) const {
  std::vector<int64_t> off;
  quad_point_count(&off);
  parallel_for(n_patches(), threads, [&](int s) {
    const Patch &pt = patches[s];
    DirData dd[3];
    for (int d = 0; d < 3; ++d) {
      int slab = d == 0 ? pt.a : (d == 1 ? pt.b : pt.c);
      dd[d] = direction_data(knots[d][slab], pt.p[d], pt.ne[d]);
    }
    int64_t k = off[s];
    for_each_point(*this, pt, s, dd, [&](int, int, const int *, const double *F, double, double, const double *,
                                         const double *) {
      xyz[3 * k] = F[0];
      xyz[3 * k + 1] = F[1];
      xyz[3 * k + 2] = F[2];
      ++k;
    });
  });
}

// j_k = <J, w_k> = sum over points of weight * det DF * J(x_q) . w_k(x_q)
void HostSetup::points_load(const double *J, double *out) const {
  std::vector<int64_t> off;
  quad_point_count(&off);
  int np = n_patches();
  std::vector<std::vector<double>> loc(np);
  parallel_for(np, threads, [&](int s) {
    const Patch &pt = patches[s];
    DirData dd[3];
    for (int d = 0; d < 3; ++d) {
      int slab = d == 0 ? pt.a : (d == 1 ? pt.b : pt.c);
      dd[d] = direction_data(knots[d][slab], pt.p[d], pt.ne[d]);
    }
    loc[s].assign(pt.n_dofs, 0.0);
    int64_t k = off[s];
    for_each_point(*this, pt, s, dd, [&](int, int nloc, const int *lid, const double *, double det, double w,
                                         const double *, const double *V) {
      const double *Jq = J + 3 * k;
      ++k;
      double c = w * det;
      if (Jq[0] == 0.0 && Jq[1] == 0.0 && Jq[2] == 0.0) return;
      for (int a = 0; a < nloc; ++a)
        loc[s][lid[a]] += c * (Jq[0] * V[3 * a] + Jq[1] * V[3 * a + 1] + Jq[2] * V[3 * a + 2]);
    });
  });
  std::fill(out, out + n_edges, 0.0);
  for (int s = 0; s < np; ++s)
    for (int l = 0; l < patches[s].n_dofs; ++l) out[patches[s].l2g[l]] += loc[s][l];
}

// ----------------------------------------------------------------- regions
// any(mask) over inclusive element boxes, via a 3-D prefix sum
struct Prefix3 {
  int n0, n1, n2;
  std::vector<int> S;
  Prefix3(const std::vector<uint8_t> &m, int e0, int e1, int e2) : n0(e0), n1(e1), n2(e2) {
    S.assign((size_t)(n0 + 1) * (n1 + 1) * (n2 + 1), 0);
    for (int k = 0; k < n2; ++k)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n0; ++i)
          at(i + 1, j + 1, k + 1) = m[i + n0 * (j + n1 * k)] + at(i, j + 1, k + 1) + at(i + 1, j, k + 1) +
                                    at(i + 1, j + 1, k) - at(i, j, k + 1) - at(i, j + 1, k) - at(i + 1, j, k) +
                                    at(i, j, k);
  }
  int &at(int i, int j, int k) { return S[i + (size_t)(n0 + 1) * (j + (size_t)(n1 + 1) * k)]; }
  int sum(const int lo[3], const int hi[3]) {
    int i0 = lo[0], j0 = lo[1], k0 = lo[2], i1 = hi[0] + 1, j1 = hi[1] + 1, k1 = hi[2] + 1;
    return at(i1, j1, k1) - at(i0, j1, k1) - at(i1, j0, k1) - at(i1, j1, k0) + at(i0, j0, k1) + at(i0, j1, k0) +
           at(i1, j0, k0) - at(i0, j0, k0);
  }
};

void HostSetup::regions() {
  touch_c.assign(n_edges, 0);
  touch_i.assign(n_edges, 0);
  cnode.assign(n_nodes, 0);
  for (int s = 0; s < n_patches(); ++s) {
    const Patch &pt = patches[s];
    int ne = pt.ne[0] * pt.ne[1] * pt.ne[2];
    std::vector<uint8_t> mc(ne), mi(ne);
    for (int e = 0; e < ne; ++e) {
      mc[e] = sigma_el[el_off[s] + e] > 0.0;
      mi[e] = !mc[e];
    }
    Prefix3 Pc(mc, pt.ne[0], pt.ne[1], pt.ne[2]), Pi(mi, pt.ne[0], pt.ne[1], pt.ne[2]);
    int l = 0;
    for (int comp = 0; comp < 3; ++comp) {
      int m[3];
      local_dims(pt, comp, m);
      for (int k = 0; k < m[2]; ++k)
        for (int j = 0; j < m[1]; ++j)
          for (int i = 0; i < m[0]; ++i, ++l) {
            int lo[3], hi[3];
            dof_support(pt, comp, i, j, k, lo, hi);
            int64_t g = pt.l2g[l];
            if (Pc.sum(lo, hi) > 0) touch_c[g] = 1;
            if (Pi.sum(lo, hi) > 0) touch_i[g] = 1;
          }
    }
    for (int k = 0; k < pt.n[2]; ++k)
      for (int j = 0; j < pt.n[1]; ++j)
        for (int i = 0; i < pt.n[0]; ++i) {
          int idx[3] = {i, j, k}, lo[3], hi[3];
          for (int d = 0; d < 3; ++d) {
            lo[d] = std::max(idx[d] - pt.p[d], 0);
            hi[d] = std::min(idx[d], pt.ne[d] - 1);
          }
          if (Pc.sum(lo, hi) > 0) cnode[node_id(off[0][pt.a] + i, off[1][pt.b] + j, off[2][pt.c] + k)] = 1;
        }
  }
}

// -------------------------------------------------------------------- tree
void HostSetup::bfs_pass(const std::vector<int64_t> &edges, std::vector<uint8_t> &visited,
                         const std::vector<int64_t> &u, const std::vector<int64_t> &v) {
  if (edges.empty()) return;
  const int64_t ROOT = n_nodes;
  auto key = [&](int64_t x) { return x == ROOT ? (int64_t)-1 : x; };
  std::vector<int64_t> nodes;
  nodes.reserve(2 * edges.size());
  for (int64_t e : edges) {
    nodes.push_back(key(u[e]));
    nodes.push_back(key(v[e]));
  }
  std::sort(nodes.begin(), nodes.end());
  nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
  auto index = [&](int64_t x) {
    return (int64_t)(std::lower_bound(nodes.begin(), nodes.end(), key(x)) - nodes.begin());
  };
  size_t nn = nodes.size();
  std::vector<int64_t> deg(nn + 1, 0);
  for (int64_t e : edges) {
    deg[index(u[e]) + 1]++;
    deg[index(v[e]) + 1]++;
  }
  for (size_t i = 0; i < nn; ++i) deg[i + 1] += deg[i];
  std::vector<int64_t> fill(deg.begin(), deg.end() - 1), adj_e(deg[nn]), adj_o(deg[nn]);
  for (int64_t e : edges) {  // ascending edge ids -> per-node lists ascending
    int64_t a = index(u[e]), b = index(v[e]);
    adj_e[fill[a]] = e; adj_o[fill[a]++] = b;
    adj_e[fill[b]] = e; adj_o[fill[b]++] = a;
  }
  auto gid = [&](int64_t i) { return nodes[i] < 0 ? ROOT : nodes[i]; };
  std::deque<int64_t> q;
  auto run = [&]() {
    while (!q.empty()) {
      int64_t x = q.front();
      q.pop_front();
      for (int64_t t = deg[x]; t < deg[x + 1]; ++t) {
        int64_t y = adj_o[t];
        if (!visited[gid(y)]) {
          visited[gid(y)] = 1;
          tree[adj_e[t]] = 1;
          q.push_back(y);
        }
      }
    }
  };
  for (size_t i = 0; i < nn; ++i)
    if (visited[gid(i)]) q.push_back((int64_t)i);
  run();
  for (size_t i = 0; i < nn; ++i)
    if (!visited[gid(i)]) {
      visited[gid(i)] = 1;
      q.push_back((int64_t)i);
      run();
    }
}

void HostSetup::build_tree() {
  const int64_t ROOT = n_nodes;
  std::vector<int64_t> u(n_edges), v(n_edges);
  in_graph.assign(n_edges, 0);
  gtype.assign(n_edges, 0);
  tree.assign(n_edges, 0);
  for (int64_t g = 0; g < n_edges; ++g) {
    int d;
    int64_t I, J, K;
    edge_coords(g, d, I, J, K);
    int64_t n0 = node_id(I, J, K);
    int64_t n1 = node_id(I + (d == 0), J + (d == 1), K + (d == 2));
    u[g] = boundary_node(n0) ? ROOT : n0;
    v[g] = boundary_node(n1) ? ROOT : n1;
    in_graph[g] = touch_i[g] && !dirichlet[g];
    gtype[g] = in_graph[g] && cnode[n0] && cnode[n1];
  }
  std::vector<uint8_t> visited(n_nodes + 1, 0);
  visited[ROOT] = 1;
  auto two_pass = [&](const std::vector<int64_t> &edges) {
    std::vector<int64_t> a, b;
    for (int64_t e : edges) (gtype[e] ? a : b).push_back(e);
    bfs_pass(a, visited, u, v);
    bfs_pass(b, visited, u, v);
  };
  // stage 1: wirebasket
  std::vector<int64_t> st;
  for (int64_t g = 0; g < n_edges; ++g)
    if (in_graph[g] && kind[g] == 2) st.push_back(g);
  two_pass(st);
  // stage 2: faces in ascending face id
  int64_t foff[3] = {0, (int64_t)(P[0] + 1) * P[1] * P[2],
                     (int64_t)(P[0] + 1) * P[1] * P[2] + (int64_t)P[0] * (P[1] + 1) * P[2]};
  std::vector<std::pair<int64_t, int64_t>> keyed;
  for (int64_t g = 0; g < n_edges; ++g) {
    if (!in_graph[g] || kind[g] != 1) continue;
    int d;
    int64_t c[3];
    edge_coords(g, d, c[0], c[1], c[2]);
    int f = -1;
    for (int e = 0; e < 3; ++e)
      if (e != d && is_sb[e][c[e]]) f = e;
    // plane index: position of c[f] among the slab planes
    int64_t gpos = (c[f] == N[f] - 1) ? P[f] : slab_start(f, c[f]);
    int in1 = (f == 0) ? 1 : 0, in2 = (f == 2) ? 1 : 2;
    int t1 = slab_start(in1, c[in1]), t2 = slab_start(in2, c[in2]);
    int64_t fid = foff[f] + gpos + (int64_t)(P[f] + 1) * (t1 + (int64_t)P[in1] * t2);
    keyed.push_back({fid, g});
  }
  std::sort(keyed.begin(), keyed.end());
  for (size_t i = 0; i < keyed.size();) {
    size_t j = i;
    std::vector<int64_t> grp;
    while (j < keyed.size() && keyed[j].first == keyed[i].first) grp.push_back(keyed[j++].second);
    two_pass(grp);
    i = j;
  }
  // stage 3: patch interiors in ascending patch id
  keyed.clear();
  for (int64_t g = 0; g < n_edges; ++g) {
    if (!in_graph[g] || kind[g] != 0) continue;
    int d;
    int64_t c[3];
    edge_coords(g, d, c[0], c[1], c[2]);
    int64_t s = slab_start(0, c[0]) + (int64_t)P[0] * (slab_start(1, c[1]) + (int64_t)P[1] * slab_start(2, c[2]));
    keyed.push_back({s, g});
  }
  std::sort(keyed.begin(), keyed.end());
  for (size_t i = 0; i < keyed.size();) {
    size_t j = i;
    std::vector<int64_t> grp;
    while (j < keyed.size() && keyed[j].first == keyed[i].first) grp.push_back(keyed[j++].second);
    two_pass(grp);
    i = j;
  }
  // stage 4: Kruskal, Gamma-type edges first
  std::vector<int64_t> parent(n_nodes + 1);
  std::iota(parent.begin(), parent.end(), 0);
  std::function<int64_t(int64_t)> find = [&](int64_t x) {
    int64_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) { int64_t n = parent[x]; parent[x] = r; x = n; }
    return r;
  };
  for (int64_t g = 0; g < n_edges; ++g)
    if (tree[g]) parent[find(u[g])] = find(v[g]);
  for (int pass = 0; pass < 2; ++pass)
    for (int64_t g = 0; g < n_edges; ++g) {
      if (!in_graph[g] || tree[g] || (pass == 0 && !gtype[g])) continue;
      int64_t a = find(u[g]), b = find(v[g]);
      if (a != b) {
        tree[g] = 1;
        parent[a] = b;
      }
    }
}

void HostSetup::classify() {
  cls.assign(n_edges, CLS_R);
  for (int64_t g = 0; g < n_edges; ++g) {
    bool shared = n_share[g] >= 2;
    if (dirichlet[g]) { cls[g] = CLS_E; continue; }
    if (tree[g] && touch_i[g]) {
      if (!gtype[g]) cls[g] = CLS_E;
      else if (shared) cls[g] = CLS_P;
    } else if (in_graph[g] && !tree[g] && kind[g] == 2 && shared) {
      cls[g] = CLS_P;
    }
  }
}

// -------------------------------------------------------------- decomposition
static void restrict_reorder(const Csr &A, const std::vector<int32_t> &perm /* local -> kept or -1 */,
                             const std::vector<int32_t> &order /* kept -> local */, const Csr *B, double beta,
                             Csr &out) {
  // out = (A + beta*B) restricted to kept rows/cols, kept order; B has A's pattern
  int nk = (int)order.size();
  out.n = nk;
  out.ptr.assign(nk + 1, 0);
  out.col.clear();
  out.val.clear();
  std::vector<std::pair<int32_t, double>> row;
  for (int r = 0; r < nk; ++r) {
    int lr = order[r];
    row.clear();
    for (int t = A.ptr[lr]; t < A.ptr[lr + 1]; ++t) {
      int c = perm[A.col[t]];
      if (c < 0) continue;
      double x = A.val[t] + (B ? beta * B->val[t] : 0.0);
      row.push_back({c, x});
    }
    std::sort(row.begin(), row.end());
    for (auto &e : row) {
      out.col.push_back(e.first);
      out.val.push_back(e.second);
    }
    out.ptr[r + 1] = (int32_t)out.col.size();
  }
}

void HostSetup::decompose() {
  int np = n_patches();
  std::vector<std::tuple<int64_t, int32_t, int32_t>> copies;
  coarse_of_edge.assign(n_edges, -1);
  n_coarse = 0;
  free_edges.clear();
  for (int64_t g = 0; g < n_edges; ++g) {
    if (cls[g] == CLS_P) coarse_of_edge[g] = n_coarse++;
    if (cls[g] != CLS_E) free_edges.push_back(g);
  }
  parallel_for(np, threads, [&](int s) {
    Patch &pt = patches[s];
    pt.i_loc.clear(); pt.b_loc.clear(); pt.p_loc.clear();
    for (int l = 0; l < pt.n_dofs; ++l) {
      int64_t g = pt.l2g[l];
      if (cls[g] == CLS_R && n_share[g] < 2) pt.i_loc.push_back(l);
      else if (cls[g] == CLS_R) pt.b_loc.push_back(l);
      else if (cls[g] == CLS_P) pt.p_loc.push_back(l);
    }
    pt.ni = (int)pt.i_loc.size();
    pt.nb = (int)pt.b_loc.size();
    pt.np = (int)pt.p_loc.size();
    std::vector<int32_t> order;
    order.insert(order.end(), pt.i_loc.begin(), pt.i_loc.end());
    order.insert(order.end(), pt.b_loc.begin(), pt.b_loc.end());
    order.insert(order.end(), pt.p_loc.begin(), pt.p_loc.end());
    std::vector<int32_t> perm(pt.n_dofs, -1);
    for (size_t k = 0; k < order.size(); ++k) perm[order[k]] = (int32_t)k;
    pt.loc2kept = perm;
    restrict_reorder(pt.M, perm, order, &pt.K, dt, pt.Wk);
    restrict_reorder(pt.M, perm, order, nullptr, 0.0, pt.Mk);
    pt.kept_glob.resize(order.size());
    pt.load_w.resize(order.size());
    for (size_t k = 0; k < order.size(); ++k) {
      pt.kept_glob[k] = pt.l2g[order[k]];
      pt.load_w[k] = 1.0 / n_share[pt.kept_glob[k]];
    }
  });
  for (int s = 0; s < np; ++s) {
    const Patch &pt = patches[s];
    for (int k = 0; k < pt.nb; ++k) copies.emplace_back(pt.l2g[pt.b_loc[k]], s, k);
  }
  std::sort(copies.begin(), copies.end());
  lam.clear();
  for (size_t i = 0; i < copies.size();) {
    size_t j = i;
    while (j < copies.size() && std::get<0>(copies[j]) == std::get<0>(copies[i])) ++j;
    for (size_t x = i; x < j; ++x)
      for (size_t y = x + 1; y < j; ++y)
        lam.push_back({std::get<0>(copies[x]), std::get<1>(copies[x]), std::get<2>(copies[x]),
                       std::get<1>(copies[y]), std::get<2>(copies[y])});
    i = j;
  }
}

// -------------------------------------------------------------------- build
void HostSetup::nl_tables() {
  nl = NlTables();
  for (int s = 0; s < n_patches(); ++s) {
    const Patch &pt = patches[s];
    int ne = pt.ne[0] * pt.ne[1] * pt.ne[2];
    for (int e = 0; e < ne; ++e)
      if (nl_element(s, e)) {
        nl.patches.push_back(s);
        break;
      }
  }
  // per patch tables in parallel, then concatenated in patch order
  const int nb = (int)nl.patches.size();
  std::vector<NlTables> part(nb);
  parallel_for(nb, threads, [&](int b) {
    const int s = nl.patches[b];
    const Patch &pt = patches[s];
    DirData dd[3];
    for (int d = 0; d < 3; ++d) {
      int slab = d == 0 ? pt.a : (d == 1 ? pt.b : pt.c);
      dd[d] = direction_data(knots[d][slab], pt.p[d], pt.ne[d]);
    }
    NlTables &t = part[b];
    int cur = -1;
    for_each_point(*this, pt, s, dd, [&](int el, int nloc, const int *lid, const double *, double det, double w,
                                         const double *U, const double *) {
      if (!nl_element(s, el)) return;
      if (el != cur) {
        cur = el;
        t.el_batch.push_back(b);
        t.nloc.push_back(nloc);
        t.nq.push_back(0);
        t.g_off.push_back((int64_t)t.G.size());
        t.q_off.push_back((int64_t)t.cq.size());
        t.d_off.push_back((int64_t)t.kept.size());
        for (int a = 0; a < nloc; ++a) {
          t.kept.push_back(pt.loc2kept[lid[a]]);
          t.glob.push_back(pt.l2g[lid[a]]);
        }
      }
      t.nq.back()++;
      double g = std::sqrt(w / det);
      for (int a = 0; a < 3 * nloc; ++a) t.G.push_back(U[a] * g);
      t.cq.push_back(1.0 / std::sqrt(w * det));
    });
  });
  for (int b = 0; b < nb; ++b) {
    NlTables &t = part[b];
    int64_t go = (int64_t)nl.G.size(), qo = (int64_t)nl.cq.size(), dof = (int64_t)nl.kept.size();
    for (size_t e = 0; e < t.nloc.size(); ++e) {
      nl.el_batch.push_back(t.el_batch[e]);
      nl.nloc.push_back(t.nloc[e]);
      nl.nq.push_back(t.nq[e]);
      nl.g_off.push_back(go + t.g_off[e]);
      nl.q_off.push_back(qo + t.q_off[e]);
      nl.d_off.push_back(dof + t.d_off[e]);
    }
    nl.G.insert(nl.G.end(), t.G.begin(), t.G.end());
    nl.cq.insert(nl.cq.end(), t.cq.begin(), t.cq.end());
    nl.kept.insert(nl.kept.end(), t.kept.begin(), t.kept.end());
    nl.glob.insert(nl.glob.end(), t.glob.begin(), t.glob.end());
  }
}

int HostSetup::build(const ieti_problem *pr, int nthreads, std::string &err) {
  auto t0 = std::chrono::steady_clock::now();
  threads = nthreads;
  int rc = validate(pr, err);
  if (rc) return rc;
  lattice();
  assemble_all();
  regions();
  build_tree();
  classify();
  decompose();
  if (nonlinear) nl_tables();
  t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return IETI_OK;
}

}  // namespace ieti
