// C ABI of the solver (declared in include/ieti.h).  Marshals arguments, keeps
// the error text, and never lets an exception cross the boundary.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "device.h"
#include "host_setup.h"
#include "shard.h"

struct ieti_ctx {
  ieti::HostSetup hs;
  ieti::CoarseTree tree;
  ieti_options opt{};
  ieti::DeviceState *dev = nullptr;
  std::string err;
};

static thread_local std::string g_setup_err;

static int check_options(const ieti_options *o, std::string &err) {
  if (!o) { err = "options is NULL"; return IETI_ERR_INVALID_ARG; }
  if (o->precision != IETI_PREC_FP64 && o->precision != IETI_PREC_MIXED) { err = "bad precision"; return IETI_ERR_INVALID_ARG; }
  if (o->precond < IETI_PRECOND_NONE || o->precond > IETI_PRECOND_DIRICHLET_STIFF) { err = "bad precond"; return IETI_ERR_INVALID_ARG; }
  if (!(o->cg_tol > 0.0) || !(o->cg_tol < 1.0)) { err = "cg_tol must be in (0, 1)"; return IETI_ERR_INVALID_ARG; }
  if (o->cg_max_it < 1) { err = "cg_max_it must be >= 1"; return IETI_ERR_INVALID_ARG; }
  if (o->max_sweeps < 1 || o->max_sweeps > 1000) { err = "max_sweeps must be in [1, 1000]"; return IETI_ERR_INVALID_ARG; }
  if (!(o->outer_tol >= 0.0)) { err = "outer_tol must be >= 0"; return IETI_ERR_INVALID_ARG; }
  if (o->device < -1) { err = "device must be >= -1"; return IETI_ERR_INVALID_ARG; }
  if (o->pcg_mode != 0 && o->pcg_mode != 1) { err = "pcg_mode must be 0 or 1"; return IETI_ERR_INVALID_ARG; }
  if (o->l2_persist < 0 || o->l2_persist > 2) { err = "l2_persist must be 0, 1 or 2"; return IETI_ERR_INVALID_ARG; }
  if (o->factor < IETI_FACTOR_FP64 || o->factor > IETI_FACTOR_BF16) { err = "bad factor"; return IETI_ERR_INVALID_ARG; }
  if (o->refactor < IETI_REFACTOR_EVERY || o->refactor > IETI_REFACTOR_NEVER) { err = "bad refactor"; return IETI_ERR_INVALID_ARG; }
  if (!(o->newton_tol >= 0.0)) { err = "newton_tol must be >= 0"; return IETI_ERR_INVALID_ARG; }
  if (o->predictor < 0 || o->predictor > 2) { err = "predictor must be 0, 1 or 2"; return IETI_ERR_INVALID_ARG; }
  if (o->autotune != 0 && o->autotune != 1) { err = "autotune must be 0 or 1"; return IETI_ERR_INVALID_ARG; }
  if (o->graph != 0 && o->graph != 1) { err = "graph must be 0 or 1"; return IETI_ERR_INVALID_ARG; }
  if (o->wait_limit < 0) { err = "wait_limit must be >= 0"; return IETI_ERR_INVALID_ARG; }
  if (o->coarse < IETI_COARSE_AUTO || o->coarse > IETI_COARSE_ND) { err = "bad coarse"; return IETI_ERR_INVALID_ARG; }
  if (o->coarse_leaf < 0) { err = "coarse_leaf must be >= 0"; return IETI_ERR_INVALID_ARG; }
  if (o->coarse_top < 0) { err = "coarse_top must be >= 0"; return IETI_ERR_INVALID_ARG; }
  if (o->deflation != 0 && o->deflation != 1) { err = "deflation must be 0 or 1"; return IETI_ERR_INVALID_ARG; }
  if (o->coarse_ranks < 0 || o->coarse_ranks > 31) { err = "coarse_ranks must be in [0, 31]"; return IETI_ERR_INVALID_ARG; }
  if (o->factor_arena_mb < 0) { err = "factor_arena_mb must be >= 0"; return IETI_ERR_INVALID_ARG; }
  if (o->precision == IETI_PREC_FP64 && o->factor != IETI_FACTOR_FP64) {
    err = "the FP64 precision mode factors in FP64 (factor must be IETI_FACTOR_FP64)";
    return IETI_ERR_INVALID_ARG;
  }
  return IETI_OK;
}

extern "C" {

int ieti_setup(const ieti_problem *problem, const ieti_options *options, ieti_ctx **out) {
  g_setup_err.clear();
  if (!out) { g_setup_err = "out is NULL"; return IETI_ERR_INVALID_ARG; }
  *out = nullptr;
  int rc = check_options(options, g_setup_err);
  if (rc) return rc;
  ieti_ctx *ctx = nullptr;
  try {
    ctx = new ieti_ctx();
    ctx->opt = *options;
    rc = ctx->hs.build(problem, options->host_threads, g_setup_err);
    // nested-dissection tree of the coarse problem: the given leaf size and top merge, or
    // the shape of least modelled solve time over the free ones (~4 TB/s streaming,
    // ~12 us per synchronised level)
    if (rc == IETI_OK) {
      const int leaf = options->coarse_leaf;
      const int top = options->coarse_top > 0 ? options->coarse_top : (leaf > 0 ? 1 : 0);
      ieti::ShardPlan plan;
      const bool aligned = options->coarse_ranks > 1;
      if (aligned) rc = ieti::build_shard_plan(ctx->hs, options->coarse_ranks, plan, g_setup_err);
      if (rc == IETI_OK)
        rc = ieti::choose_coarse_tree(ctx->hs, 4e12, 12e-6, leaf, top, ctx->tree, g_setup_err,
                                      aligned ? &plan.cuts : nullptr);
    }
    if (rc == IETI_OK && options->device >= 0)
      rc = ieti::device_setup(ctx->hs, &ctx->tree, ctx->opt, &ctx->dev, g_setup_err);
  } catch (const std::bad_alloc &) {
    g_setup_err = "host allocation failed";
    rc = IETI_ERR_OOM;
  } catch (const std::exception &e) {
    g_setup_err = std::string("setup failed: ") + e.what();
    rc = IETI_ERR_INVALID_ARG;
  }
  if (rc) {
    delete ctx;
    return rc;
  }
  *out = ctx;
  return IETI_OK;
}

const char *ieti_setup_error(void) { return g_setup_err.c_str(); }

int64_t ieti_num_dofs(const ieti_ctx *ctx) { return ctx ? ctx->hs.n_edges : -1; }

int ieti_get_info(const ieti_ctx *ctx, ieti_info *info) {
  if (!ctx || !info) return IETI_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  const ieti::HostSetup &hs = ctx->hs;
  info->n_dofs = hs.n_edges;
  info->n_free = (int64_t)hs.free_edges.size();
  info->n_lambda = (int64_t)hs.lam.size();
  info->n_coarse = hs.n_coarse;
  for (const auto &pt : hs.patches) {
    info->sum_ni += pt.ni;
    info->sum_nb += pt.nb;
    info->sum_np += pt.np;
    info->max_n = std::max<int64_t>(info->max_n, pt.ni + pt.nb + pt.np);
  }
  info->t_setup_host_ms = hs.t_ms;
  if (ctx->dev) ieti::device_info(ctx->dev, info);
  return IETI_OK;
}

int ieti_load_vector(const ieti_ctx *ctx, const ieti_coil *coil, double *j_out) {
  if (!ctx || !coil || !j_out) return IETI_ERR_INVALID_ARG;
  try {
    ctx->hs.coil_load(*coil, j_out);
  } catch (...) {
    return IETI_ERR_OOM;
  }
  return IETI_OK;
}

int ieti_quad_points(const ieti_ctx *ctx, double *xyz, int64_t *n_points) {
  if (!ctx || !n_points) return IETI_ERR_INVALID_ARG;
  try {
    int64_t n = ctx->hs.quad_point_count();
    if (xyz) {
      if (*n_points < n) return IETI_ERR_INVALID_ARG;
      ctx->hs.quad_points(xyz);
    }
    *n_points = n;
  } catch (...) {
    return IETI_ERR_OOM;
  }
  return IETI_OK;
}

int ieti_load_vector_points(const ieti_ctx *ctx, const double *J_xyz, double *j_out) {
  if (!ctx || !J_xyz || !j_out) return IETI_ERR_INVALID_ARG;
  try {
    ctx->hs.points_load(J_xyz, j_out);
  } catch (...) {
    return IETI_ERR_OOM;
  }
  return IETI_OK;
}

int ieti_dof_classes(const ieti_ctx *ctx, int8_t *cls, int8_t *tree) {
  if (!ctx) return IETI_ERR_INVALID_ARG;
  for (int64_t g = 0; g < ctx->hs.n_edges; ++g) {
    if (cls) cls[g] = ctx->hs.cls[g];
    if (tree) tree[g] = (int8_t)ctx->hs.tree[g];
  }
  return IETI_OK;
}

int ieti_patch_csr(const ieti_ctx *ctx, int32_t patch, int32_t which, int32_t *n_rows, int64_t *nnz, int32_t *ptr,
                   int32_t *col, double *val) {
  if (!ctx || patch < 0 || patch >= ctx->hs.n_patches() || (which != 0 && which != 1)) return IETI_ERR_INVALID_ARG;
  const ieti::Patch &pt = ctx->hs.patches[patch];
  const ieti::Csr &A = which == 0 ? pt.K : pt.M;
  if (n_rows) *n_rows = A.n;
  if (nnz) *nnz = (int64_t)A.col.size();
  if (ptr) std::memcpy(ptr, A.ptr.data(), A.ptr.size() * sizeof(int32_t));
  if (col) std::memcpy(col, A.col.data(), A.col.size() * sizeof(int32_t));
  if (val) std::memcpy(val, A.val.data(), A.val.size() * sizeof(double));
  return IETI_OK;
}

int ieti_step(ieti_ctx *ctx, const double *j_next, int32_t j_mem, ieti_stats *stats) {
  if (!ctx || !j_next) return IETI_ERR_INVALID_ARG;
  if (!ctx->dev) { ctx->err = "host-only context: no device"; return IETI_ERR_NO_DEVICE; }
  try {
    return ieti::device_step(ctx->dev, j_next, j_mem, stats, ctx->err);
  } catch (...) {
    ctx->err = "step failed on the host";
    return IETI_ERR_OOM;
  }
}

int ieti_solution(const ieti_ctx *ctx, double *a_out, int64_t len, int32_t out_mem) {
  if (!ctx || !a_out || len != ctx->hs.n_edges) return IETI_ERR_INVALID_ARG;
  if (!ctx->dev) return IETI_ERR_NO_DEVICE;
  return ieti::device_solution(ctx->dev, a_out, len, out_mem, const_cast<ieti_ctx *>(ctx)->err);
}

int ieti_set_state(ieti_ctx *ctx, const double *a, int64_t len, int32_t a_mem) {
  if (!ctx || !a || len != ctx->hs.n_edges) return IETI_ERR_INVALID_ARG;
  if (!ctx->dev) return IETI_ERR_NO_DEVICE;
  return ieti::device_set_state(ctx->dev, a, len, a_mem, ctx->err);
}

int ieti_kernel_stats(ieti_ctx *ctx, ieti_kernel_stat *out, int32_t reset) {
  if (!ctx || !out) return IETI_ERR_INVALID_ARG;
  if (!ctx->dev) return IETI_ERR_NO_DEVICE;
  ieti::device_kernel_stats(ctx->dev, out, reset != 0);
  return IETI_OK;
}

int ieti_coarse_level_times(ieti_ctx *ctx, double *us, int32_t n, int32_t reset) {
  if (!ctx || (!us && n > 0) || n < 0) return IETI_ERR_INVALID_ARG;
  if (!ctx->dev) return IETI_ERR_NO_DEVICE;
  ieti::device_coarse_level_times(ctx->dev, us, n, reset != 0);
  return IETI_OK;
}

int ieti_pcg_phase_times(ieti_ctx *ctx, double *work_us, double *wait_us, double *sub_us, int32_t reset) {
  if (!ctx || !work_us || !wait_us) return IETI_ERR_INVALID_ARG;
  if (!ctx->dev) return IETI_ERR_NO_DEVICE;
  ieti::device_pcg_trace(ctx->dev, work_us, wait_us, sub_us, reset != 0);
  return IETI_OK;
}

int ieti_potrf_batched(int32_t batch, double *base_dev, const int64_t *offsets, const int32_t *n,
                       const int32_t *n_pivots, int32_t *status_out, void *stream) {
  g_setup_err.clear();
  if (batch < 1 || !base_dev || !offsets || !n || !n_pivots || !status_out) {
    g_setup_err = "ieti_potrf_batched: invalid arguments";
    return IETI_ERR_INVALID_ARG;
  }
  for (int32_t b = 0; b < batch; ++b)
    if (n[b] < 1 || n_pivots[b] < 0 || n_pivots[b] > n[b] || offsets[b] < 0) {
      g_setup_err = "ieti_potrf_batched: bad size, pivot count or offset of matrix " + std::to_string(b);
      return IETI_ERR_INVALID_ARG;
    }
  try {
    return ieti::device_potrf_batched(batch, base_dev, offsets, n, n_pivots, status_out, (cudaStream_t)stream,
                                      g_setup_err);
  } catch (...) {
    g_setup_err = "ieti_potrf_batched: host allocation failed";
    return IETI_ERR_OOM;
  }
}

int ieti_potrf_batched_f32(int32_t batch, float *base_dev, const int64_t *offsets, const int32_t *n,
                           const int32_t *ld, const int32_t *n_pivots, int32_t factor, int32_t *status_out,
                           void *stream) {
  g_setup_err.clear();
  if (batch < 1 || !base_dev || !offsets || !n || !ld || !n_pivots || !status_out ||
      factor < IETI_FACTOR_FP32 || factor > IETI_FACTOR_BF16) {
    g_setup_err = "ieti_potrf_batched_f32: invalid arguments";
    return IETI_ERR_INVALID_ARG;
  }
  const bool tc = factor != IETI_FACTOR_FP32;
  for (int32_t b = 0; b < batch; ++b)
    if (n[b] < 1 || ld[b] < n[b] || n_pivots[b] < 0 || n_pivots[b] > n[b] || offsets[b] < 0 ||
        (tc && (ld[b] % 4 != 0 || offsets[b] % 4 != 0))) {
      g_setup_err = "ieti_potrf_batched_f32: bad size, leading dimension, pivot count or offset of matrix " +
                    std::to_string(b);
      return IETI_ERR_INVALID_ARG;
    }
  try {
    return ieti::device_potrf_batched_f32(batch, base_dev, offsets, n, ld, n_pivots, factor, status_out,
                                          (cudaStream_t)stream, g_setup_err);
  } catch (...) {
    g_setup_err = "ieti_potrf_batched_f32: host allocation failed";
    return IETI_ERR_OOM;
  }
}

// Variant of ieti_potrf_batched that allocates no device memory (static scratch).
int ieti_potrf_batched_noalloc(int32_t batch, double *base_dev, const int64_t *offsets, const int32_t *n,
                               const int32_t *n_pivots, int32_t *status_out, void *stream) {
  g_setup_err.clear();
  if (batch < 1 || !base_dev || !offsets || !n || !n_pivots || !status_out) {
    g_setup_err = "ieti_potrf_batched_noalloc: invalid arguments";
    return IETI_ERR_INVALID_ARG;
  }
  for (int32_t b = 0; b < batch && b <= IETI_NOALLOC_MAX_BATCH; ++b)
    if (n[b] < 1 || n_pivots[b] < 0 || n_pivots[b] > n[b] || offsets[b] < 0) {
      g_setup_err = "ieti_potrf_batched_noalloc: bad size, pivot count or offset of matrix " + std::to_string(b);
      return IETI_ERR_INVALID_ARG;
    }
  try {
    return ieti::device_potrf_batched_noalloc(batch, base_dev, offsets, n, n_pivots, status_out,
                                              (cudaStream_t)stream, g_setup_err);
  } catch (...) {
    g_setup_err = "ieti_potrf_batched_noalloc: host allocation failed";
    return IETI_ERR_OOM;
  }
}

int ieti_coarse_tree(const ieti_ctx *ctx, int32_t *n_nodes, int64_t *n_s, int32_t *elim_pos, int32_t *k0,
                     int32_t *nk, int32_t *parent, int64_t *s_off, int32_t *s_idx) {
  if (!ctx) return IETI_ERR_INVALID_ARG;
  const ieti::CoarseTree &t = ctx->tree;
  if (n_nodes) *n_nodes = t.n_nodes;
  if (n_s) *n_s = (int64_t)t.s_idx.size();
  if (elim_pos)
    for (int64_t g = 0; g < ctx->hs.n_edges; ++g) {
      const int64_t c = ctx->hs.coarse_of_edge[g];
      elim_pos[g] = c < 0 || t.perm.empty() ? -1 : t.perm[c];
    }
  for (int p = 0; p < t.n_nodes; ++p) {
    if (k0) k0[p] = t.k0[p];
    if (nk) nk[p] = t.nk[p];
    if (parent) parent[p] = t.parent[p];
  }
  if (s_off)
    for (int p = 0; p <= t.n_nodes; ++p) s_off[p] = t.n_nodes ? t.s_off[p] : 0;
  if (s_idx) std::copy(t.s_idx.begin(), t.s_idx.end(), s_idx);
  return IETI_OK;
}

int ieti_shard_plan(const ieti_ctx *ctx, int32_t n_ranks, int32_t *rank_of_patch, int32_t *lam_owner,
                    int32_t *lam_peer, int32_t *coarse_owner) {
  if (!ctx) return IETI_ERR_INVALID_ARG;
  try {
    ieti::ShardPlan plan;
    std::string e;
    int rc = ieti::build_shard_plan(ctx->hs, n_ranks, plan, e);
    if (rc) {
      const_cast<ieti_ctx *>(ctx)->err = e;
      return rc;
    }
    if (rank_of_patch) std::copy(plan.rank_of_patch.begin(), plan.rank_of_patch.end(), rank_of_patch);
    if (lam_owner) std::copy(plan.lam_owner.begin(), plan.lam_owner.end(), lam_owner);
    if (lam_peer) std::copy(plan.lam_peer.begin(), plan.lam_peer.end(), lam_peer);
    if (coarse_owner) std::copy(plan.coarse_owner.begin(), plan.coarse_owner.end(), coarse_owner);
  } catch (...) {
    const_cast<ieti_ctx *>(ctx)->err = "ieti_shard_plan: host allocation failed";
    return IETI_ERR_OOM;
  }
  return IETI_OK;
}

int ieti_shard_coarse(const ieti_ctx *ctx, int32_t n_ranks, int32_t *node_rank) {
  if (!ctx || !node_rank) return IETI_ERR_INVALID_ARG;
  try {
    ieti::ShardPlan plan;
    std::vector<int32_t> nr;
    std::string e;
    int rc = ieti::build_shard_plan(ctx->hs, n_ranks, plan, e);
    if (!rc) rc = ieti::shard_coarse_nodes(ctx->hs, ctx->tree, plan, nr, e);
    if (rc) {
      const_cast<ieti_ctx *>(ctx)->err = e;
      return rc;
    }
    std::copy(nr.begin(), nr.end(), node_rank);
  } catch (...) {
    const_cast<ieti_ctx *>(ctx)->err = "ieti_shard_coarse: host allocation failed";
    return IETI_ERR_OOM;
  }
  return IETI_OK;
}

int ieti_multipliers(const ieti_ctx *ctx, int32_t *s, int32_t *pos_s, int32_t *t, int32_t *pos_t) {
  if (!ctx) return IETI_ERR_INVALID_ARG;
  const auto &L = ctx->hs.lam;
  for (size_t l = 0; l < L.size(); ++l) {
    if (s) s[l] = L[l].s;
    if (pos_s) pos_s[l] = L[l].pos_s;
    if (t) t[l] = L[l].t;
    if (pos_t) pos_t[l] = L[l].pos_t;
  }
  return IETI_OK;
}

int ieti_patch_blocks(const ieti_ctx *ctx, int32_t *ni, int32_t *nb, int32_t *np, int32_t *coarse_of_copy) {
  if (!ctx) return IETI_ERR_INVALID_ARG;
  int64_t k = 0;
  for (size_t p = 0; p < ctx->hs.patches.size(); ++p) {
    const ieti::Patch &pt = ctx->hs.patches[p];
    if (ni) ni[p] = pt.ni;
    if (nb) nb[p] = pt.nb;
    if (np) np[p] = pt.np;
    for (int q = pt.ni + pt.nb; q < pt.ni + pt.nb + pt.np; ++q, ++k)
      if (coarse_of_copy) coarse_of_copy[k] = (int32_t)ctx->hs.coarse_of_edge[pt.kept_glob[q]];
  }
  return IETI_OK;
}

const char *ieti_last_error(const ieti_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

void ieti_destroy(ieti_ctx *ctx) {
  if (!ctx) return;
  ieti::device_destroy(ctx->dev);
  delete ctx;
}

}  // extern "C"
