// Patch-sharded layout for several ranks (see shard.h).
#include "shard.h"

#include <algorithm>
#include <cmath>
#include <functional>

namespace ieti {

int build_shard_plan(const HostSetup &hs, int n_ranks, ShardPlan &plan, std::string &err) {
  if (n_ranks < 1 || n_ranks > 31) {
    err = "n_ranks must be in [1, 31]";
    return IETI_ERR_INVALID_ARG;
  }
  const int np_ = hs.n_patches();
  if (n_ranks > np_) {
    err = "more ranks than patches";
    return IETI_ERR_INVALID_ARG;
  }
  plan = ShardPlan();
  plan.n_ranks = n_ranks;
  plan.rank_of_patch.assign(np_, -1);
  plan.rank_weight.assign(n_ranks, 0.0);
  // the work of a patch per PCG iteration grows with its local size
  std::vector<double> w(np_);
  for (int s = 0; s < np_; ++s) {
    const Patch &pt = hs.patches[s];
    w[s] = (double)(pt.ni + pt.nb + pt.np);
  }
  auto pid = [&](int a, int b, int c) { return a + hs.P[0] * (b + hs.P[1] * c); };
  // recursive coordinate bisection: the box's longest side is cut at the slab boundary
  // whose left part's weight best matches the left ranks' share
  std::function<void(const int *, int, int)> split = [&](const int *box, int r0, int r1) {
    if (r1 - r0 == 1) {
      for (int c = box[4]; c < box[5]; ++c)
        for (int b = box[2]; b < box[3]; ++b)
          for (int a = box[0]; a < box[1]; ++a) {
            plan.rank_of_patch[pid(a, b, c)] = r0;
            plan.rank_weight[r0] += w[pid(a, b, c)];
          }
      return;
    }
    const int ext[3] = {box[1] - box[0], box[3] - box[2], box[5] - box[4]};
    int d = 0;
    for (int e = 1; e < 3; ++e)
      if (ext[e] > ext[d]) d = e;
    const int nl = (r1 - r0) / 2;
    const double share = (double)nl / (double)(r1 - r0);
    std::vector<double> slab(ext[d], 0.0);
    double total = 0;
    for (int c = box[4]; c < box[5]; ++c)
      for (int b = box[2]; b < box[3]; ++b)
        for (int a = box[0]; a < box[1]; ++a) {
          const int idx[3] = {a, b, c};
          slab[idx[d] - box[2 * d]] += w[pid(a, b, c)];
          total += w[pid(a, b, c)];
        }
    int best = 1;
    double acc = 0, best_gap = 1e300;
    for (int m = 1; m < ext[d]; ++m) {
      acc += slab[m - 1];
      const double gap = std::fabs(acc / total - share);
      if (gap < best_gap) {
        best_gap = gap;
        best = m;
      }
    }
    int bl[6], br[6];
    std::copy(box, box + 6, bl);
    std::copy(box, box + 6, br);
    bl[2 * d + 1] = box[2 * d] + best;
    br[2 * d] = box[2 * d] + best;
    BoxCut bc;
    std::copy(box, box + 6, bc.box);
    bc.d = d;
    bc.m = box[2 * d] + best;
    plan.cuts.push_back(bc);
    split(bl, r0, r0 + nl);
    split(br, r0 + nl, r1);
  };
  const int root[6] = {0, hs.P[0], 0, hs.P[1], 0, hs.P[2]};
  split(root, 0, n_ranks);
  for (int s = 0; s < np_; ++s)
    if (plan.rank_of_patch[s] < 0) {
      err = "shard plan left a patch without a rank";
      return IETI_ERR_INVALID_ARG;
    }
  for (int r = 0; r < n_ranks; ++r)
    if (plan.rank_weight[r] == 0.0) {
      err = "shard plan left a rank without patches (more ranks than the grid can be cut into)";
      return IETI_ERR_INVALID_ARG;
    }
  const int64_t m = (int64_t)hs.lam.size();
  plan.lam_owner.resize(m);
  plan.lam_peer.resize(m);
  for (int64_t l = 0; l < m; ++l) {
    const int rs = plan.rank_of_patch[hs.lam[l].s], rt = plan.rank_of_patch[hs.lam[l].t];
    plan.lam_owner[l] = rs;
    plan.lam_peer[l] = rt != rs ? rt : -1;
  }
  plan.coarse_owner.assign(hs.n_coarse, INT32_MAX);
  plan.coarse_ranks.assign(hs.n_coarse, 0);
  for (int s = 0; s < np_; ++s) {
    const Patch &pt = hs.patches[s];
    const int r = plan.rank_of_patch[s];
    for (int k = pt.ni + pt.nb; k < pt.ni + pt.nb + pt.np; ++k) {
      const int64_t c = hs.coarse_of_edge[pt.kept_glob[k]];
      plan.coarse_owner[c] = std::min(plan.coarse_owner[c], r);
      plan.coarse_ranks[c] |= 1 << r;
    }
  }
  return IETI_OK;
}

int shard_coarse_nodes(const HostSetup &hs, const CoarseTree &t, const ShardPlan &plan,
                       std::vector<int32_t> &node_rank, std::string &err) {
  node_rank.assign(t.n_nodes, -1);
  auto pid = [&](int a, int b, int c) { return a + hs.P[0] * (b + hs.P[1] * c); };
  for (int p = 0; p < t.n_nodes; ++p) {
    const int *bx = t.box.data() + 6 * (size_t)p;
    int r = -2;  // -2: no patch seen yet
    for (int c = bx[4]; c < bx[5] && r != -1; ++c)
      for (int b = bx[2]; b < bx[3] && r != -1; ++b)
        for (int a = bx[0]; a < bx[1]; ++a) {
          const int q = plan.rank_of_patch[pid(a, b, c)];
          if (r == -2) r = q;
          else if (q != r) {
            r = -1;
            break;
          }
        }
    node_rank[p] = r < 0 ? -1 : r;
  }
  // the subtree property the exchange relies on
  for (int p = 0; p < t.n_nodes; ++p)
    if (t.parent[p] >= 0 && node_rank[t.parent[p]] >= 0 && node_rank[t.parent[p]] != node_rank[p]) {
      err = "shard_coarse_nodes: a node's parent is owned by another rank";
      return IETI_ERR_INVALID_ARG;
    }
  return IETI_OK;
}

}  // namespace ieti
