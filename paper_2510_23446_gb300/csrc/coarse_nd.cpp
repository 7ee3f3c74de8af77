// Nested-dissection tree of the primal coarse problem (see coarse_nd.h).
#include "coarse_nd.h"

#include <algorithm>
#include <functional>

namespace ieti {

namespace {

struct RawNode {
  int box[6];
  std::vector<int32_t> dofs;   // coarse ids, ascending
  int parent = -1, depth = 0;
  std::vector<int> kids;
};

}  // namespace

int CoarseTree::front_index(int p, int32_t x) const {
  if (x >= k0[p] && x < k0[p] + nk[p]) return x - k0[p];
  const int32_t *b = s_idx.data() + s_off[p], *e = s_idx.data() + s_off[p + 1];
  const int32_t *it = std::lower_bound(b, e, x);
  if (it == e || *it != x) return -1;
  return nk[p] + (int)(it - b);
}

int build_coarse_tree(const HostSetup &hs, int leaf_max, int top, CoarseTree &t, std::string &err,
                      const std::vector<BoxCut> *cuts) {
  t = CoarseTree();
  t.nc = hs.n_coarse;
  t.leaf_max = std::max(1, leaf_max);
  t.top = std::max(0, top);
  const int64_t nc = hs.n_coarse;
  if (nc == 0) return IETI_OK;
  if (nc >= (int64_t)INT32_MAX) {
    err = "coarse problem too large for the nested-dissection solver";
    return IETI_ERR_TOO_LARGE;
  }
  // patch index range of every coarse unknown: the patches holding a copy of it
  std::vector<int32_t> lo(3 * nc, INT32_MAX), hi(3 * nc, -1);
  for (const Patch &pt : hs.patches) {
    const int idx[3] = {pt.a, pt.b, pt.c};
    for (int k = pt.ni + pt.nb; k < pt.ni + pt.nb + pt.np; ++k) {
      const int64_t c = hs.coarse_of_edge[pt.kept_glob[k]];
      for (int e = 0; e < 3; ++e) {
        lo[3 * c + e] = std::min(lo[3 * c + e], idx[e]);
        hi[3 * c + e] = std::max(hi[3 * c + e], idx[e]);
      }
    }
  }
  for (int64_t c = 0; c < nc; ++c)
    if (hi[3 * c] < 0) {
      err = "a coarse unknown has no patch copy";
      return IETI_ERR_INVALID_ARG;
    }
  // recursive bisection of the patch grid
  std::vector<RawNode> raw;
  std::function<int(const int *, int, std::vector<int32_t> &&)> rec = [&](const int *box, int parent,
                                                                          std::vector<int32_t> &&alive) -> int {
    const int k = (int)raw.size();
    raw.emplace_back();
    std::copy(box, box + 6, raw[k].box);
    raw[k].parent = parent;
    raw[k].depth = parent < 0 ? 0 : raw[parent].depth + 1;
    int ext[3] = {box[1] - box[0], box[3] - box[2], box[5] - box[4]};
    if ((int64_t)ext[0] * ext[1] * ext[2] <= t.leaf_max) {
      raw[k].dofs = std::move(alive);
      return k;
    }
    int d = 0;
    for (int e = 1; e < 3; ++e)
      if (ext[e] > ext[d]) d = e;
    int m = box[2 * d] + ext[d] / 2;
    if (cuts)
      for (const BoxCut &bc : *cuts)
        if (std::equal(box, box + 6, bc.box)) {
          d = bc.d;
          m = bc.m;
          break;
        }
    std::vector<int32_t> mine, left, right;
    for (int32_t c : alive) {
      if (lo[3 * c + d] < m && hi[3 * c + d] >= m) mine.push_back(c);
      else if (hi[3 * c + d] < m) left.push_back(c);
      else right.push_back(c);
    }
    raw[k].dofs = std::move(mine);
    int bl[6], br[6];
    std::copy(box, box + 6, bl);
    std::copy(box, box + 6, br);
    bl[2 * d + 1] = m;
    br[2 * d] = m;
    const int a = rec(bl, k, std::move(left));
    raw[k].kids.push_back(a);
    const int b = rec(br, k, std::move(right));
    raw[k].kids.push_back(b);
    return k;
  };
  {
    std::vector<int32_t> all(nc);
    for (int64_t c = 0; c < nc; ++c) all[c] = (int32_t)c;
    const int root_box[6] = {0, hs.P[0], 0, hs.P[1], 0, hs.P[2]};
    rec(root_box, -1, std::move(all));
  }
  // the separators of the top levels (depth < top) form one dense root block
  if (t.top > 1) {
    for (size_t k = 1; k < raw.size(); ++k)
      if (raw[k].depth < t.top) {
        raw[0].dofs.insert(raw[0].dofs.end(), raw[k].dofs.begin(), raw[k].dofs.end());
        raw[k].dofs.clear();
      }
    std::sort(raw[0].dofs.begin(), raw[0].dofs.end());
  }
  // remove empty nodes (their children move up to the nearest non-empty ancestor)
  std::vector<int> roots;
  std::vector<std::vector<int>> kids(raw.size());
  std::function<void(int, int)> attach = [&](int k, int up) {
    if (raw[k].dofs.empty()) {
      for (int c : raw[k].kids) attach(c, up);
      return;
    }
    if (up < 0) roots.push_back(k);
    else kids[up].push_back(k);
    for (int c : raw[k].kids) attach(c, k);
  };
  attach(0, -1);
  // postorder numbering and elimination order
  std::vector<int> order;
  std::function<void(int)> post = [&](int k) {
    for (int c : kids[k]) post(c);
    order.push_back(k);
  };
  for (int r : roots) post(r);
  const int NN = (int)order.size();
  t.n_nodes = NN;
  std::vector<int> id_of(raw.size(), -1);
  for (int p = 0; p < NN; ++p) id_of[order[p]] = p;
  t.k0.resize(NN);
  t.nk.resize(NN);
  t.ns.assign(NN, 0);
  t.parent.assign(NN, -1);
  t.box.resize(6 * (size_t)NN);
  t.perm.assign(nc, -1);
  int32_t pos = 0;
  for (int p = 0; p < NN; ++p) {
    const RawNode &r = raw[order[p]];
    t.k0[p] = pos;
    t.nk[p] = (int32_t)r.dofs.size();
    for (int32_t c : r.dofs) t.perm[c] = pos++;
    std::copy(r.box, r.box + 6, t.box.begin() + 6 * (size_t)p);
    for (int c : kids[order[p]]) t.parent[id_of[c]] = p;
  }
  if (pos != nc) {
    err = "nested dissection lost coarse unknowns";
    return IETI_ERR_INVALID_ARG;
  }
  // S_p: ancestor unknowns touching a patch of p's box
  t.s_off.assign(NN + 1, 0);
  std::vector<int32_t> buf;
  for (int p = 0; p < NN; ++p) {
    buf.clear();
    const int *bx = t.box.data() + 6 * (size_t)p;
    for (int a = t.parent[p]; a >= 0; a = t.parent[a])
      for (int32_t c : raw[order[a]].dofs) {
        bool touch = true;
        for (int e = 0; e < 3 && touch; ++e) touch = lo[3 * c + e] < bx[2 * e + 1] && hi[3 * c + e] >= bx[2 * e];
        if (touch) buf.push_back(t.perm[c]);
      }
    std::sort(buf.begin(), buf.end());
    t.ns[p] = (int32_t)buf.size();
    t.s_idx.insert(t.s_idx.end(), buf.begin(), buf.end());
    t.s_off[p + 1] = (int64_t)t.s_idx.size();
  }
  // children, levels
  t.child_ptr.assign(NN + 1, 0);
  for (int p = 0; p < NN; ++p)
    if (t.parent[p] >= 0) t.child_ptr[t.parent[p] + 1]++;
  for (int p = 0; p < NN; ++p) t.child_ptr[p + 1] += t.child_ptr[p];
  t.child_idx.assign(t.child_ptr[NN], 0);
  {
    std::vector<int32_t> fill(t.child_ptr.begin(), t.child_ptr.end() - 1);
    for (int p = 0; p < NN; ++p)
      if (t.parent[p] >= 0) t.child_idx[fill[t.parent[p]]++] = p;
  }
  t.height.assign(NN, 0);
  t.depth.assign(NN, 0);
  for (int p = 0; p < NN; ++p)
    for (int k = t.child_ptr[p]; k < t.child_ptr[p + 1]; ++k)
      t.height[p] = std::max(t.height[p], t.height[t.child_idx[k]] + 1);
  for (int p = NN - 1; p >= 0; --p) t.depth[p] = t.parent[p] < 0 ? 0 : t.depth[t.parent[p]] + 1;
  for (int p = 0; p < NN; ++p) {
    t.n_height = std::max(t.n_height, t.height[p] + 1);
    t.n_depth = std::max(t.n_depth, t.depth[p] + 1);
  }
  // a child's S set lies in its parent's front (what the extend-add relies on)
  for (int p = 0; p < NN; ++p) {
    if (t.parent[p] < 0) continue;
    for (int64_t k = t.s_off[p]; k < t.s_off[p + 1]; ++k)
      if (t.front_index(t.parent[p], t.s_idx[k]) < 0) {
        err = "nested dissection: a child's coupling set is not in its parent's front";
        return IETI_ERR_INVALID_ARG;
      }
  }
  return IETI_OK;
}

double coarse_tree_bytes(const CoarseTree &t) {
  double b = 0;
  for (int p = 0; p < t.n_nodes; ++p) b += 8.0 * ((double)(t.nk[p] + t.ns[p]) * t.nk[p] + (double)t.nk[p] * t.ns[p]);
  return b;
}

int coarse_tree_levels(const CoarseTree &t) { return t.n_nodes ? t.n_height + std::max(t.n_depth - 1, 0) : 0; }

int choose_coarse_tree(const HostSetup &hs, double bw, double latency, int leaf_fixed, int top_fixed,
                       CoarseTree &t, std::string &err, const std::vector<BoxCut> *cuts) {
  std::vector<int> leaves = {1, 8, 16, 27, 64, 125}, tops = {0, 2, 3};
  if (leaf_fixed > 0) leaves = {leaf_fixed};
  if (top_fixed > 0) tops = {top_fixed > 1 ? top_fixed : 0};
  double best = 1e300;
  bool any = false;
  for (int leaf : leaves)
    for (int top : tops) {
      CoarseTree c;
      int rc = build_coarse_tree(hs, leaf, top, c, err, cuts);
      if (rc) return rc;
      // blocks wider than 2048 unknowns leave a ring stage of the solve a single row:
      // only the candidate without merged top levels may have them (unless fixed)
      int widest = 0;
      for (int p = 0; p < c.n_nodes; ++p) widest = std::max({widest, c.nk[p], c.ns[p]});
      if (top > 0 && widest > 2048 && top_fixed == 0) continue;
      const double model = coarse_tree_bytes(c) / bw + coarse_tree_levels(c) * latency;
      if (!any || model < best * (1.0 - 1e-9)) {
        best = model;
        t = std::move(c);
        any = true;
      }
    }
  return IETI_OK;
}

}  // namespace ieti
