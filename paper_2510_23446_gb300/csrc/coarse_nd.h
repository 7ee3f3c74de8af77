// Nested-dissection structure of the primal coarse problem (Sec. 3: the coarse Schur
// complement S_c = sum_s A_s^T C_s A_s).  Two primal unknowns couple only when some
// patch holds copies of both, and every primal unknown sits on patch interfaces, so
// the patch grid itself gives a nested dissection: a box of patches is cut in the
// middle of its longest side and the unknowns whose patches lie on both sides of the
// cut form that node's separator block K_p.  The tree is stored in postorder; the
// unknowns are renumbered in elimination order, so that each node's block is the
// contiguous range [k0, k0 + nk) and every unknown of an ancestor comes later.
//
// Fill (multifrontal view): the factor's column block of node p couples to the
// ancestor unknowns that touch a patch of p's box, S_p (ascending).  A child's S set
// is contained in its parent's front [K_p; S_p], which is what the extend-add and
// the solves use.  Pure host code.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "host_setup.h"

namespace ieti {

struct CoarseTree {
  int64_t nc = 0;
  int n_nodes = 0;
  int leaf_max = 1;
  int top = 0;                          // separators of depth < top merged into the root
  std::vector<int32_t> perm;            // coarse id -> position in elimination order
  // per node, postorder (children before their parent)
  std::vector<int32_t> k0, nk, ns;      // own block [k0, k0 + nk), |S_p|
  std::vector<int32_t> parent;          // -1 for a root
  std::vector<int32_t> height, depth;   // leaves have height 0, roots depth 0
  std::vector<int32_t> box;             // [6 * p]: lo0, hi0, lo1, hi1, lo2, hi2 (patch index ranges, hi exclusive)
  std::vector<int64_t> s_off;           // S_p = s_idx[s_off[p] .. s_off[p + 1])
  std::vector<int32_t> s_idx;
  std::vector<int32_t> child_ptr, child_idx;
  int n_height = 0, n_depth = 0;        // levels of the forward (by height) and backward (by depth) sweeps
  // index of a position x of the parent's front [K_p; S_p] (x = global elimination position)
  int front_index(int p, int32_t x) const;
};

// Build the tree for the coarse unknowns of `hs` (boxes of leaf_max patches or fewer
// are not cut further; with top > 1 the separators of the top `top` levels form one
// root block; empty nodes are removed and their children re-attached).
// cuts (optional): boxes {x0, x1, y0, y1, z0, z1} with a prescribed cut {d, m}: a box
// equal to one of them is cut at plane m of direction d instead of the midpoint of its
// longest side (the cuts of a patch-sharded plan, so that every rank's patches form
// whole subtrees)
struct BoxCut {
  int box[6];
  int d, m;
};
int build_coarse_tree(const HostSetup &hs, int leaf_max, int top, CoarseTree &t, std::string &err,
                      const std::vector<BoxCut> *cuts = nullptr);

// Algorithmic bytes of one coarse solve on the tree (Z rows forward, Lt rows backward)
// and its grid-synchronised phases (levels by height, then by depth below the roots).
double coarse_tree_bytes(const CoarseTree &t);
int coarse_tree_levels(const CoarseTree &t);

// Tree shape of least modelled solve time over a fixed candidate list of leaf sizes
// and top merges: bytes / bw + phases * latency.  leaf > 0 / top > 0 fix that
// parameter (top 1: no merge).
int choose_coarse_tree(const HostSetup &hs, double bw, double latency, int leaf, int top, CoarseTree &t,
                       std::string &err, const std::vector<BoxCut> *cuts = nullptr);

}  // namespace ieti
