// Patch-sharded layout of the dual-primal solve for several ranks (Sec. 3: the patch
// problems are independent; the interface problem couples them through the jumps of
// the multipliers, the coarse right-hand side and the PCG dot products).
//
// The patch grid is cut by recursive coordinate bisection into n_ranks boxes balanced by
// the patches' local sizes.  A multiplier (copy in patch s) - (copy in patch t), s < t,
// belongs to the rank holding s; it is cut when t lies on another rank, whose partial
// jump (its copy's contribution) then crosses once per PCG iteration.  A coarse unknown
// belongs to the lowest rank holding one of its copies; the coarse right-hand side is
// summed over the ranks holding copies.  Pure host code.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "coarse_nd.h"
#include "host_setup.h"

namespace ieti {

struct ShardPlan {
  int n_ranks = 1;
  std::vector<int32_t> rank_of_patch;   // [n_patches]
  std::vector<int32_t> lam_owner;       // [n_lambda] rank of the multiplier's lower patch
  std::vector<int32_t> lam_peer;        // [n_lambda] rank of the upper patch when it differs, else -1
  std::vector<int32_t> coarse_owner;    // [n_coarse] lowest rank holding a copy
  std::vector<int32_t> coarse_ranks;    // [n_coarse] bit mask of the ranks holding copies (n_ranks <= 31)
  std::vector<double> rank_weight;      // [n_ranks] summed local sizes
  std::vector<BoxCut> cuts;             // the bisection's cuts (box, direction, plane)
};

int build_shard_plan(const HostSetup &hs, int n_ranks, ShardPlan &plan, std::string &err);

// The coarse solve on the same ranks: node p of the nested-dissection tree belongs to
// rank r when every patch of its box is on r (its rows and the subtree below it are
// computed there), else -1: a shared node of the top, computed by every rank once the
// owned subtrees' updates into it are summed over the ranks (one allreduce per solve;
// a descendant of an owned node is owned by the same rank, an ancestor of a shared
// node is shared).
int shard_coarse_nodes(const HostSetup &hs, const CoarseTree &t, const ShardPlan &plan,
                       std::vector<int32_t> &node_rank, std::string &err);

}  // namespace ieti
