// Host-side setup of the tree-cotree IETI-DP solver: spline spaces and patch
// matrices (Sec. 2.2), lattice numbering, the hierarchical tree-cotree gauge and
// e/p/r classes (Sec. 3), multipliers and the primal map.  Pure C++17.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ieti.h"

namespace ieti {

enum : int8_t { CLS_E = 0, CLS_P = 1, CLS_R = 2 };

struct Csr {                       // square CSR, sorted columns
  int n = 0;
  std::vector<int32_t> ptr, col;
  std::vector<double> val;
};

struct Patch {
  int a = 0, b = 0, c = 0;
  int p[3]{}, ne[3]{}, n[3]{};     // degree, elements, H^1 functions per direction
  int n_dofs = 0;                  // local edge DOFs
  std::vector<int64_t> l2g;        // local DOF -> global edge
  Csr K, M;                        // local numbering, same pattern
  // decomposition (local DOF ids, ascending)
  std::vector<int32_t> i_loc, b_loc, p_loc;
  // kept numbering [i | b | p]
  int ni = 0, nb = 0, np = 0;
  Csr Wk, Mk;                      // W = M + dt K and M in the kept numbering
  std::vector<int64_t> kept_glob;  // kept index -> global edge
  std::vector<double> load_w;      // kept index -> 1/n_share
  std::vector<int32_t> loc2kept;   // local DOF -> kept index (-1: eliminated)
};

// Quadrature tables of the elements with the nonlinear reluctivity (one entry per
// element of a patch listed in `patches`): at point q of element e and its local
// function a, G[q][a][:] = (DF c_hat_a) sqrt(w / det) and cq[q] = 1 / sqrt(w det),
// so that B_q = cq[q] sum_a x_a G[q][a], the stiffness is sum_q nu G_a.G_b and
// the residual sum_q nu (B_q . G[q][a]) / cq[q].
struct NlTables {
  std::vector<int32_t> patches;                 // global ids of the patches holding such elements
  std::vector<int32_t> el_batch;                // element -> position in `patches`
  std::vector<int32_t> nloc, nq;                // per element
  std::vector<int64_t> g_off, q_off, d_off;     // per element offsets into G / cq / kept,glob
  std::vector<double> G, cq;
  std::vector<int32_t> kept;                    // per element function: kept index in its patch, -1 eliminated
  std::vector<int64_t> glob;                    // per element function: global edge
};

struct Multiplier {                // lambda = (copy in s) - (copy in t), s < t
  int64_t edge;
  int32_t s, pos_s, t, pos_t;      // pos_* = index inside that patch's b-list
};

struct HostSetup {
  // problem
  int P[3]{};
  std::vector<int32_t> n_el[3], degree[3];          // [d][slab]
  std::vector<std::vector<double>> knots[3];        // [d][slab] full knot vector
  std::vector<double> ctrl;                         // as given
  std::vector<int64_t> ctrl_off;                    // per patch offset (doubles)
  std::vector<double> sigma_el, nu_el;
  std::vector<int64_t> el_off;
  bool nonlinear = false;                           // nu(|B|) law in the conducting elements
  double law[4]{};                                  // nu0, k1, k2, k3
  NlTables nl;
  double dt = 0;
  int threads = 0;
  // lattice
  std::vector<int64_t> off[3];
  int64_t N[3]{}, E[3]{}, edge_off[3]{};
  int64_t n_edges = 0, n_nodes = 0;
  std::vector<uint8_t> is_sb[3];                    // lattice index on a slab plane
  // per edge
  std::vector<uint8_t> dirichlet, kind, n_share, touch_c, touch_i, gtype, in_graph, tree;
  std::vector<int8_t> cls;
  std::vector<uint8_t> cnode;                       // per node
  // patches and decomposition
  std::vector<Patch> patches;
  std::vector<Multiplier> lam;
  int64_t n_coarse = 0;
  std::vector<int64_t> coarse_of_edge;              // -1 unless primal
  std::vector<int64_t> free_edges;                  // r + p, ascending
  double t_ms = 0;

  int build(const ieti_problem *pr, int threads, std::string &err);
  // helpers
  int64_t edge_id(int d, int64_t I, int64_t J, int64_t K) const;
  void edge_coords(int64_t g, int &d, int64_t &I, int64_t &J, int64_t &K) const;
  int64_t node_id(int64_t I, int64_t J, int64_t K) const { return I + N[0] * (J + N[1] * K); }
  bool boundary_node(int64_t n) const;
  int slab_start(int d, int64_t I) const;
  int n_patches() const { return P[0] * P[1] * P[2]; }
  // load vector of a coil potential, global numbering
  void coil_load(const ieti_coil &coil, double *out) const;
  // quadrature points of the assembly (patch, element, point order): count, offsets
  // per patch, physical coordinates; load vector of a field sampled at them
  int64_t quad_point_count(std::vector<int64_t> *patch_off = nullptr) const;
  void quad_points(double *xyz) const;
  void points_load(const double *J, double *out) const;

 private:
  int validate(const ieti_problem *pr, std::string &err);
  void lattice();
  void assemble_all();
  void assemble_patch(Patch &pt) const;
  void regions();
  void build_tree();
  void bfs_pass(const std::vector<int64_t> &edges, std::vector<uint8_t> &visited,
                const std::vector<int64_t> &u, const std::vector<int64_t> &v);
  void classify();
  void decompose();
  void nl_tables();
  bool nl_element(int s, int el) const { return nonlinear && sigma_el[el_off[s] + el] > 0.0; }
};

}  // namespace ieti
