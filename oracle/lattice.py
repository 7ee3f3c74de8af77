"""Global control-mesh numbering for a structured grid of conforming patches.

Sec. 2.2 requires pairwise matching basis functions on interfaces; with open knot
vectors that match across each shared face, the control points of all patches form
one global lattice (I, J, K) in which neighbouring patches share the lattice planes
of their common face.  An edge DOF of the spline edge space is then a lattice edge
(Sec. 3 puts the tree on the control mesh); a node is a lattice point.

Numbering (the library uses the same published convention, written separately):
* node id  = I + N0*(J + N1*K);
* edge id  : direction-0 edges first, id = I + (N0-1)*(J + N1*K); then direction 1,
  offset E0, id = I + N0*(J + (N1-1)*K); then direction 2, offset E0+E1,
  id = I + N0*(J + N1*K).  An edge of direction d at (I,J,K) joins node (I,J,K) to
  the node one step further in d.
* patch-local edge DOFs: component-major, then (i, j, k) with i fastest; component
  d has n_d - 1 functions in direction d and n_e in the others.
"""
from __future__ import annotations

import numpy as np


class Lattice:
    def __init__(self, prob):
        self.prob = prob
        self.P = tuple(int(x) for x in prob.P)
        self.nslab = [[int(prob.n_el[d][a]) + int(prob.degree[d][a]) for a in range(self.P[d])]
                      for d in range(3)]
        self.off = []
        self.N = []
        for d in range(3):
            o = [0]
            for a in range(self.P[d] - 1):
                o.append(o[-1] + self.nslab[d][a] - 1)
            self.off.append(np.asarray(o, dtype=np.int64))
            self.N.append(int(o[-1] + self.nslab[d][-1]))
        N0, N1, N2 = self.N
        self.E = [(N0 - 1) * N1 * N2, N0 * (N1 - 1) * N2, N0 * N1 * (N2 - 1)]
        self.edge_off = [0, self.E[0], self.E[0] + self.E[1]]
        self.n_edges = sum(self.E)
        self.n_nodes = N0 * N1 * N2
        # slab-boundary lattice planes per direction
        self.sb = [np.asarray(sorted(set(self.off[d].tolist()) | {self.N[d] - 1}), dtype=np.int64)
                   for d in range(3)]
        self._edge_arrays()

    # ---------------- edges ----------------
    def edge_id(self, d, I, J, K):
        N0, N1, _ = self.N
        if d == 0:
            return self.edge_off[0] + I + (N0 - 1) * (J + N1 * K)
        if d == 1:
            return self.edge_off[1] + I + N0 * (J + (N1 - 1) * K)
        return self.edge_off[2] + I + N0 * (J + N1 * K)

    def _edge_arrays(self):
        N0, N1, N2 = self.N
        dirs, Is, Js, Ks = [], [], [], []
        for d, shape in enumerate([(N2, N1, N0 - 1), (N2, N1 - 1, N0), (N2 - 1, N1, N0)]):
            K, J, I = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]),
                                  indexing="ij")
            dirs.append(np.full(K.size, d))
            Is.append(I.ravel()); Js.append(J.ravel()); Ks.append(K.ravel())
        self.edir = np.concatenate(dirs)
        self.eI = np.concatenate(Is); self.eJ = np.concatenate(Js); self.eK = np.concatenate(Ks)
        coords = np.stack([self.eI, self.eJ, self.eK], axis=1)
        step = np.eye(3, dtype=np.int64)[self.edir]
        self.node0 = self.node_id(coords[:, 0], coords[:, 1], coords[:, 2])
        c1 = coords + step
        self.node1 = self.node_id(c1[:, 0], c1[:, 1], c1[:, 2])
        # per transverse direction: on the global boundary / on a slab-boundary plane
        on_bnd = np.zeros(self.n_edges, dtype=bool)
        n_sb = np.zeros(self.n_edges, dtype=np.int64)
        n_internal_sb = np.zeros(self.n_edges, dtype=np.int64)
        for e in range(3):
            ce = coords[:, e]
            trans = self.edir != e
            at_b = trans & ((ce == 0) | (ce == self.N[e] - 1))
            at_sb = trans & np.isin(ce, self.sb[e])
            on_bnd |= at_b
            n_sb += at_sb
            n_internal_sb += at_sb & ~at_b
        self.dirichlet = on_bnd                    # tangential edge lying on the boundary
        self.kind = n_sb                           # 0 interior, 1 face, 2 wirebasket
        self.n_share = 2 ** n_internal_sb          # patches sharing the edge
        self.coords = coords

    # ---------------- nodes ----------------
    def node_id(self, I, J, K):
        N0, N1, _ = self.N
        return I + N0 * (J + N1 * K)

    def node_coords(self, n):
        N0, N1, _ = self.N
        return n % N0, (n // N0) % N1, n // (N0 * N1)

    def is_boundary_node(self, n):
        I, J, K = self.node_coords(n)
        return ((I == 0) | (I == self.N[0] - 1) | (J == 0) | (J == self.N[1] - 1)
                | (K == 0) | (K == self.N[2] - 1))

    # ---------------- patches ----------------
    def patch_sizes(self, s):
        a, b, c = self.prob.patch_index(s)
        return self.nslab[0][a], self.nslab[1][b], self.nslab[2][c]

    def patch_local_to_global(self, s):
        """Global edge id of every patch-local edge DOF (component-major, i fastest)."""
        a, b, c = self.prob.patch_index(s)
        n0, n1, n2 = self.patch_sizes(s)
        o = (self.off[0][a], self.off[1][b], self.off[2][c])
        out = []
        for d, shape in enumerate([(n2, n1, n0 - 1), (n2, n1 - 1, n0), (n2 - 1, n1, n0)]):
            k, j, i = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]),
                                  indexing="ij")
            out.append(self.edge_id(d, i.ravel() + o[0], j.ravel() + o[1], k.ravel() + o[2]))
        return np.concatenate(out).astype(np.int64)

    def patch_node_ids(self, s):
        a, b, c = self.prob.patch_index(s)
        n0, n1, n2 = self.patch_sizes(s)
        k, j, i = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
        return np.unique(self.node_id(i.ravel() + self.off[0][a], j.ravel() + self.off[1][b],
                                      k.ravel() + self.off[2][c]))

    def patches_of_edges(self):
        """List of sharing patch ids (ascending) per global edge."""
        owners = [[] for _ in range(self.n_edges)]
        for s in range(self.prob.n_patches):
            for g in self.patch_local_to_global(s):
                owners[g].append(s)
        return owners
