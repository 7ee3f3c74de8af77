"""Tree-cotree gauge and the e / p / r splitting of Sec. 3.

Sec. 3: a tree is built on the control mesh of the insulating region, "globally on
the wirebasket first", then "extended into the subdomain faces and at last into the
subdomain interiors"; tree DOFs inside Omega_I and all Dirichlet DOFs are eliminated
(e); tree DOFs on Gamma are primal (p); everything else is remaining (r).

Readings (the paper fixes only the stage order; the tie-breaks below are ours and
are shared, as a written specification, with the library):

* Regions by support: an edge DOF touches Omega_C (Omega_I) when the support of its
  basis function, in any patch holding it, contains an element with sigma > 0
  (sigma == 0).  Omega_I edges = edges touching Omega_I; Gamma edges touch both.
  A node is a conductor node when the support of its H^1 function contains a
  conducting element; on the kernel of W (gradients) the potential is constant
  over each connected set of conductor nodes.
* Graph: nodes and non-Dirichlet edges of Omega_I; all nodes on the outer boundary
  are merged into one ROOT (the PEC boundary is one connected conductor).
* Gamma-type edges: graph edges whose two end nodes are conductor nodes (this
  includes every Gamma edge).  Consistency (Sec. 3: tree DOFs coupled across Gamma
  take their values from the conducting side) needs the tree restricted to
  Gamma to be connected: otherwise a path of eliminated edges joins two Gamma nodes
  and a_e = 0 forces a gauge-invariant line integral of A to zero.  In the paper's
  two-subdomain test Gamma touches the boundary and this holds through ROOT; with
  a conductor inside the domain it must be built in.  So every stage below first
  runs over its Gamma-type edges, then over the rest.
* Stage 1 wirebasket edges (two transverse lattice indices on slab planes); stage 2
  face edges face by face in ascending face id; stage 3 interior edges patch by
  patch in ascending patch id.  Each pass is a multi-source BFS whose sources are
  the already-reached nodes of the pass's edges (ROOT first, then ascending node
  id), neighbours taken in ascending edge id, a node adopting the edge by which it
  is first reached; nodes still unreached start new BFS trees in ascending node id.
  Stage 4: Kruskal in ascending edge id (Gamma-type edges first, then all) joins
  any components left.
* Classes: Dirichlet -> e.  Omega_I tree edge: Gamma-type and shared by >= 2
  patches -> p, Gamma-type inside one patch -> r (the conductor fixes it), else ->
  e.  Omega_I cotree wirebasket edge (shared by 4 patches) -> p, so that every
  insulating patch keeps its whole wirebasket fixed and its local problem stays
  non-singular when the global tree is cut inside it (needed with many insulating
  patches; the paper treats two subdomains).  Everything else -> r.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from .lattice import Lattice

CLS_E, CLS_P, CLS_R = 0, 1, 2


def _box_any(mask, lo, hi):
    """any(mask[z0:z1+1, y0:y1+1, x0:x1+1]) for per-DOF inclusive windows."""
    S = np.zeros(tuple(m + 1 for m in mask.shape))
    S[1:, 1:, 1:] = mask.astype(np.float64).cumsum(0).cumsum(1).cumsum(2)
    z0, y0, x0 = lo
    z1, y1, x1 = hi
    tot = (S[z1 + 1, y1 + 1, x1 + 1] - S[z0, y1 + 1, x1 + 1] - S[z1 + 1, y0, x1 + 1]
           - S[z1 + 1, y1 + 1, x0] + S[z0, y0, x1 + 1] + S[z0, y1 + 1, x0]
           + S[z1 + 1, y0, x0] - S[z0, y0, x0])
    return tot > 0.5


def conductor_nodes(prob, s):
    """Flag per patch control point (k, j, i order, i fastest): H^1 support meets sigma > 0."""
    ne = prob.patch_n_el(s)
    pd = prob.patch_degree(s)
    n = [ne[d] + pd[d] for d in range(3)]
    sig = prob.patch_sigma(s)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = [i.ravel(), j.ravel(), k.ravel()]
    lo = [np.clip(idx[d] - pd[d], 0, ne[d] - 1) for d in range(3)]
    hi = [np.clip(idx[d], 0, ne[d] - 1) for d in range(3)]
    return _box_any(sig > 0, (lo[2], lo[1], lo[0]), (hi[2], hi[1], hi[0]))


def support_flags(prob, s):
    """(touches_C, touches_I) for every patch-local edge DOF of patch s."""
    ne = prob.patch_n_el(s)
    pd = prob.patch_degree(s)
    n = [ne[d] + pd[d] for d in range(3)]
    sig = prob.patch_sigma(s)                 # (E2, E1, E0)
    out_c, out_i = [], []
    for comp in range(3):
        shape = [n[d] - (1 if d == comp else 0) for d in range(3)]
        k, j, i = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]),
                              indexing="ij")
        idx = [i.ravel(), j.ravel(), k.ravel()]
        lo, hi = [], []
        for d in range(3):
            if d == comp:          # D_i: elements i+1-p .. i
                a, b = idx[d] + 1 - pd[d], idx[d]
            else:                  # N_j: elements j-p .. j
                a, b = idx[d] - pd[d], idx[d]
            lo.append(np.clip(a, 0, ne[d] - 1))
            hi.append(np.clip(b, 0, ne[d] - 1))
        zl, yl, xl = lo[2], lo[1], lo[0]
        zh, yh, xh = hi[2], hi[1], hi[0]
        out_c.append(_box_any(sig > 0, (zl, yl, xl), (zh, yh, xh)))
        out_i.append(_box_any(sig == 0, (zl, yl, xl), (zh, yh, xh)))
    return np.concatenate(out_c), np.concatenate(out_i)


class Gauge:
    def __init__(self, prob, lat: Lattice | None = None, reverse_ties=False,
                 gamma_tree_primal=True):
        # reverse_ties: take every BFS tie-break in descending order instead (a second,
        # different tree for the gauge-invariance pin).  gamma_tree_primal=False
        # eliminates Gamma tree edges instead of making them primal (the inconsistent
        # gauge Sec. 3 warns about; used only to show that the pins catch it).
        self.reverse_ties = reverse_ties
        self.gamma_tree_primal = gamma_tree_primal
        self.prob = prob
        L = self.lat = lat or Lattice(prob)
        self.touch_c = np.zeros(L.n_edges, dtype=bool)
        self.touch_i = np.zeros(L.n_edges, dtype=bool)
        for s in range(prob.n_patches):
            g = L.patch_local_to_global(s)
            c, i = support_flags(prob, s)
            self.touch_c[g] |= c
            self.touch_i[g] |= i
        self.gamma = self.touch_c & self.touch_i
        self.in_graph = self.touch_i & ~L.dirichlet
        self.cnode = np.zeros(L.n_nodes, dtype=bool)
        for s in range(prob.n_patches):
            self.cnode[L.patch_node_ids(s)] |= conductor_nodes(prob, s)
        self.gtype = self.in_graph & self.cnode[L.node0] & self.cnode[L.node1]
        self.ROOT = L.n_nodes
        bnd0 = L.is_boundary_node(L.node0)
        bnd1 = L.is_boundary_node(L.node1)
        self.u = np.where(bnd0, self.ROOT, L.node0)
        self.v = np.where(bnd1, self.ROOT, L.node1)
        self.tree = np.zeros(L.n_edges, dtype=bool)
        self.visited = np.zeros(L.n_nodes + 1, dtype=bool)
        self._build_tree()
        self._classify()

    # ---------------- tree ----------------
    def _stage(self, edges):
        """Multi-source BFS over the given (ascending) edge ids."""
        adj = {}
        for e in edges:
            a, b = int(self.u[e]), int(self.v[e])
            adj.setdefault(a, []).append((int(e), b))
            adj.setdefault(b, []).append((int(e), a))
        nodes = sorted(adj.keys(), key=lambda x: -1 if x == self.ROOT else x)
        if self.reverse_ties:
            nodes = nodes[:1] + nodes[1:][::-1] if nodes and nodes[0] == self.ROOT else nodes[::-1]
            for k in adj:
                adj[k] = adj[k][::-1]
        q = deque(x for x in nodes if self.visited[x])

        def run():
            while q:
                x = q.popleft()
                for e, y in adj[x]:
                    if not self.visited[y]:
                        self.visited[y] = True
                        self.tree[e] = True
                        q.append(y)
        run()
        for x in nodes:
            if not self.visited[x]:
                self.visited[x] = True
                q.append(x)
                run()

    def _build_tree(self):
        L = self.lat
        self.visited[self.ROOT] = True
        ids = np.nonzero(self.in_graph)[0]
        # stage 1: wirebasket
        self._two_pass(ids[L.kind[ids] == 2])
        # stage 2: faces in ascending face id
        fids = ids[L.kind[ids] == 1]
        fkey = self._face_ids(fids)
        order = np.lexsort((fids, fkey))
        fids, fkey = fids[order], fkey[order]
        for grp in np.split(np.arange(len(fids)), np.nonzero(np.diff(fkey))[0] + 1):
            if len(grp):
                self._two_pass(fids[grp])
        # stage 3: patch interiors in ascending patch id
        iids = ids[L.kind[ids] == 0]
        pkey = self._interior_patch(iids)
        order = np.lexsort((iids, pkey))
        iids, pkey = iids[order], pkey[order]
        for grp in np.split(np.arange(len(iids)), np.nonzero(np.diff(pkey))[0] + 1):
            if len(grp):
                self._two_pass(iids[grp])
        # stage 4: Kruskal over all graph edges in ascending id
        parent = np.arange(L.n_nodes + 1)

        def find(x):
            r = x
            while parent[r] != r:
                r = parent[r]
            while parent[x] != r:
                parent[x], x = r, parent[x]
            return r
        for e in np.nonzero(self.tree)[0]:
            parent[find(self.u[e])] = find(self.v[e])
        for e in np.concatenate([ids[self.gtype[ids]], ids]):
            if self.tree[e]:
                continue
            a, b = find(self.u[e]), find(self.v[e])
            if a != b:
                self.tree[e] = True
                parent[a] = b

    def _two_pass(self, edges):
        """One stage: its Gamma-type edges first, then the remaining ones."""
        g = self.gtype[edges]
        if np.any(g):
            self._stage(edges[g])
        if np.any(~g):
            self._stage(edges[~g])

    def _slab_start(self, d, I):
        return np.searchsorted(self.lat.off[d], I, side="right") - 1

    def _face_ids(self, eids):
        L = self.lat
        P = L.P
        out = np.zeros(len(eids), dtype=np.int64)
        foff = [0, (P[0] + 1) * P[1] * P[2], (P[0] + 1) * P[1] * P[2] + P[0] * (P[1] + 1) * P[2]]
        for k, e in enumerate(eids):
            d = L.edir[e]
            c = L.coords[e]
            f = [x for x in range(3) if x != d and c[x] in set(L.sb[x].tolist())][0]
            g = int(np.searchsorted(L.sb[f], c[f]))
            inplane = [x for x in range(3) if x != f]
            t = [int(self._slab_start(x, c[x])) for x in inplane]
            out[k] = foff[f] + g + (P[f] + 1) * (t[0] + P[inplane[0]] * t[1])
        return out

    def _interior_patch(self, eids):
        L = self.lat
        P = L.P
        t = [self._slab_start(d, L.coords[eids, d]) for d in range(3)]
        return t[0] + P[0] * (t[1] + P[1] * t[2])

    # ---------------- classes ----------------
    def _classify(self):
        L = self.lat
        cls = np.full(L.n_edges, CLS_R, dtype=np.int8)
        shared = L.n_share >= 2
        tree_i = self.tree & self.touch_i
        cls[tree_i & ~self.gtype] = CLS_E
        cls[tree_i & self.gtype & shared] = CLS_P if self.gamma_tree_primal else CLS_E
        cot_wb = self.in_graph & ~self.tree & (L.kind == 2) & shared
        cls[cot_wb] = CLS_P
        cls[L.dirichlet] = CLS_E
        self.cls = cls

    def tree_counts(self):
        """(#graph nodes incl. ROOT, #tree edges, #components) of the Omega_I graph."""
        ids = np.nonzero(self.in_graph)[0]
        nodes = np.unique(np.concatenate([self.u[ids], self.v[ids]]))
        parent = {int(x): int(x) for x in nodes}

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x
        for e in ids:
            a, b = find(int(self.u[e])), find(int(self.v[e]))
            if a != b:
                parent[a] = b
        comps = len({find(int(x)) for x in nodes})
        return len(nodes), int(self.tree.sum()), comps
