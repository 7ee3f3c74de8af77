"""Pins of the tree-cotree gauge and the e/p/r classes (Sec. 3)."""
import numpy as np
import pytest
import scipy.linalg as sla

from workloads import make_problem, small_problem
from oracle.gauge import Gauge, CLS_E, CLS_P, CLS_R
from oracle.lattice import Lattice
from oracle.manufactured import FieldEval
from oracle.stepping import OracleProblem


def _problems():
    return [make_problem("c1"), small_problem(),
            small_problem(P=(3, 2, 2), n_el=((2, 3, 2), (2, 3), (3, 2)),
                          degree=((1, 2, 1), (2, 1), (1, 2)),
                          conductor=((0.3, 0.7), (0, 1), (0, 1)), name="uneven"),
            small_problem(P=(3, 3, 3), n_el=((2, 2, 2), (2, 2, 2), (2, 2, 2)),
                          degree=((1, 1, 1), (1, 1, 1), (1, 1, 1)),
                          conductor=((0.4, 0.6), (0.4, 0.6), (0.4, 0.6)), name="buried")]


@pytest.mark.parametrize("prob", _problems(), ids=lambda p: p.name)
def test_tree_is_spanning_forest(prob):
    """Each component of the Omega_I graph (ROOT merged): #tree edges = #nodes - 1."""
    G = Gauge(prob)
    n_nodes, n_tree, n_comp = G.tree_counts()
    assert n_tree == n_nodes - n_comp
    # acyclic: union-find over the tree edges never closes a cycle
    parent = {}

    def find(x):
        while parent.setdefault(x, x) != x:
            x = parent[x]
        return x
    for e in np.nonzero(G.tree)[0]:
        a, b = find(int(G.u[e])), find(int(G.v[e]))
        assert a != b
        parent[a] = b
    assert not np.any(G.tree & ~G.in_graph)


@pytest.mark.parametrize("prob", _problems(), ids=lambda p: p.name)
def test_classes(prob):
    G = Gauge(prob)
    L = G.lat
    assert np.all(G.cls[L.dirichlet] == CLS_E)
    assert np.all(G.gtype[G.gamma & G.in_graph])
    gt = G.tree & G.gtype & (L.n_share >= 2)
    assert np.all(G.cls[gt] == CLS_P)
    assert np.all(G.cls[G.tree & G.touch_i & ~G.gtype] == CLS_E)
    # nothing that touches only the conductor is eliminated
    conductor_only = G.touch_c & ~G.touch_i & ~L.dirichlet
    assert np.all(G.cls[conductor_only] == CLS_R)


@pytest.mark.parametrize("prob", _problems(), ids=lambda p: p.name)
def test_local_blocks_nonsingular(prob):
    """Sec. 3: the splitting yields a non-singular W_rr on every patch; the interior
    blocks W_ii of the Dirichlet preconditioner are non-singular too."""
    op = OracleProblem(prob)
    dec = op.dec
    for s in range(prob.n_patches):
        W = (op.asm.M[s] + prob.dt * op.asm.K[s]).toarray()
        r = np.concatenate([dec.i_loc[s], dec.b_loc[s]])
        for idx in (r, dec.i_loc[s]):
            if len(idx) == 0:
                continue
            ev = np.linalg.eigvalsh(W[np.ix_(idx, idx)])
            assert ev[0] > 1e-10 * ev[-1], (s, ev[0], ev[-1])
    # and the global gauged system is non-singular
    ev = np.linalg.eigvalsh(op.mono.W.toarray())
    assert ev[0] > 1e-12 * ev[-1]


def test_eliminated_edges_gaugeable():
    """a_e = 0 must be reachable by adding a discrete gradient that vanishes on the
    conductor: after contracting ROOT and each group of conductor nodes joined by
    Gamma-type tree edges, the eliminated tree edges must form a forest (no path of
    eliminated edges between two fixed nodes)."""
    for prob in _problems():
        G = Gauge(prob)
        parent = {}

        def find(x):
            while parent.setdefault(x, x) != x:
                x = parent[x]
            return x
        for e in np.nonzero(G.tree & G.gtype)[0]:
            parent[find(int(G.u[e]))] = find(int(G.v[e]))
        # conductor nodes on the boundary are ROOT; all other conductor nodes keep
        # their groups; eliminated edges must not close a cycle
        for e in np.nonzero(G.tree & (G.cls == CLS_E))[0]:
            a, b = find(int(G.u[e])), find(int(G.v[e]))
            assert a != b, (prob.name, e)
            parent[a] = b


def _fields(op, steps=3):
    fe = FieldEval(op.prob, op.asm)
    a = op.run_monolithic(steps)[-1]
    curls, consts = [], []
    for s, pe in enumerate(fe.pe):
        c = a[op.asm.l2g[s]][pe.loc]
        curls.append(np.einsum("ea,eqai->eqi", c, fe.curls[s]))
        cond = (op.prob.patch_sigma(s).reshape(-1) > 0)
        consts.append(np.einsum("ea,eqai->eqi", c, fe.vals[s])[cond])
    return np.concatenate([x.ravel() for x in curls]), np.concatenate([x.ravel() for x in consts])


@pytest.mark.parametrize("idx", [0, 2, 3])
def test_gauge_invariance(idx):
    """B = curl A everywhere and A in Omega_C do not depend on the tree (Sec. 2:
    only gradients in Omega_I are undetermined), provided the Gamma tree DOFs are
    primal (Sec. 3); eliminating them instead must change the conductor field."""
    prob = _problems()[idx]
    op1 = OracleProblem(prob)
    op2 = OracleProblem(prob, reverse_ties=True)
    assert np.any(op1.gauge.tree != op2.gauge.tree)
    B1, A1 = _fields(op1)
    B2, A2 = _fields(op2)
    assert np.linalg.norm(B1 - B2) <= 1e-9 * np.linalg.norm(B1)
    assert np.linalg.norm(A1 - A2) <= 1e-9 * np.linalg.norm(A1)
    bad = OracleProblem(prob, gamma_tree_primal=False)
    if np.any(bad.gauge.cls != op1.gauge.cls):
        B3, A3 = _fields(bad)
        assert np.linalg.norm(A1 - A3) > 1e-4 * np.linalg.norm(A1)
