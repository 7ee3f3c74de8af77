"""Host logic of the nested-dissection coarse solve (Sec. 3: the coarse Schur
complement S_c), checked on CPU against the oracle's dense S_c.

The library builds, for every context, a nested dissection of the patch grid: tree
nodes in postorder own contiguous blocks of the elimination order, and node p couples
to the ancestor unknowns S_p.  The device factors S_c along this tree (multifrontal)
and solves with one forward and one backward sweep.  These tests take the tree from
the library (ieti_coarse_tree, host-only context) and the coarse matrix from the
oracle, and check

* the tree is a valid elimination structure: a permutation, postorder blocks, and
  every pair of coupled unknowns lies on one root path;
* the fronts hold the whole fill: every structural entry of the Cholesky factor of
  S_c (in elimination order) below a node's block lies in that node's S_p;
* the multifrontal algebra the kernels implement (fronts from the K columns of S_c,
  extend-add of the children's update matrices, D^{-1} and Lbar = F_SK D^{-1}, the
  forward sweep by height and the backward sweep by depth), run here in numpy on the
  library's tree, solves S_c q = c exactly (against numpy's dense solve).
"""
import numpy as np
import pytest

from workloads import make_problem, small_problem
from oracle.stepping import OracleProblem

CASES = {
    "c1": lambda: make_problem("c1"),
    "buried": lambda: small_problem(P=(3, 3, 3), n_el=((2, 2, 2),) * 3, degree=((1, 1, 1),) * 3,
                                    conductor=((0.4, 0.6),) * 3),
    "ragged_p23": lambda: small_problem(P=(4, 3, 2), n_el=((3, 2, 5, 2), (2, 4, 2), (3, 2)),
                                        degree=((2, 3, 2, 2), (3, 2, 2), (2, 3)),
                                        conductor=((0.2, 0.8), (0.3, 0.7), (0.0, 1.0)), sigma=50.0, dt=0.01),
    "c4_family": lambda: make_problem("c4", patches_per_dir=3, el_range=(2, 3)),
}

_ORACLE = {}


@pytest.fixture(scope="module")
def ieti():
    try:
        from paper_2510_23446_gb300 import ieti as mod
    except Exception as e:   # noqa: BLE001
        pytest.skip(f"library not built: {e}")
    return mod


def _setup(ieti, name, leaf, top=0):
    if name not in _ORACLE:
        prob = CASES[name]()
        I = OracleProblem(prob).ietidp()
        _ORACLE[name] = (prob, I.Sc, np.nonzero(I.dec.gauge.cls == 1)[0])
    prob, Sc, prim = _ORACLE[name]
    S = ieti.Solver.from_problem(prob, device=-1, coarse_leaf=leaf, coarse_top=top)
    t = S.coarse_tree()
    S.close()
    # oracle coarse index i (primal edges ascending) -> elimination position
    pos = t["elim_pos"][prim]
    assert np.all(pos >= 0) and np.array_equal(np.sort(pos), np.arange(len(prim)))
    Sp = np.zeros_like(Sc)
    Sp[np.ix_(pos, pos)] = Sc
    return t, Sp


def _nodes(t):
    nn = len(t["k0"])
    S = [t["s_idx"][t["s_off"][p]:t["s_off"][p + 1]] for p in range(nn)]
    kids = [[] for _ in range(nn)]
    for p in range(nn):
        if t["parent"][p] >= 0:
            kids[t["parent"][p]].append(p)
    return nn, S, kids


# (leaf size, top merge): coarse_top k >= 2 merges the separators of the top k levels
SHAPES = [(1, 0), (8, 0), (1, 2), (1, 3)]


@pytest.mark.parametrize("leaf,top", SHAPES)
@pytest.mark.parametrize("name", list(CASES))
def test_tree_is_an_elimination_structure(ieti, name, leaf, top):
    t, Sp = _setup(ieti, name, leaf, top)
    nn, S, kids = _nodes(t)
    nc = Sp.shape[0]
    assert nn > 0 and t["k0"][0] == 0 and t["k0"][-1] + t["nk"][-1] == nc
    assert np.all(t["k0"][1:] == t["k0"][:-1] + t["nk"][:-1]) and np.all(t["nk"] > 0)
    assert all(t["parent"][p] > p or t["parent"][p] == -1 for p in range(nn))
    node = np.repeat(np.arange(nn), t["nk"])
    anc = [set() for _ in range(nn)]
    for p in range(nn - 1, -1, -1):
        q = t["parent"][p]
        anc[p] = ({q} | anc[q]) if q >= 0 else set()
    # coupled unknowns (S_c entry) on one root path, S_p ancestors only, sorted
    I, J = np.nonzero(np.abs(Sp) > 1e-14 * np.abs(Sp).max())
    for i, j in zip(I, J):
        a, b = node[i], node[j]
        assert a == b or a in anc[b] or b in anc[a]
    for p in range(nn):
        assert np.all(np.diff(S[p]) > 0)
        assert all(node[x] in anc[p] for x in S[p])


@pytest.mark.parametrize("leaf,top", SHAPES)
@pytest.mark.parametrize("name", list(CASES))
def test_fronts_hold_the_fill(ieti, name, leaf, top):
    t, Sp = _setup(ieti, name, leaf, top)
    nn, S, _ = _nodes(t)
    L = np.linalg.cholesky(Sp)
    tiny = 1e-12 * np.abs(L).max()
    for p in range(nn):
        k0, nk = t["k0"][p], t["nk"][p]
        rows = np.nonzero(np.abs(L[k0 + nk:, k0:k0 + nk]).max(axis=1) > tiny)[0] + k0 + nk
        assert set(rows.tolist()) <= set(S[p].tolist()), (p, sorted(set(rows) - set(S[p])))


def _multifrontal_solve(t, Sp, c):
    """The device algorithm, step by step, in numpy."""
    nn, S, kids = _nodes(t)
    k0, nk = t["k0"], t["nk"]
    front = [np.concatenate([np.arange(k0[p], k0[p] + nk[p]), S[p]]) for p in range(nn)]
    height = np.zeros(nn, dtype=int)
    for p in range(nn):
        for ch in kids[p]:
            height[p] = max(height[p], height[ch] + 1)
    depth = np.zeros(nn, dtype=int)
    for p in range(nn - 1, -1, -1):
        depth[p] = 0 if t["parent"][p] < 0 else depth[t["parent"][p]] + 1
    Dinv, Lbar, U = [None] * nn, [None] * nn, [None] * nn
    for h in range(height.max() + 1):
        for p in np.nonzero(height == h)[0]:
            f = front[p]
            m, n = len(f), nk[p]
            F = np.zeros((m, m))
            F[:, :n] = Sp[np.ix_(f, f[:n])]          # original entries in the K columns
            F[:n, :] = F[:, :n].T
            for ch in kids[p]:                      # extend-add of the children's updates
                idx = np.searchsorted(f, S[ch])
                assert np.array_equal(f[idx], S[ch])
                F[np.ix_(idx, idx)] += U[ch]
            Dinv[p] = np.linalg.inv(F[:n, :n])
            Lbar[p] = F[n:, :n] @ Dinv[p]
            U[p] = F[n:, n:] - Lbar[p] @ F[:n, n:]
    q = np.zeros_like(c)
    u = [None] * nn
    for h in range(height.max() + 1):              # forward, by height
        for p in np.nonzero(height == h)[0]:
            f = front[p]
            n = nk[p]
            g = np.concatenate([c[f[:n]], np.zeros(len(f) - n)])
            for ch in kids[p]:
                g[np.searchsorted(f, S[ch])] += u[ch]
            q[f[:n]] = Dinv[p] @ g[:n]
            u[p] = g[n:] - Lbar[p] @ g[:n]
    for d in range(1, depth.max() + 1):            # backward, by depth
        for p in np.nonzero(depth == d)[0]:
            q[k0[p]:k0[p] + nk[p]] -= Lbar[p].T @ q[S[p]]
    return q


@pytest.mark.parametrize("leaf,top", SHAPES + [(2, 0)])
@pytest.mark.parametrize("name", list(CASES))
def test_multifrontal_sweeps_solve_the_coarse_problem(ieti, name, leaf, top):
    t, Sp = _setup(ieti, name, leaf, top)
    c = np.random.default_rng(7).standard_normal(Sp.shape[0])
    q = _multifrontal_solve(t, Sp, c)
    ref = np.linalg.solve(Sp, c)
    assert np.linalg.norm(q - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("name", ["c4_family", "ragged_p23"])
def test_top_merge_forms_one_root_block(ieti, name):
    """coarse_top = 2 moves the first bisection level's separators into the root: fewer
    nodes, a larger last block, the same unknowns."""
    t1, _ = _setup(ieti, name, 1, 1)
    t2, _ = _setup(ieti, name, 1, 2)
    assert len(t2["nk"]) < len(t1["nk"])
    assert t2["nk"][-1] > t1["nk"][-1] and t2["nk"].sum() == t1["nk"].sum()
