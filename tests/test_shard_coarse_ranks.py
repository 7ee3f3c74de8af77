"""The coarse solve on the patch-sharded ranks (Sec. 3: the primal Schur complement
S_c, factored along the nested dissection of the patch grid), with two and three gloo
ranks on CPU.

With the library's node owners (ieti_shard_coarse) a rank factors and solves the nodes
it owns (whole subtrees), the ranks sum their owned subtrees' contributions into the
shared top fronts (one allreduce of update matrices at setup, one of update vectors per
solve), every rank factors and solves the shared top, and each rank finishes the
backward sweep of its own subtrees.  The algebra is the multifrontal sweep of
tests/test_coarse_tree.py (the device algorithm in numpy) on the library's tree; S_c
comes from the oracle.  Each rank's coarse values (its owned nodes and the shared top)
must equal numpy's dense solve, and together the ranks must cover every unknown."""
import os
import socket

import numpy as np
import pytest

from test_coarse_tree import CASES, _nodes

NAMES = ["c4_family", "ragged_p23"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem(name, world, aligned=False):
    from paper_2510_23446_gb300 import ieti
    from oracle.stepping import OracleProblem
    prob = CASES[name]()
    I = OracleProblem(prob).ietidp()
    prim = np.nonzero(I.dec.gauge.cls == 1)[0]
    S = ieti.Solver.from_problem(prob, device=-1, coarse_leaf=1, coarse_ranks=world if aligned else 0)
    t = S.coarse_tree()
    nr = S.shard_coarse(world)
    S.close()
    pos = t["elim_pos"][prim]
    Sp = np.zeros_like(I.Sc)
    Sp[np.ix_(pos, pos)] = I.Sc
    return t, nr, Sp


def _rank_main(rank, world, port, name, aligned, out_q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, nr, Sp = _problem(name, world, aligned)
        nn, S, kids = _nodes(t)
        k0, nk = t["k0"], t["nk"]
        front = [np.concatenate([np.arange(k0[p], k0[p] + nk[p]), S[p]]) for p in range(nn)]
        depth = np.zeros(nn, dtype=int)
        for p in range(nn - 1, -1, -1):
            depth[p] = 0 if t["parent"][p] < 0 else depth[t["parent"][p]] + 1
        mine = [p for p in range(nn) if nr[p] == rank]            # postorder
        shared = [p for p in range(nn) if nr[p] < 0]
        Dinv, Lbar, U = {}, {}, {}

        def factor(p, extra):
            f, n = front[p], nk[p]
            F = np.zeros((len(f), len(f)))
            F[:, :n] = Sp[np.ix_(f, f[:n])]
            F[:n, :] = F[:, :n].T
            F += extra
            for ch in kids[p]:
                if ch in U:
                    idx = np.searchsorted(f, S[ch])
                    F[np.ix_(idx, idx)] += U[ch]
            Dinv[p] = np.linalg.inv(F[:n, :n])
            Lbar[p] = F[n:, :n] @ Dinv[p]
            U[p] = F[n:, n:] - Lbar[p] @ F[:n, n:]

        def allreduce(parts):
            flat = torch.from_numpy(np.concatenate([x.ravel() for x in parts]) if parts else np.zeros(0))
            dist.all_reduce(flat)
            out, o = [], 0
            for x in parts:
                out.append(flat[o:o + x.size].numpy().reshape(x.shape))
                o += x.size
            return out

        # setup: owned subtrees, then their update matrices summed into the shared fronts
        for p in mine:
            factor(p, 0.0)
        parts = []
        for p in shared:
            G = np.zeros((len(front[p]), len(front[p])))
            for ch in kids[p]:
                if nr[ch] == rank:
                    idx = np.searchsorted(front[p], S[ch])
                    G[np.ix_(idx, idx)] += U[ch]
            parts.append(G)
        to_shared = lambda x: t["parent"][x] >= 0 and nr[t["parent"][x]] < 0   # noqa: E731
        for ch in [x for x in U if to_shared(x)]:
            del U[ch]                                 # now inside the summed shared fronts
        for p, G in zip(shared, allreduce(parts)):
            factor(p, G)
        # one solve
        c = np.random.default_rng(7).standard_normal(Sp.shape[0])
        q = np.full(Sp.shape[0], np.nan)
        u = {}

        def forward(p, extra):
            f, n = front[p], nk[p]
            g = np.concatenate([c[f[:n]], np.zeros(len(f) - n)]) + extra
            for ch in kids[p]:
                if ch in u:  # the owned children of a shared node are in `extra` already
                    g[np.searchsorted(f, S[ch])] += u[ch]
            q[f[:n]] = Dinv[p] @ g[:n]
            u[p] = g[n:] - Lbar[p] @ g[:n]

        for p in mine:
            forward(p, 0.0)
        parts = []
        for p in shared:
            g = np.zeros(len(front[p]))
            for ch in kids[p]:
                if nr[ch] == rank:
                    g[np.searchsorted(front[p], S[ch])] += u[ch]
            parts.append(g)
        sums = allreduce(parts)
        for ch in [x for x in u if to_shared(x)]:
            del u[ch]                                 # now inside the summed shared fronts
        for p, g in zip(shared, sums):
            forward(p, g)
        for p in sorted(shared, key=lambda x: depth[x]) + sorted(mine, key=lambda x: depth[x]):
            if t["parent"][p] >= 0:
                q[k0[p]:k0[p] + nk[p]] -= Lbar[p].T @ q[S[p]]
        known = np.concatenate([np.arange(k0[p], k0[p] + nk[p]) for p in mine + shared]) if mine + shared \
            else np.zeros(0, dtype=int)
        out_q.put((rank, known, q[known], [int(p) for p in mine]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("aligned", [False, True])
@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", NAMES)
def test_sharded_coarse_solve_equals_dense(name, world, aligned):
    """aligned: the tree cut where the plan cuts the patch grid (option coarse_ranks)."""
    pytest.importorskip("torch")
    try:
        from paper_2510_23446_gb300 import ieti  # noqa: F401
    except Exception as e:   # noqa: BLE001
        pytest.skip(f"library not built: {e}")
    import torch.multiprocessing as mp
    t, nr, Sp = _problem(name, world, aligned)
    nn = len(t["k0"])
    par = t["parent"]
    # ownership: whole subtrees per rank, a shared top, every rank owning something
    assert all(nr[par[p]] < 0 or nr[par[p]] == nr[p] for p in range(nn) if par[p] >= 0)
    assert all(nr[par[p]] < 0 for p in range(nn) if par[p] >= 0 and nr[p] < 0)
    assert set(nr[nr >= 0]) == set(range(world)) and (nr < 0).any()
    ref = np.linalg.solve(Sp, np.random.default_rng(7).standard_normal(Sp.shape[0]))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, aligned, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    covered = np.zeros(Sp.shape[0], dtype=int)
    owned = []
    for rank, known, vals, mine in res:
        assert np.linalg.norm(vals - ref[known]) <= 1e-10 * np.linalg.norm(ref), rank
        covered[known] += 1
        owned += mine
    assert np.all(covered >= 1)
    assert sorted(owned) == sorted(int(p) for p in np.nonzero(nr >= 0)[0])   # each owned node on one rank


@pytest.mark.parametrize("name", NAMES)
def test_aligned_tree_shrinks_the_shared_top(name):
    """Cutting the tree where the ranks are cut leaves no more shared bytes than the
    midpoint tree, the same unknowns, and a shared top of only rank-spanning boxes."""
    try:
        from paper_2510_23446_gb300 import ieti
    except Exception as e:   # noqa: BLE001
        pytest.skip(f"library not built: {e}")
    prob = CASES[name]()

    def shared_bytes(world, aligned):
        S = ieti.Solver.from_problem(prob, device=-1, coarse_leaf=1, coarse_ranks=world if aligned else 0)
        t = S.coarse_tree()
        nr = S.shard_coarse(world)
        S.close()
        nk, ns = t["nk"], np.diff(t["s_off"])
        byt = 8.0 * ((nk + ns) * nk + nk * ns)
        return byt[nr < 0].sum(), int(nk.sum())

    for world in (2, 3, 4):
        (b0, n0), (b1, n1) = shared_bytes(world, False), shared_bytes(world, True)
        assert n0 == n1 and b1 <= b0 * (1 + 1e-12), (world, b0, b1)
