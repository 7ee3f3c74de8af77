"""Patch-sharded layout of the dual-primal solve (Sec. 3: independent patch problems
coupled through the multiplier jumps, the coarse right-hand side and the PCG dot
products), exercised by two and three gloo ranks on CPU.

Each rank holds only its patches' interface and primal copies (seeded per global copy,
so that the ranks agree on the values).  With the library's plan (ieti_shard_plan) a
rank computes its partial jumps of the multipliers it touches, sends the partials of the
cut multipliers to their owners (one exchange per peer, in ascending multiplier order on
both sides), sums the coarse right-hand side over the ranks holding copies, and reduces
the owned multipliers' dot product.  The results must equal the single-process values
computed from all copies; every multiplier and coarse unknown must have exactly one
owner, and the partition must be balanced."""
import os
import socket

import numpy as np
import pytest

from workloads import small_problem, make_problem

CASES = {
    "ragged_p23": lambda: small_problem(P=(4, 3, 2), n_el=((3, 2, 5, 2), (2, 4, 2), (3, 2)),
                                        degree=((2, 3, 2, 2), (3, 2, 2), (2, 3)),
                                        conductor=((0.2, 0.8), (0.3, 0.7), (0.0, 1.0)), sigma=50.0, dt=0.01),
    "c4_family": lambda: make_problem("c4", patches_per_dir=3, el_range=(2, 3)),
}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _structure(name, n_ranks):
    from paper_2510_23446_gb300 import ieti
    prob = CASES[name]()
    S = ieti.Solver.from_problem(prob, device=-1)
    out = dict(plan=S.shard_plan(n_ranks), lam=S.multipliers(), blk=S.patch_blocks(), n_coarse=S.info()["n_coarse"])
    S.close()
    return out


def _copy_values(blk, seed):
    """Per patch: seeded interface-copy values u_s and primal-copy values v_s (by global copy index)."""
    nb, np_ = blk["nb"], blk["np"]
    rng = np.random.default_rng(seed)
    ub = rng.standard_normal(int(nb.sum()))
    vp = rng.standard_normal(int(np_.sum()))
    bo = np.concatenate([[0], np.cumsum(nb)])
    po = np.concatenate([[0], np.cumsum(np_)])
    return [ub[bo[s]:bo[s + 1]] for s in range(len(nb))], [vp[po[s]:po[s + 1]] for s in range(len(np_))], po


def _rank_main(rank, world, port, name, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st = _structure(name, world)
        plan, lam, blk = st["plan"], st["lam"], st["blk"]
        mine = plan["rank_of_patch"] == rank
        u, v, po = _copy_values(blk, 11)
        m = len(lam["s"])
        # partial jumps of every multiplier this rank touches (+copy in s, -copy in t)
        part = np.zeros(m)
        for l in range(m):
            if mine[lam["s"][l]]:
                part[l] += u[lam["s"][l]][lam["pos_s"][l]]
            if mine[lam["t"][l]]:
                part[l] -= u[lam["t"][l]][lam["pos_t"][l]]
        # cut multipliers: the non-owner sends its partials to the owner, one exchange per
        # peer, ascending multiplier ids on both sides
        own = plan["lam_owner"] == rank
        for peer in range(world):
            if peer == rank:
                continue
            send = np.nonzero((plan["lam_owner"] == peer) & (plan["lam_peer"] == rank))[0]
            recv = np.nonzero(own & (plan["lam_peer"] == peer))[0]
            ops = []
            if len(send):
                ops.append(dist.P2POp(dist.isend, torch.from_numpy(part[send].copy()), peer))
            rb = torch.zeros(len(recv), dtype=torch.float64)
            if len(recv):
                ops.append(dist.P2POp(dist.irecv, rb, peer))
            for w in dist.batch_isend_irecv(ops) if ops else []:
                w.wait()
            part[recv] += rb.numpy()
        jump = np.where(own, part, 0.0)
        # coarse right-hand side: sum over the copies this rank holds, reduced over ranks
        c = np.zeros(st["n_coarse"])
        for s in np.nonzero(mine)[0]:
            np.add.at(c, blk["coarse_of_copy"][po[s]:po[s + 1]], v[s])
        ct = torch.from_numpy(c)
        dist.all_reduce(ct)
        # dot product over the owned multipliers
        dt = torch.tensor([float(jump @ jump)], dtype=torch.float64)
        dist.all_reduce(dt)
        q.put((rank, jump, ct.numpy(), float(dt.item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", list(CASES))
def test_sharded_exchange_reproduces_the_serial_quantities(name, world):
    pytest.importorskip("torch")
    try:
        from paper_2510_23446_gb300 import ieti  # noqa: F401
    except Exception as e:   # noqa: BLE001
        pytest.skip(f"library not built: {e}")
    import torch.multiprocessing as mp
    st = _structure(name, world)
    plan, lam, blk = st["plan"], st["lam"], st["blk"]
    u, v, po = _copy_values(blk, 11)
    m = len(lam["s"])
    ref_jump = np.array([u[lam["s"][l]][lam["pos_s"][l]] - u[lam["t"][l]][lam["pos_t"][l]] for l in range(m)])
    ref_c = np.zeros(st["n_coarse"])
    for s in range(len(blk["nb"])):
        np.add.at(ref_c, blk["coarse_of_copy"][po[s]:po[s + 1]], v[s])
    # every patch on one rank, every rank some patches, the cut crosses some multipliers
    assert set(np.unique(plan["rank_of_patch"])) == set(range(world))
    assert np.array_equal(plan["lam_owner"], plan["rank_of_patch"][lam["s"]])
    cut = plan["lam_peer"] >= 0
    assert cut.any() and np.all(plan["lam_peer"][cut] == plan["rank_of_patch"][lam["t"]][cut])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    jump = np.zeros(m)
    for rank, j, c, dot in res:
        jump += j                                    # each multiplier completed by its owner only
        assert np.allclose(c, ref_c, rtol=0, atol=1e-12)
        assert abs(dot - ref_jump @ ref_jump) <= 1e-12 * (ref_jump @ ref_jump)
    assert np.allclose(jump, ref_jump, rtol=0, atol=1e-12)


def test_shard_plan_is_balanced():
    try:
        from paper_2510_23446_gb300 import ieti
    except Exception as e:   # noqa: BLE001
        pytest.skip(f"library not built: {e}")
    prob = make_problem("c2")
    S = ieti.Solver.from_problem(prob, device=-1)
    blk = S.patch_blocks()
    w = (blk["ni"] + blk["nb"] + blk["np"]).astype(float)
    for n in (2, 4, 8):
        plan = S.shard_plan(n)
        load = np.bincount(plan["rank_of_patch"], weights=w, minlength=n)
        assert load.min() > 0 and load.max() / load.mean() < 1.35, (n, load)
    with pytest.raises(ieti.IetiError):
        S.shard_plan(0)
    S.close()
