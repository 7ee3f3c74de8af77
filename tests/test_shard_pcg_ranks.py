"""The whole preconditioned CG of the dual problem (Sec. 3-4) on patch-sharded ranks,
two and three gloo ranks on CPU, against the serial oracle.

Each rank holds the local operators of its patches only (taken from the oracle's
IETI-DP: the r-block factor, W_rp, Phi, the Dirichlet block S_bb, B_s and B_D,s) and the
multipliers it owns (ieti_shard_plan: the rank of the multiplier's lower patch).  Per
iteration it exchanges exactly what the plan names: the search direction and the
residual on the cut multipliers its patches touch (owner -> peer), its partial jumps of
the cut multipliers (peer -> owner), the coarse right-hand side (a sum over the ranks;
the coarse solve is replicated) and the dot products (sums over the owned multipliers).
The iterates must be the serial PCG's: the same iteration count and lambda within
1e-10, so the sharded layout computes the paper's method and nothing else."""
import os
import socket

import numpy as np
import pytest
import scipy.linalg as sla

from workloads import make_problem, small_problem

CASES = {
    "ragged_p23": lambda: small_problem(P=(4, 3, 2), n_el=((3, 2, 5, 2), (2, 4, 2), (3, 2)),
                                        degree=((2, 3, 2, 2), (3, 2, 2), (2, 3)),
                                        conductor=((0.2, 0.8), (0.3, 0.7), (0.0, 1.0)), sigma=50.0, dt=0.01),
    "c4_family": lambda: make_problem("c4", patches_per_dir=3, el_range=(2, 3)),
}
TOL = 1e-9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _setup(name, world):
    from paper_2510_23446_gb300 import ieti
    from oracle.ietidp import PRECOND_STIFF, local_rhs
    from oracle.stepping import OracleProblem
    prob = CASES[name]()
    S = ieti.Solver.from_problem(prob, device=-1)
    rop = S.shard_plan(world)["rank_of_patch"]
    S.close()
    op = OracleProblem(prob)
    I = op.ietidp(PRECOND_STIFF)
    d, _ = I.rhs(local_rhs(op.dec, np.zeros(op.asm.lat.n_edges), op.asm.j_global))
    return op, I, d, rop


def _rank_main(rank, world, port, name, out_q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        op, I, d, rop = _setup(name, world)
        dec = op.dec
        lam = dec.lam                                    # (edge, s, pos_s, t, pos_t), s < t
        m = dec.m
        lo = np.array([x[1] for x in lam])
        hi = np.array([x[3] for x in lam])
        owner = rop[lo]
        peer = np.where(rop[hi] != owner, rop[hi], -1)
        own = owner == rank
        mine = [s for s in range(dec.n_patches) if rop[s] == rank]
        touch = np.zeros(m, dtype=bool)                 # multipliers this rank's patches touch
        touch[(rop[lo] == rank) | (rop[hi] == rank)] = True

        def to_peers(v):
            """owner -> peer: the values of the cut multipliers a peer's patches touch."""
            v = np.where(own, v, 0.0)
            for other in range(world):
                if other == rank:
                    continue
                send = np.nonzero(own & (peer == other))[0]
                recv = np.nonzero((owner == other) & (peer == rank))[0]
                ops = []
                if len(send):
                    ops.append(dist.P2POp(dist.isend, torch.from_numpy(v[send].copy()), other))
                rb = torch.zeros(len(recv), dtype=torch.float64)
                if len(recv):
                    ops.append(dist.P2POp(dist.irecv, rb, other))
                for w in dist.batch_isend_irecv(ops) if ops else []:
                    w.wait()
                v[recv] = rb.numpy()
            return v

        def to_owners(part):
            """peer -> owner: partial jumps of the cut multipliers, summed at the owner."""
            part = part.copy()
            for other in range(world):
                if other == rank:
                    continue
                send = np.nonzero((owner == other) & (peer == rank))[0]
                recv = np.nonzero(own & (peer == other))[0]
                ops = []
                if len(send):
                    ops.append(dist.P2POp(dist.isend, torch.from_numpy(part[send].copy()), other))
                rb = torch.zeros(len(recv), dtype=torch.float64)
                if len(recv):
                    ops.append(dist.P2POp(dist.irecv, rb, other))
                for w in dist.batch_isend_irecv(ops) if ops else []:
                    w.wait()
                part[recv] += rb.numpy()
            return np.where(own, part, 0.0)

        def allsum(x):
            t = torch.from_numpy(np.atleast_1d(np.asarray(x, dtype=np.float64)).copy())
            dist.all_reduce(t)
            return t.numpy()

        def apply_F(p_own):
            p = to_peers(p_own)
            xs, c = {}, np.zeros(dec.n_coarse)
            for s in mine:
                x = sla.cho_solve(I.Wrr_f[s], I._BT(s, p))
                xs[s] = x
                np.add.at(c, dec.A[s], I.Wrp[s].T @ x)
            qc = I._coarse_solve(allsum(c)) if dec.n_coarse else c
            part = np.zeros(m)
            for s in mine:
                part += I._B(s, xs[s] + I.Phi[s] @ qc[dec.A[s]])
            return to_owners(part)

        def apply_M(r_own):
            r = to_peers(r_own)
            part = np.zeros(m)
            for s in mine:
                part += I.BD[s] @ (I.Wbb_S[s] @ (I.BD[s].T @ r))
            return to_owners(part)

        dot = lambda a, b: float(allsum(float(np.dot(a[own], b[own])))[0])   # noqa: E731
        # the serial PCG of the oracle, on owned multipliers
        tol = 1e-10
        lam_v = np.zeros(m)
        r = np.where(own, d, 0.0)
        nd = np.sqrt(dot(r, r))
        z = apply_M(r)
        p = z.copy()
        rz = dot(r, z)
        it = 0
        while it < 5000:
            q = apply_F(p)
            alpha = rz / dot(p, q)
            lam_v += alpha * p
            r -= alpha * q
            it += 1
            if np.sqrt(dot(r, r)) / nd <= tol:
                break
            z = apply_M(r)
            rz_new = dot(r, z)
            p = z + rz_new / rz * p
            rz = rz_new
        out_q.put((rank, np.nonzero(own)[0], lam_v[own], it, int(touch.sum())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", list(CASES))
def test_sharded_pcg_equals_serial(name, world):
    pytest.importorskip("torch")
    try:
        from paper_2510_23446_gb300 import ieti  # noqa: F401
    except Exception as e:   # noqa: BLE001
        pytest.skip(f"library not built: {e}")
    import torch.multiprocessing as mp
    op, I, d, rop = _setup(name, world)
    lam_ref, it_ref, _ = I.pcg(d, 1e-10)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    lam = np.full(len(d), np.nan)
    for rank, idx, vals, it, n_touch in res:
        assert it == it_ref, (rank, it, it_ref)
        assert np.all(np.isnan(lam[idx]))             # every multiplier owned once
        lam[idx] = vals
        assert n_touch < len(d)                        # a rank sees only part of the multipliers
    assert not np.isnan(lam).any()
    assert np.linalg.norm(lam - lam_ref) <= TOL * np.linalg.norm(lam_ref)
