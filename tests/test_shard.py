"""The particle-sharded exchange of a tempering stage (Sec. 3.1.4's ensemble parallelism)
on CPU ranks: gloo, world sizes 2 and 4.

Given fixed weights, the offspring indices come from the oracle's systematic resampling
(the same on every rank); each rank then holds its block of particles, and the routing
plan with its point-to-point exchange must give every rank exactly the rows that the
one-rank gather (row i <- row idx[i]) puts in its block, bit for bit, for arrays of
several shapes and types.  The all-gather of the weights must reproduce the whole
ensemble's nll and log G in particle order.
"""
import os
import socket

import numpy as np
import torch
import torch.multiprocessing as mp

from oracle import filter as OF


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ensemble(N, seed):
    r = np.random.default_rng(seed)
    # a few heavy particles, so that most offspring cross ranks
    w = r.gamma(0.2, size=N)
    w /= w.sum()
    m = torch.tensor(r.normal(size=(N, 12)), dtype=torch.float32)
    dW = torch.tensor(r.normal(size=(N, 3, 4)), dtype=torch.float64)
    nll = torch.tensor(r.gamma(2.0, size=N), dtype=torch.float64)
    logG = torch.tensor(r.normal(size=N), dtype=torch.float64)
    idx = torch.tensor(OF.systematic_resample(w, OF.resample_offset(7, 3)), dtype=torch.int64)
    return m, dW, nll, logG, idx


def _rank(rank, ws, port, N, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_2402_06927_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    m, dW, nll, logG, idx = _ensemble(N, 11)
    B = N // ws
    blk = slice(rank * B, (rank + 1) * B)
    gn, gl = shard.allgather_weights(nll[blk].contiguous(), logG[blk].contiguous())
    plan = shard.routing_plan(idx, ws, rank)
    new = shard.exchange_rows(plan, [m[blk].contiguous(), dW[blk].contiguous(), nll[blk].contiguous()])
    moved = sum(v.numel() for v in plan.recv.values())
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, gn.numpy(), gl.numpy(), [t.numpy() for t in new], moved))


def _run(ws, N):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, N, q)) for r in range(ws)]
    for p in procs:
        p.start()
    outs = sorted((q.get(timeout=300) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return outs


def test_two_and_four_rank_exchange_equals_one_rank_gather():
    for ws, N in ((2, 16), (4, 64)):
        m, dW, nll, logG, idx = _ensemble(N, 11)
        ref = [m[idx], dW[idx], nll[idx]]
        outs = _run(ws, N)
        B = N // ws
        crossed = 0
        for rank, gn, gl, new, moved in outs:
            assert np.array_equal(gn, nll.numpy()) and np.array_equal(gl, logG.numpy())
            for a, r in zip(new, ref):
                assert np.array_equal(a, r[rank * B:(rank + 1) * B].numpy())
            crossed += moved
        # the case exercises rows that cross ranks as well as local ones
        assert 0 < crossed < N


def test_routing_plan_covers_every_row_once():
    # host logic alone: the plans of all ranks move every new row exactly once, and what
    # rank p sends to rank q is what q receives from p, in the same order
    from paper_2402_06927_gb300 import shard
    for ws, N, seed in ((2, 10, 1), (3, 12, 2), (4, 64, 3), (8, 64, 4)):
        _, _, _, _, idx = _ensemble(N, seed)
        B = N // ws
        plans = [shard.routing_plan(idx, ws, r) for r in range(ws)]
        for r, p in enumerate(plans):
            dst = torch.cat([p.local_dst] + [p.recv[q] for q in sorted(p.recv)])
            assert sorted(dst.tolist()) == list(range(B))
            assert torch.equal(idx[r * B:(r + 1) * B][p.local_dst], p.local_src + r * B)
            for q, rows in p.recv.items():
                assert torch.equal(plans[q].send[r] + q * B, idx[r * B:(r + 1) * B][rows])
