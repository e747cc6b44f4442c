"""Particle-sharded filter across ranks (Sec. 3.1.4's ensemble parallelism, one GPU per
rank): the host logic of the exchange that a tempering stage needs.

Rank r of R holds the B = N / R particles r B .. (r + 1) B - 1 of the ensemble.  Every
step of the cycle that is per particle (the forecast window, the likelihood, PCN
jittering, nudging) runs on the rank's own block.  A tempering stage couples the
particles through their weights only, so its exchange is:

1. an all-gather of every particle's negative log-weight terms (nll and log G, FP64),
   so that every rank holds the whole ensemble's phi = nll - log G;
2. the same tempering search and the same systematic resampling on every rank (the
   kernels are deterministic and take the same inputs, the resampling the same uniform),
   so that every rank holds the same offspring indices idx [N];
3. the row moves: new particle i takes the rows of particle idx[i].  Rows whose parent
   lives on the same rank are gathered locally; the others are sent by the parent's
   rank and received by the child's, with point-to-point copies (NCCL send/recv on GPU
   ranks, gloo on CPU ranks).

``routing_plan`` turns idx into this rank's local gathers, sends and receives, and
``exchange_rows`` performs them for any number of arrays with rows on the first axis.
The plan is a pure function of idx, N, R and the rank, so every rank computes its own
part of the same global permutation without a further exchange.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Sequence

import torch


@dataclass
class RoutingPlan:
    """The row moves of one rank for one resampling.

    local_dst, local_src: new local row local_dst[k] takes old local row local_src[k];
    send[q]: old local rows (in order) that rank q receives from this rank;
    recv[q]: new local rows (in the same order) that take the rows rank q sends."""
    rank: int
    block: int
    local_dst: torch.Tensor
    local_src: torch.Tensor
    send: Dict[int, torch.Tensor] = field(default_factory=dict)
    recv: Dict[int, torch.Tensor] = field(default_factory=dict)


def routing_plan(idx: torch.Tensor, world: int, rank: int) -> RoutingPlan:
    """Plan of rank ``rank`` for offspring indices idx [N] (global, int) with N = B world."""
    idx = idx.to("cpu", torch.int64)
    N = idx.numel()
    if N % world:
        raise ValueError("the ensemble must split evenly across the ranks")
    B = N // world
    owner = idx // B
    mine = slice(rank * B, (rank + 1) * B)
    dst_all = torch.arange(B, dtype=torch.int64)
    own = owner[mine]
    loc = own == rank
    plan = RoutingPlan(rank, B, dst_all[loc], idx[mine][loc] - rank * B)
    for q in range(world):
        if q == rank:
            continue
        # rows of rank q's new block whose parents are mine, in q's row order
        q_idx = idx[q * B:(q + 1) * B]
        from_me = (q_idx // B) == rank
        if bool(from_me.any()):
            plan.send[q] = q_idx[from_me] - rank * B
        # rows of my new block whose parents live on rank q, in my row order
        from_q = own == q
        if bool(from_q.any()):
            plan.recv[q] = dst_all[from_q]
    return plan


def exchange_rows(plan: RoutingPlan, arrays: Sequence[torch.Tensor], group=None) -> List[torch.Tensor]:
    """New local arrays after the resampling of ``plan``: every array [B, ...] gathered
    locally where the parent is local and exchanged point to point where it is not.  All
    sends and receives of all arrays are posted at once (torch.distributed P2P ops)."""
    import torch.distributed as dist
    out = [torch.empty_like(a) for a in arrays]
    dev = arrays[0].device if arrays else torch.device("cpu")
    ld = plan.local_dst.to(dev)
    ls = plan.local_src.to(dev)
    for a, o in zip(arrays, out):
        o[ld] = a[ls]
    ops, bufs = [], []
    for q, rows in sorted(plan.send.items()):
        r = rows.to(dev)
        for a in arrays:
            sb = a[r].contiguous()
            bufs.append(sb)
            ops.append(dist.P2POp(dist.isend, sb, q, group))
    recv_bufs = []
    for q, rows in sorted(plan.recv.items()):
        for a in arrays:
            rb = torch.empty((rows.numel(),) + tuple(a.shape[1:]), dtype=a.dtype, device=dev)
            recv_bufs.append((q, rb))
            ops.append(dist.P2POp(dist.irecv, rb, q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    k = 0
    for q, rows in sorted(plan.recv.items()):
        r = rows.to(dev)
        for o in out:
            o[r] = recv_bufs[k][1]
            k += 1
    return out


def allgather_weights(nll: torch.Tensor, logG: torch.Tensor, group=None):
    """(nll, logG) of the whole ensemble on every rank, in rank order (FP64 all-gather)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    both = torch.stack([nll, logG])
    parts = [torch.empty_like(both) for _ in range(world)]
    dist.all_gather(parts, both, group=group)
    full = torch.cat(parts, dim=1)
    return full[0].contiguous(), full[1].contiguous()
