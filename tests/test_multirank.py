"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2).

bench.py --gpus N runs N independent replicas (the filter couples every particle
at each tempering stage, so nothing is sharded); its only multi-rank logic is the
process group, the barrier and the max / sum reductions of the timing, and the
reference arm, which rank 0 alone runs.  The GPU machine runs the same code on NCCL.
"""
import contextlib
import io
import os
import socket
import types

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    r, w = bench.dist_setup()
    out = {"rank": r, "ws": w, "backend": dist.get_backend(),
           "max": bench.reduce_max(float(r) + 1.5, w), "sum": bench.reduce_sum(float(r) + 1.0, w)}
    bench.barrier(w)
    if r != 0:
        # the reference arm: every rank but 0 leaves at once, without work or output
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            out["ref_rc"] = bench.run_reference(types.SimpleNamespace(warmup=3, steps=1))
        out["ref_out"] = buf.getvalue()
    bench.barrier(w)
    dist.destroy_process_group()
    q.put(out)


def test_replica_ranks_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["ws"] == 2 and o["backend"] == "gloo"
        assert o["max"] == 2.5            # the slowest rank's time
        assert o["sum"] == 3.0            # the units every rank processed
    r1 = next(o for o in outs if o["rank"] == 1)
    assert r1["ref_rc"] == 0 and r1["ref_out"] == ""
