"""The N > 1 path of bench.py on CPU: independent replicas under torch.distributed (gloo,
world size 2).  The whole-job figures are the slowest rank's time and the sum of the units all
ranks processed; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 1.5 (r + 1) seconds, 100 (r + 1) units
        t, u = bench.aggregate(dist, 1.5 * (rank + 1), 100.0 * (rank + 1), "cpu")
        out.put((rank, t, u))
        # the reference arm: only rank 0 works and prints
        class A:
            workload = "c0"
            ref_iters = 3
            warmup = 0
            steps = 1
            gpus = world
        import io
        import contextlib
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(A, rank, world)
        out.put((rank, "ref", buf.getvalue().strip().startswith("{")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_replicas_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = [q.get(timeout=5) for _ in range(4)]
    agg = {r: (t, u) for r, t, u in got if t != "ref"}
    ref = {r: printed for r, tag, printed in got if tag == "ref"}
    assert agg[0] == agg[1] == (3.0, 300.0)
    assert ref == {0: True, 1: False}
