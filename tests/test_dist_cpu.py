"""Multi-process (gloo, world_size 2) check of bench.py's replica aggregation, on CPU.

bench.py runs N independent replicas (one per GPU) of the frame; the whole-job
value is the frames of all ranks divided by the slowest rank's time.  The
aggregation uses a MAX all-reduce of each rank's elapsed time; here two CPU
ranks with different timings must agree on the same result.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 100.0 + 50.0 * rank  # rank 1 is slower
    ms, fps = bench.aggregate_replicas(elapsed, steps=10, world=world, device=torch.device("cpu"))
    q.put((rank, ms, fps))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, ms, fps in res:
        assert ms == pytest.approx(150.0)                 # the slowest rank's time
        assert fps == pytest.approx(2 * 10 / 0.150)       # frames of both ranks / that time
