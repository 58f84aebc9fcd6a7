"""Host logic of bench.py's multi-GPU path.  The method has no exchange step
between independent problems, so N GPUs run N replicas: one process per GPU,
a barrier around the timed steps, the slowest rank's time and the work of
all ranks.  Two gloo ranks on the CPU check that logic (the solves
themselves need a GPU)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup(world)
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = 10.0 * (r + 1)  # the last rank is the slowest replica
    units = 1.0e6 * (r + 1)
    q.put((r, bench.allreduce_max(ms, w), bench.allreduce_sum(units, w), bench.replica_rate(units, ms, w)))
    bench.barrier(w)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0] * world
    slowest = 10.0 * world
    units = 1.0e6 * world * (world + 1) / 2
    for r, mx, total, rate in out:
        assert mx == slowest and total == units
        assert rate == pytest.approx(units / (slowest * 1e-3) / 1e6)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.allreduce_max(3.5, 1) == 3.5 and bench.allreduce_sum(2.0, 1) == 2.0
    assert bench.replica_rate(2.0e6, 4.0, 1) == pytest.approx(2.0e6 / 4.0e-3 / 1e6)
