"""The multi-GPU path is replicas only: each rank runs its own chains and the ranks meet only in the
benchmark's host-side reductions (barrier, max of the timed milliseconds, sum of the updates).  Two gloo
ranks on the CPU check those reductions and the whole-job value built from them."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(torch, world)
        ms = [1000.0, 2500.0][rank]          # rank 1 is the slowest
        units = [4864, 9728][rank]
        q.put((rank, bench.allreduce_max(torch, world, ms), bench.allreduce_sum(torch, world, units),
               bench.replica_value(torch, world, units, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, total, value in out:
        assert ms_max == 2500.0
        assert total == 4864 + 9728
        assert abs(value - (4864 + 9728) / 2.5) < 1e-9
