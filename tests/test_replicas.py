"""Multi-rank bench path (replicas: one independent problem per rank), run as
two gloo ranks on the CPU: the slowest rank's times decide and the whole-job
throughput counts every rank's iterations."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed 100 (r + 1) ms for 10 steps and 200 (r + 1) ms end to end
    res = bench.combine_ranks(100.0 * (rank + 1), 200.0 * (rank + 1), 10, world, "cpu")
    out[rank] = torch.tensor(res, dtype=torch.float64)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    shared = mgr.list([None] * world)
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, shared)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        total_ms, e2e_ms, value, e2e_value = shared[r].tolist()
        assert total_ms == 200.0 and e2e_ms == 400.0
        assert value == pytest.approx(world * 10 / 0.2)
        assert e2e_value == pytest.approx(world * 10 / 0.4)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(50.0, 80.0, 5, 1) == (50.0, 80.0, 100.0, 62.5)
