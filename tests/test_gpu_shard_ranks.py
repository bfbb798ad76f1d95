"""The sharded solve across processes: two ranks (gloo, 127.0.0.1) on one
GPU, each a handle over its switching states, step ShardedFista (gradient,
all_reduce of the gradient on the host, replicated prox and momentum); their
iterates match the unsharded solve.  The ranks never wait on each other inside
a kernel: the exchange is gloo's host-side sum between launches."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from synth import Geometry, Switching
    import oracle
    g = Geometry(X=12, Y=10, Z=16, T=40, N=11, P=3, k=5, pulses_per_cycle=4)
    sw = Switching((0.4, 0.9, 0.0), (1.0, 1.0, 0.0), (0.05, 0.1, 1.0), 2.5)
    rng = np.random.default_rng(81)
    K = rng.standard_normal(g.k_shape())
    c = np.maximum(rng.standard_normal(g.c_shape()), 0)
    y = oracle.forward(g, sw, K, c) + 0.05 * rng.standard_normal(g.y_shape())
    L = oracle.power(g, sw, K, rng.standard_normal(g.c_shape()), 100)
    return g, sw, K, y, 1.0 / L


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2510_23739_gb300 as swl
    from paper_2510_23739_gb300 import shard
    g, sw, K, y, alpha = _problem()
    m0, m1 = shard.state_ranges(min(g.N, g.pulses_per_cycle), world)[rank]
    op = shard.make_shard(swl.Operator, g, K, sw, m0, m1)
    yd = torch.tensor(shard.shard_measurements(y, g, m0, m1), dtype=torch.float32,
                      device="cuda")
    prm = swl.SolveParams(step=alpha, lambda_l1=2e-3, lambda_tv=3e-3, inner_iters=10,
                          max_iters=15)
    op.fista_init(yd, prm)
    runner = shard.ShardedFista(op)
    runner.step(15)
    c = op.fista_get().cpu().numpy()
    op.check_device()
    op.close()
    out[rank] = torch.tensor(c)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_match_the_unsharded_solve():
    import paper_2510_23739_gb300 as swl
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    shared = mgr.list([None] * world)
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, shared)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    g, sw, K, y, alpha = _problem()
    op = swl.Operator(g, K, sw)
    try:
        want, _ = op.solve(torch.tensor(y, dtype=torch.float32, device="cuda"),
                           swl.SolveParams(step=alpha, lambda_l1=2e-3, lambda_tv=3e-3,
                                           inner_iters=10, max_iters=15))
        want = want.cpu().numpy().astype(np.float64)
    finally:
        op.close()
    c0, c1 = shared[0].numpy(), shared[1].numpy()
    assert np.array_equal(c0, c1)  # both replicas took the same summed gradients
    assert np.linalg.norm(c0 - want) <= 1e-5 * np.linalg.norm(want)
