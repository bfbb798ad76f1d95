"""Sharding one problem over switching states, host side: the state
partition, the pulses of a shard and their local cycle structure, and two
gloo ranks on the CPU whose partial data-fit gradients (each from the oracle
on its shard's pulses) sum over an all-reduce to the oracle's full gradient."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2510_23739_gb300 import shard
from synth import Geometry, Switching

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("states,world", [(10, 1), (10, 2), (10, 3), (8, 8), (3, 2), (60, 7)])
def test_state_ranges_partition_the_states(states, world):
    rs = shard.state_ranges(states, world)
    assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == states
    assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
    sizes = [m1 - m0 for m0, m1 in rs]
    assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.state_ranges(states, states + 1)


@pytest.mark.parametrize("N,ncyc,world", [(60, 10, 2), (11, 4, 3), (8, 3, 2), (5, 8, 2), (7, 7, 7)])
def test_shard_pulses_cover_the_train_once_with_their_states(N, ncyc, world):
    Q = min(N, ncyc)
    seen = []
    for m0, m1 in shard.state_ranges(Q, world):
        idx = shard.shard_pulses(N, ncyc, m0, m1)
        seen.extend(idx.tolist())
        # local pulse i is state m0 + (i mod (m1 - m0)): the shard's own cycle
        assert np.array_equal(idx % ncyc, m0 + np.arange(idx.size) % (m1 - m0))
        assert np.all(np.diff(idx) > 0)
        g = shard.shard_geometry(Geometry(X=4, Y=4, Z=4, T=8, N=N, P=2, k=3,
                                          pulses_per_cycle=ncyc), m0, m1)
        assert (g.N, g.pulses_per_cycle) == (idx.size, m1 - m0)
    assert sorted(seen) == list(range(N))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    g = Geometry(X=6, Y=5, Z=7, T=12, N=11, P=3, k=3, pulses_per_cycle=4)
    sw = Switching((0.4, 0.9, 0.0), (1.0, 1.0, 0.0), (0.05, 0.1, 1.0), 2.5)
    rng = np.random.default_rng(70)
    K = rng.standard_normal(g.k_shape())
    c = rng.random(g.c_shape())
    y = rng.standard_normal(g.y_shape())
    return g, sw, K, c, y


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    g, sw, K, c, y = _problem()
    S = oracle.switch_matrix(g, sw)
    m0, m1 = shard.state_ranges(min(g.N, g.pulses_per_cycle), world)[rank]
    idx = shard.shard_pulses(g.N, g.pulses_per_cycle, m0, m1)
    gr = shard.shard_geometry(g, m0, m1)
    yr = shard.shard_measurements(y, g, m0, m1)
    Sr = S[idx]
    resid = oracle.forward(gr, sw, K, c, S=Sr) - yr
    part = torch.tensor(oracle.adjoint(gr, sw, K, resid, S=Sr))
    dist.all_reduce(part, op=dist.ReduceOp.SUM)
    out[rank] = part
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_sum_partial_gradients_to_the_full_gradient(world):
    import oracle
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    shared = mgr.list([None] * world)
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, shared)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    g, sw, K, c, y = _problem()
    want = oracle.adjoint(g, sw, K, oracle.forward(g, sw, K, c) - y)
    for r in range(world):
        got = shared[r].numpy()
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
