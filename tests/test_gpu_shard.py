"""One problem sharded over switching states, emulated on one GPU: the
shards' gradients, each continuing the P^T sum of the previous shard, give
the unsharded gradient bit for bit, and so does the whole sharded FISTA
(gradient, sum, replicated prox and momentum) against the unsharded solve;
a shard's gradient against the oracle on its pulses checks the state offset."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_23739_gb300 as sw
from paper_2510_23739_gb300 import shard
from synth import Geometry, Switching

pytestmark = pytest.mark.gpu

GEOM = Geometry(X=12, Y=10, Z=16, T=40, N=11, P=3, k=5, pulses_per_cycle=4)
SWITCH = Switching((0.4, 0.9, 0.0), (1.0, 1.0, 0.0), (0.05, 0.1, 1.0), 2.5)
RANGES = [(0, 1), (1, 3), (3, 4)]  # uneven shards of the 4 states


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def problem():
    rng = np.random.default_rng(80)
    K = rng.standard_normal(GEOM.k_shape())
    c = np.maximum(rng.standard_normal(GEOM.c_shape()), 0)
    y = oracle.forward(GEOM, SWITCH, K, c) + 0.05 * rng.standard_normal(GEOM.y_shape())
    L = oracle.power(GEOM, SWITCH, K, rng.standard_normal(GEOM.c_shape()), 100)
    return K, y, 1.0 / L


def _pin_tc(op):
    # whole tile-states per CTA and one fixed tiling: each state's sums run
    # in the same order whatever the shard
    for kid in (0, 1):
        op.tc_configure(kid, tiles_per_cta=1, ctas_per_sm=1)
        op.tc_schedule(kid, split=1, buffers=1)


def _ops(K, precision):
    full = sw.Operator(GEOM, K, SWITCH, precision=precision)
    shards = [shard.make_shard(sw.Operator, GEOM, K, SWITCH, m0, m1, precision=precision)
              for m0, m1 in RANGES]
    if precision != "fp32":
        for op in [full] + shards:
            _pin_tc(op)
    return full, shards


def _params(alpha, iters):
    return sw.SolveParams(step=alpha, lambda_l1=2e-3, lambda_tv=3e-3, inner_iters=10,
                          max_iters=iters)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_chained_shard_gradients_are_the_unsharded_gradient(problem, precision):
    K, y, alpha = problem
    full, shards = _ops(K, precision)
    try:
        yd = dev(y)
        full.fista_init(yd, _params(alpha, 5))
        for op, (m0, m1) in zip(shards, RANGES):
            op.fista_init(shard.shard_measurements(yd, GEOM, m0, m1), _params(alpha, 5))
        # a few iterations first, so that the momentum iterate is not zero
        full.fista_step(3)
        for _ in range(3):
            g = None
            for op in shards:
                g = op.fista_gradient(carry=g)
            for op in shards:
                op.fista_step_external(g)
        want = full.fista_gradient()
        got = None
        for op in shards:
            got = op.fista_gradient(carry=got)
        for op in [full] + shards:
            op.check_device()
        assert torch.equal(got, want)
        assert torch.equal(shards[0].fista_get(), full.fista_get())
    finally:
        for op in [full] + shards:
            op.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_emulated_sharded_fista_is_the_unsharded_solve(problem, precision):
    K, y, alpha = problem
    iters = 20
    full, shards = _ops(K, precision)
    try:
        yd = dev(y)
        want, _ = full.solve(yd, _params(alpha, iters))
        for op, (m0, m1) in zip(shards, RANGES):
            op.fista_init(shard.shard_measurements(yd, GEOM, m0, m1), _params(alpha, iters))
        shard.emulate_fista(shards, iters)
        outs = [op.fista_get() for op in shards]
        for op in [full] + shards:
            op.check_device()
        for o in outs:
            assert torch.equal(o, want)
    finally:
        for op in [full] + shards:
            op.close()


def test_shard_gradient_matches_oracle_on_its_pulses(problem):
    """At xi = 0 a shard's gradient is -H_r^T y_r, H_r the rows of H of its
    pulses: the oracle with the full train's S restricted to those pulses."""
    K, y, alpha = problem
    S = oracle.switch_matrix(GEOM, SWITCH)
    for m0, m1 in RANGES:
        op = shard.make_shard(sw.Operator, GEOM, K, SWITCH, m0, m1)
        try:
            yr = shard.shard_measurements(y, GEOM, m0, m1)
            op.fista_init(dev(yr), _params(alpha, 1))
            got = op.fista_gradient().cpu().numpy().astype(np.float64)
            op.check_device()
        finally:
            op.close()
        idx = shard.shard_pulses(GEOM.N, GEOM.pulses_per_cycle, m0, m1)
        want = -oracle.adjoint(shard.shard_geometry(GEOM, m0, m1), SWITCH, K, yr, S=S[idx])
        assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
