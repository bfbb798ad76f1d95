"""One problem sharded over switching states (host-side bookkeeping).

The measurement operator is block diagonal over pulses (Eq.
(acoustic-full-forward)), and pulses at the same position in their
OFF-switching cycle share one switching state (Eq. (final-H)), so the
data-fit gradient H^T (H c - y) is a sum over states of independent terms.
A shard takes the states [m0, m1): all pulses n with n mod pulses_per_cycle
in that range, in cycle-major order, on a handle whose geometry has
pulses_per_cycle = m1 - m0 and N = their count, and whose state offset is m0.
Each shard computes its part of the gradient at the (replicated) momentum
iterate; one sum over shards (an all-reduce of P Z S values) gives the
gradient, and every shard then applies the same gradient step, prox and
momentum to its replica.

``emulate_fista`` runs the shards one after another on one GPU, each
gradient continuing the P^T sum of the previous shard (swopt_fista_gradient's
carry), which reproduces the unsharded gradient's bits.  ``ShardedFista``
runs one shard per rank with ``torch.distributed.all_reduce`` as the sum
(the collective's order of addition decides the last bits there).
"""
from __future__ import annotations

import copy
import dataclasses

import numpy as np


def state_ranges(states: int, world: int):
    """Contiguous ranges [m0, m1) of the states for ``world`` shards, sizes
    differing by at most one (every state costs the same A and A^T work)."""
    if states < 1 or world < 1:
        raise ValueError("need at least one state and one shard")
    if world > states:
        raise ValueError(f"{world} shards for {states} switching states")
    base, extra = divmod(states, world)
    out, m = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((m, m + n))
        m += n
    return out


def shard_pulses(N: int, pulses_per_cycle: int, m0: int, m1: int) -> np.ndarray:
    """Global indices of the pulses of states [m0, m1), cycle-major: local
    pulse i of the shard is state m0 + (i mod (m1 - m0)) of the train."""
    if not (0 <= m0 < m1 <= min(N, pulses_per_cycle)):
        raise ValueError(f"state range [{m0}, {m1}) outside the train's states")
    out = []
    for cyc in range((N + pulses_per_cycle - 1) // pulses_per_cycle):
        for m in range(m0, m1):
            n = cyc * pulses_per_cycle + m
            if n < N:
                out.append(n)
    idx = np.asarray(out, dtype=np.int64)
    # the local cycle structure must give every local pulse its global state
    local_state = m0 + np.arange(idx.size) % (m1 - m0)
    assert np.array_equal(local_state, idx % pulses_per_cycle)
    return idx


def shard_geometry(geom, m0: int, m1: int):
    """The shard's geometry: its pulse count and m1 - m0 pulses per cycle."""
    n = int(shard_pulses(geom.N, geom.pulses_per_cycle, m0, m1).size)
    if dataclasses.is_dataclass(geom):
        return dataclasses.replace(geom, N=n, pulses_per_cycle=m1 - m0)
    g = copy.copy(geom)
    g.N, g.pulses_per_cycle = n, m1 - m0
    return g


def make_shard(Operator, geom, K, sw, m0: int, m1: int, precision: str = "fp32"):
    """A handle for the states [m0, m1) of ``geom``'s train."""
    op = Operator(shard_geometry(geom, m0, m1), K, sw, precision=precision)
    op.set_state_offset(m0)
    return op


def shard_measurements(y, geom, m0: int, m1: int):
    """The shard's measurements y[pulses of the shard] (numpy or torch)."""
    idx = shard_pulses(geom.N, geom.pulses_per_cycle, m0, m1)
    try:
        import torch
        if isinstance(y, torch.Tensor):
            return y[torch.as_tensor(idx, device=y.device)].contiguous()
    except ImportError:
        pass
    return np.ascontiguousarray(np.asarray(y)[idx])


def emulate_fista(shards, iters: int):
    """``iters`` FISTA iterations of the shards (each after fista_init with
    its measurements and the same explicit step), one after another on one
    GPU: the gradient of shard r continues the P^T sum of shard r - 1, and
    every shard then takes the summed gradient.  Returns the last gradient
    buffer."""
    g = None
    for _ in range(iters):
        g = None
        for op in shards:
            g = op.fista_gradient(carry=g)
        for op in shards:
            op.fista_step_external(g)
    return g


class ShardedFista:
    """One shard per rank: gradient, ``all_reduce`` (sum) over the process
    group, then the replicated update.  The caller runs ``fista_init`` on
    the rank's shard with its measurements and an explicit step."""

    def __init__(self, op, group=None):
        self.op = op
        self.group = group

    def step(self, iters: int = 1):
        import torch.distributed as dist
        for _ in range(iters):
            g = self.op.fista_gradient()
            dist.all_reduce(g, op=dist.ReduceOp.SUM, group=self.group)
            self.op.fista_step_external(g)
