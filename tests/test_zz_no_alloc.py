"""The allocation-free TV prox (swopt_prox_tv_static) against the handle-based
swopt_prox_tv, both called through the C-ABI.

swopt_prox_tv_static serves callers that must not allocate device memory
(a framework whose allocator owns the GPU's memory, a real-time loop that
cannot take cudaMalloc's synchronisation): its scratch is a static device
array.  This file is collected last so that a failure here does not hide
the rest of the suite, and it runs alone as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2510_23739_gb300 as sw
from synth import Geometry, Switching

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


def _static(z, out, shape, tau, iters, momentum):
    P, Y, X, Z = shape
    return sw.lib().swopt_prox_tv_static(P, Y, X, Z, ctypes.c_void_p(z.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), float(tau), int(iters),
                                         sw.MOMENTUM[momentum],
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _operator(g):
    K = np.random.default_rng(0).standard_normal(g.k_shape())
    s = Switching(tuple([0.1] * (g.P - 1) + [0.0]), tuple([1.0] * (g.P - 1) + [0.0]),
                  tuple([0.0] * (g.P - 1) + [1.0]), 2.0)
    return sw.Operator(g, K, s)


@pytest.mark.parametrize("momentum", ["beck_teboulle", "paper_printed"])
def test_static_scratch_prox_matches_handle_prox_twice(momentum):
    g = Geometry(X=13, Y=11, Z=37, T=8, N=1, P=3, k=1, pulses_per_cycle=1)
    op = _operator(g)
    rng = np.random.default_rng(1)
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        z = torch.tensor(rng.standard_normal(g.c_shape()), dtype=torch.float32, device="cuda")
        ref = op.prox_tv(z, 0.15 + 0.1 * call, 10, momentum)
        out = torch.full_like(z, float("nan"))
        st = _static(z, out, g.c_shape(), 0.15 + 0.1 * call, 10, momentum)
        assert st == 0, sw.lib().swopt_last_error()
        torch.cuda.synchronize()
        assert _rel(out, ref) <= 1e-5
    op.close()


def test_static_scratch_at_its_maximum_size():
    # P*Y*X*Z = 2*64*64*64 = 2^19, the documented maximum (the medium workload's volume)
    g = Geometry(X=64, Y=64, Z=64, T=8, N=1, P=2, k=1, pulses_per_cycle=1)
    op = _operator(g)
    rng = np.random.default_rng(2)
    for call in range(2):
        z = torch.tensor(rng.standard_normal(g.c_shape()), dtype=torch.float32, device="cuda")
        ref = op.prox_tv(z, 0.3, 10)
        out = torch.empty_like(z)
        assert _static(z, out, g.c_shape(), 0.3, 10, "beck_teboulle") == 0
        torch.cuda.synchronize()
        assert _rel(out, ref) <= 1e-5
    op.close()


def test_static_scratch_rejects_volumes_above_the_limit():
    z = torch.zeros(8, device="cuda")
    out = torch.zeros(8, device="cuda")
    st = _static(z, out, (2, 64, 64, 65), 0.1, 10, "beck_teboulle")
    assert st == 2  # SWOPT_ERR_SHAPE, before any GPU work
    assert b"static scratch limit" in sw.lib().swopt_last_error()
