"""Reverse-mode derivative of the unrolled solve on the GPU against the
oracle's forward-mode tangent (which is pinned against central differences):
the gradient of <w, c_K> with respect to kappa_p and mu after K FISTA
iterations with the TV prox inside, and without it."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_23739_gb300 as sw
from synth import Geometry, Switching

pytestmark = pytest.mark.gpu

GEOM = Geometry(X=8, Y=6, Z=8, T=24, N=6, P=3, k=3, pulses_per_cycle=3)
SWITCH = Switching((0.9, 1.6, 0.0), (1.0, 1.0, 0.0), (0.05, 0.1, 1.0), 2.0)


@pytest.fixture(scope="module")
def problem():
    rng = np.random.default_rng(90)
    K = 0.2 * np.abs(rng.standard_normal(GEOM.k_shape()))
    for j in range(GEOM.Z):
        K[j, 1, 1, 2 * j] += 1.0
    c_true = np.maximum(rng.standard_normal(GEOM.c_shape()), 0)
    y = oracle.forward(GEOM, SWITCH, K, c_true) + 0.05 * rng.standard_normal(GEOM.y_shape())
    L = oracle.power(GEOM, SWITCH, K, rng.standard_normal(GEOM.c_shape()), 200)
    w = rng.standard_normal(GEOM.c_shape())
    return K, y, 0.9 / L, w


@pytest.mark.parametrize("lam_tv,inner,momentum", [(0.02, 10, "beck_teboulle"),
                                                   (0.0, 0, "beck_teboulle"),
                                                   (0.02, 6, "paper_printed")])
def test_unrolled_vjp_matches_oracle_tangent(problem, lam_tv, inner, momentum):
    K, y, alpha, w = problem
    iters, lam_l1 = 8, 0.01
    op = sw.Operator(GEOM, K, SWITCH)
    try:
        params = sw.SolveParams(step=alpha, lambda_l1=lam_l1, lambda_tv=lam_tv, inner_iters=inner,
                                max_iters=iters, momentum=momentum, inner_momentum=momentum)
        yd = torch.tensor(y, dtype=torch.float32, device="cuda")
        wd = torch.tensor(w, dtype=torch.float32, device="cuda")
        c, dk, dm = op.unrolled_vjp(yd, params, wd)
        op.check_device()
    finally:
        op.close()
    got = np.concatenate([dk, [dm]])
    want = np.empty(GEOM.P + 1)
    for which in range(GEOM.P + 1):
        c_o, dc = oracle.fista_tangent(GEOM, SWITCH, K, y, alpha, iters, lam_l1, lam_tv, inner,
                                       which, momentum=momentum, inner_momentum=momentum)
        want[which] = float(np.sum(w * dc))
    c_np = c.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(c_np - c_o) <= 1e-4 * np.linalg.norm(c_o)
    assert np.abs(want).max() > 0
    assert np.linalg.norm(got - want) <= 2e-3 * np.linalg.norm(want)
    # the background species does not switch: its kappa has no effect
    assert abs(got[GEOM.P - 1]) <= 1e-6 * np.linalg.norm(want)
