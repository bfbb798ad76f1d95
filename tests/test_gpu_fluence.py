"""The diffusion-equation fluence on the GPU (FP64 conjugate gradients on the
finite-volume system of Eqs. (de)/(bc)) against the oracle's sparse direct
solve of the same system, and the fluence profile in Eq. (final-H)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_23739_gb300 as sw
from synth import Geometry, Switching

pytestmark = pytest.mark.gpu


def _medium(Y, X, Z, seed):
    rng = np.random.default_rng(seed)
    mu_a = 0.02 + 0.3 * (rng.random((Y, X, Z)) > 0.9)   # a background with absorbers
    mu_s = 8.0 + rng.random((Y, X, Z))
    src = np.zeros((Y, X))
    src[:, X // 4: 3 * X // 4] = 1.0                    # a band of illumination
    return mu_a, mu_s, src


@pytest.mark.parametrize("lateral_robin", [True, False])
def test_diffusion_fluence_matches_oracle(lateral_robin):
    Y, X, Z, dx, dz, g = 6, 10, 16, 0.02, 0.01, 0.9
    mu_a, mu_s, src = _medium(Y, X, Z, 50)
    phi, iters, rel = sw.diffusion_fluence(Y, X, Z, dx, dz, mu_a, mu_s, g, src,
                                           lateral_robin=lateral_robin, tol=1e-12)
    want = oracle.diffusion_fluence(Y, X, Z, dx, dz, mu_a, mu_s, g, src, lateral_robin)
    assert rel <= 1e-12 and iters > 1
    assert np.linalg.norm(phi - want) <= 1e-9 * np.linalg.norm(want)


def test_diffusion_fluence_converges_on_a_larger_grid():
    Y, X, Z = 32, 32, 48
    mu_a, mu_s, src = _medium(Y, X, Z, 51)
    phi, iters, rel = sw.diffusion_fluence(Y, X, Z, 0.02, 0.01, mu_a, mu_s, 0.9, src, tol=1e-10)
    assert rel <= 1e-10 and phi.min() > 0
    # the residual of the oracle's matrix at the GPU solution
    A, b = oracle.diffusion_system(Y, X, Z, 0.02, 0.01, mu_a, mu_s, 0.9, src)
    assert np.linalg.norm(A @ phi.ravel() - b) <= 1e-9 * np.linalg.norm(b)


def test_fluence_profile_enters_the_switching_model():
    """The lateral mean of the diffusion fluence replaces exp(-mu j dz) in
    Eq. (final-H): H against the oracle with the same profile; no mu
    derivative with a given profile; None restores the exponential."""
    g = Geometry(X=8, Y=6, Z=10, T=24, N=5, P=2, k=3, pulses_per_cycle=3)
    s = Switching((0.7, 0.0), (1.0, 0.0), (0.05, 1.0), 2.0)
    rng = np.random.default_rng(52)
    K = rng.standard_normal(g.k_shape())
    c = rng.random(g.c_shape())
    mu_a, mu_s, src = _medium(g.Y, g.X, g.Z, 53)
    phi3, _, _ = sw.diffusion_fluence(g.Y, g.X, g.Z, g.dx_mm, g.dz_mm, mu_a, mu_s, 0.9,
                                      np.ones((g.Y, g.X)))
    prof = phi3.mean(axis=(0, 1))
    prof = prof / prof[0]
    op = sw.Operator(g, K, s)
    try:
        cd = torch.tensor(c, dtype=torch.float32, device="cuda")
        base = op.forward(cd).clone()
        op.set_fluence(prof)
        got = op.forward(cd).cpu().numpy().astype(np.float64)
        y = torch.tensor(rng.standard_normal(g.y_shape()), dtype=torch.float32, device="cuda")
        _, dmu = op.param_grad(cd, y)
        op.set_fluence(None)
        again = op.forward(cd)
        op.check_device()
    finally:
        op.close()
    want = oracle.forward(g, s, K, c, S=oracle.switch_matrix(g, s, phi=prof))
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
    assert dmu == 0.0
    assert torch.equal(again, base)
