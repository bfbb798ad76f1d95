"""GPU precision tests: the tensor-core precisions (two-term BF16, BF16, FP8
E4M3 with per-channel equilibration) against the FP64 oracle on the large
workload's structure scaled down (32 x 32 scan, 24 depths, T = 128, 31 x 31
support, 3 species, 20 pulses), FP64 spot checks of sampled outputs of H and
H^T at the full large size (128 x 128 x 96, T = 512), and the refined solve
on the scaled-down structure.

Tolerances (relative L2), from the arithmetic:
- FP32 (CUDA cores): 1e-5.
- two-term BF16: each operand kept to 2^-16, products to about 3 2^-16; the
  tensor core's FP32 accumulation over the ~10^5 terms of an output of the
  31 x 31 support adds about sqrt(10^5) 2^-24 = 2e-5: held to 1e-4.
- three-term BF16 does not fit the 31 x 31 support (three image terms of its
  halo leave no shared memory for the kernel stages) and is refused there.
- BF16: two roundings of <= 2^-8 per product: held to 5e-3.
- FP8 E4M3: two roundings of <= 2^-4 per product (0.125 worst case, about 0.07
  rms): held to 0.1.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_23739_gb300 as sw
import synth

pytestmark = pytest.mark.gpu

LARGE = synth.workload("large_128x128x96_T512_k31_N60_P3")
TOL = {"fp32": 1e-5, "bf16x6": 1e-5, "bf16x3": 1e-4, "bf16": 5e-3, "fp8": 1e-1}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def scaled():
    """The large workload's structure, scaled down so that the oracle
    evaluates H and H^T in full."""
    prob = synth.small_variant(LARGE, X=32, Y=32, Z=24, T=128, N=20)
    g, s = prob.geom, prob.sw
    K = synth.transducer_kernel(g, seed=0)
    c = synth.tube_phantom(g, 6, seed=2)
    w = synth.gaussian(g.y_shape(), 3)
    return prob, g, s, K, c, w, oracle.forward(g, s, K, c), oracle.adjoint(g, s, K, w)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16", "fp8"])
def test_scaled_large_structure_operators_match_oracle(scaled, prec):
    prob, g, s, K, c, w, f_ref, a_ref = scaled
    assert (g.X, g.Y, g.Z, g.T, g.k, g.N, g.P) == (32, 32, 24, 128, 31, 20, 3)
    op = sw.Operator(g, K, s, precision=prec)
    f = host(op.forward(dev(c)))
    a = host(op.adjoint(dev(w)))
    op.check_device()
    op.close()
    assert rel(f, f_ref) <= TOL[prec]
    assert rel(a, a_ref) <= TOL[prec]


def test_fp8_is_deterministic_and_scales_with_the_input(scaled):
    """The per-call image scale sigma cancels: H(2 c) = 2 H(c) up to the
    E4M3 rounding of the scaled images (identical codes, so bit for bit), and
    two calls give the same bits."""
    prob, g, s, K, c, w, _, _ = scaled
    op = sw.Operator(g, K, s, precision="fp8")
    f1 = op.forward(dev(c)).clone()
    f2 = op.forward(dev(c)).clone()
    f3 = op.forward(dev(2.0 * c))
    op.check_device()
    op.close()
    assert torch.equal(f1, f2)
    assert torch.equal(2.0 * f1, f3)


def test_refined_default_schedule_on_scaled_large_structure(scaled):
    """The benchmark's refined schedule on the large workload's structure:
    2 FISTA iterations of the refined BF16 solve against the oracle's
    iterates with the same step."""
    prob, g, s, K, c, w, f_ref, _ = scaled
    y = f_ref + synth.noise_sigma(f_ref, prob.snr_db) * synth.gaussian(g.y_shape(), 9)
    op = sw.Operator(g, K, s)
    alpha = 1.0 / op.lipschitz(30)
    iters = 2
    op.set_precision("bf16")
    got, _ = op.solve(dev(y), sw.SolveParams(step=alpha, lambda_l1=prob.lam_l1,
                                             lambda_tv=prob.lam_tv, inner_iters=prob.inner,
                                             max_iters=iters, **sw.REFINED_DEFAULTS))
    op.check_device()
    op.close()
    ref = oracle.fista(g, s, K, y, alpha, iters, prob.lam_l1, prob.lam_tv, prob.inner)
    assert rel(host(got), ref) <= 1e-4


@pytest.fixture(scope="module")
def large_full():
    g, s = LARGE.geom, LARGE.sw
    K = synth.transducer_kernel(g, seed=0)
    c = synth.tube_phantom(g, LARGE.tubes, seed=0)
    rng = np.random.default_rng(11)
    # 24 measurement rows (24 x 512 = 12288 outputs of H) and 2048 entries of H^T
    nyx = np.stack([rng.integers(0, g.N, 24), rng.integers(0, g.Y, 24),
                    rng.integers(0, g.X, 24)], axis=1)
    pyxj = np.stack([rng.integers(0, g.P, 2048), rng.integers(0, g.Y, 2048),
                     rng.integers(0, g.X, 2048), rng.integers(0, g.Z, 2048)], axis=1)
    # H^T's input: N(0, 1) on the first cycle of pulses (every switching state), 0 after
    ncyc = g.pulses_per_cycle
    w = np.zeros(g.y_shape())
    w[:ncyc] = synth.gaussian((ncyc, g.Y, g.X, g.T), 12)
    f_ref = oracle.forward_at(g, s, K, c, nyx)
    a_ref = oracle.adjoint_at(g, s, K, w, pyxj)
    return g, s, K, c, w, nyx, pyxj, f_ref, a_ref


def test_three_term_split_is_refused_on_the_31_wide_support(scaled):
    prob, g, s, K, c, w, f_ref, a_ref = scaled
    with pytest.raises(sw.SwoptError, match="no tensor-core configuration fits"):
        sw.Operator(g, K, s, precision="bf16x6")


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16", "fp8"])
def test_full_large_spot_checks_against_fp64(large_full, prec):
    """FP64 spot checks at the full large size: 12288 sampled outputs of H
    (24 rows of 512 samples) and 2048 of H^T, each an independent sum the
    oracle evaluates directly."""
    g, s, K, c, w, nyx, pyxj, f_ref, a_ref = large_full
    op = sw.Operator(g, K, s, precision=prec)
    y = op.forward(dev(c))
    f = host(y[nyx[:, 0], nyx[:, 1], nyx[:, 2], :])
    del y
    wt = torch.zeros(g.y_shape(), dtype=torch.float32, device="cuda")
    ncyc = g.pulses_per_cycle
    wt[:ncyc] = dev(w[:ncyc])
    a = host(op.adjoint(wt)[pyxj[:, 0], pyxj[:, 1], pyxj[:, 2], pyxj[:, 3]])
    op.check_device()
    op.close()
    assert f.size >= 10000 and rel(f, f_ref) <= TOL[prec]
    assert rel(a, a_ref) <= TOL[prec]
