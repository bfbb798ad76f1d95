"""GPU parity: the CUDA library, called through the C-ABI, against the FP64
oracle on the same seeded inputs.

Tolerances (relative L2 unless stated): the FP32 operator <= 1e-5, proximal
maps <= 1e-5, FISTA iterates after a fixed number of iterations <= 1e-4
(all with the same step alpha on both sides).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_23739_gb300 as sw
import synth
from synth import Geometry, Switching

pytestmark = pytest.mark.gpu

TINY = synth.workload("tiny_16x16x24_T64_k7_N8_P2")
MEDIUM = synth.workload("medium_64x64x64_T256_k15_N40_P2")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


# ragged and degenerate shapes: tiles, depth chunks and windows with tails
CASES = {
    "tiny": (TINY.geom, TINY.sw, 0),
    "ragged": (Geometry(X=13, Y=11, Z=37, T=57, N=7, P=3, k=5, pulses_per_cycle=3),
               Switching((0.04, 0.09, 0.0), (1.0, 0.8, 0.0), (0.0, 0.1, 1.0), 3.0), 1),
    "k1_one_pulse": (Geometry(X=17, Y=5, Z=3, T=20, N=1, P=1, k=1, pulses_per_cycle=5),
                     Switching((0.0,), (0.0,), (1.0,), 0.0), 2),
    "pulses_below_cycle": (Geometry(X=6, Y=9, Z=33, T=40, N=3, P=2, k=9, pulses_per_cycle=10),
                           Switching((0.2, 0.0), (1.0, 0.0), (0.0, 1.0), 2.0), 3),
    "single_column": (Geometry(X=1, Y=1, Z=5, T=33, N=4, P=2, k=3, pulses_per_cycle=2),
                      Switching((0.3, 0.0), (1.0, 0.0), (0.0, 1.0), 1.0), 4),
    "support_wider_than_grid": (Geometry(X=4, Y=3, Z=8, T=48, N=5, P=2, k=11, pulses_per_cycle=5),
                                Switching((0.1, 0.0), (1.0, 0.0), (0.0, 1.0), 2.0), 5),
    "support_31": (Geometry(X=12, Y=10, Z=24, T=80, N=3, P=2, k=31, pulses_per_cycle=3),
                   Switching((0.05, 0.0), (1.0, 0.0), (0.0, 1.0), 2.0), 6),
}


def _kernel(g, seed):
    if g.k >= 3 and g.T >= 32:
        try:
            return synth.transducer_kernel(g, seed=seed)
        except Exception:
            pass
    rng = np.random.default_rng(seed)
    K = rng.standard_normal(g.k_shape())
    K[..., : g.T // 4] = 0.0  # a window that does not start at 0
    return K


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, (g, s, seed) in CASES.items():
        K = _kernel(g, seed)
        if not np.any(K):
            K = np.random.default_rng(seed).standard_normal(g.k_shape())
        out[name] = (g, s, K, sw.Operator(g, K, s))
    yield out
    for v in out.values():
        v[3].close()


@pytest.mark.parametrize("name", list(CASES))
def test_forward_matches_oracle(cases, name):
    g, s, K, op = cases[name]
    c = np.random.default_rng(10).standard_normal(g.c_shape())
    got = host(op.forward(dev(c)))
    ref = oracle.forward(g, s, K, c)
    assert rel(got, ref) <= 1e-5
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max() * 10


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_matches_oracle(cases, name):
    g, s, K, op = cases[name]
    yv = np.random.default_rng(11).standard_normal(g.y_shape())
    got = host(op.adjoint(dev(yv)))
    ref = oracle.adjoint(g, s, K, yv)
    assert rel(got, ref) <= 1e-5


def test_forward_of_phantom_matches_oracle(cases):
    g, s, K, op = cases["tiny"]
    c = synth.tube_phantom(g, TINY.tubes, seed=0, per_species=True)
    assert rel(host(op.forward(dev(c))), oracle.forward(g, s, K, c)) <= 1e-5


def test_adjoint_identity_on_gpu(cases):
    g, s, K, op = cases["ragged"]
    rng = np.random.default_rng(12)
    for _ in range(20):
        x = dev(rng.standard_normal(g.c_shape()))
        y = dev(rng.standard_normal(g.y_shape()))
        hx = op.forward(x)
        lhs = float(torch.sum(hx.double() * y.double()))
        rhs = float(torch.sum(x.double() * op.adjoint(y).double()))
        scale = float(hx.double().norm() * y.double().norm())
        assert abs(lhs - rhs) <= 1e-6 * scale


def test_operator_is_deterministic(cases):
    g, s, K, op = cases["tiny"]
    c = dev(np.random.default_rng(13).standard_normal(g.c_shape()))
    a = op.forward(c)
    b = op.forward(c)
    assert torch.equal(a, b)
    y = dev(np.random.default_rng(14).standard_normal(g.y_shape()))
    assert torch.equal(op.adjoint(y), op.adjoint(y))


@pytest.mark.parametrize("nonneg", [True, False])
def test_prox_l1_matches_oracle(cases, nonneg):
    g, s, K, op = cases["ragged"]
    z = np.random.default_rng(15).standard_normal(g.c_shape())
    x = dev(z)
    op.prox_l1(x, 0.3, nonneg)
    ref = oracle.prox_l1(z, 0.3, nonneg)
    np.testing.assert_allclose(host(x), ref, atol=1e-6)


@pytest.mark.parametrize("name", ["tiny", "ragged", "single_column"])
@pytest.mark.parametrize("momentum", ["beck_teboulle", "paper_printed", "none"])
def test_prox_tv_matches_oracle(cases, name, momentum):
    g, s, K, op = cases[name]
    z = np.random.default_rng(16).standard_normal(g.c_shape())
    got = host(op.prox_tv(dev(z), 0.2, 10, momentum))
    ref = oracle.prox_tv(z, 0.2, 10, momentum)
    assert rel(got, ref) <= 1e-5


def test_prox_tv_unaligned_input_and_medium_volume(cases, medium):
    """The TV prox keeps its state in shared memory when the volume fits there
    (the medium volume does) and reads its input column by column: an input
    that starts 4 bytes past a 16-byte boundary gives bitwise the result of
    an aligned copy, and the medium volume matches the oracle."""
    g, s, K, op = cases["tiny"]
    n = int(np.prod(g.c_shape()))
    base = torch.zeros(n + 1, device="cuda")
    z = np.random.default_rng(23).standard_normal(g.c_shape())
    base[1:] = dev(z).reshape(-1)
    zu = base[1:].view(g.c_shape())
    assert zu.data_ptr() % 16 == 4
    assert torch.equal(op.prox_tv(zu, 0.3, 6), op.prox_tv(dev(z), 0.3, 6))
    gm, _, _, opm = medium
    zm = synth.gaussian(gm.c_shape(), 24) * 0.05
    got = host(opm.prox_tv(dev(zm), 0.02, 10))
    assert rel(got, oracle.prox_tv(zm, 0.02, 10)) <= 1e-5
    opm.check_device()


def test_prox_tv_zero_iterations_and_zero_tau(cases):
    g, s, K, op = cases["tiny"]
    z = dev(np.random.default_rng(17).standard_normal(g.c_shape()))
    assert torch.equal(op.prox_tv(z, 0.5, 0), z)
    assert torch.equal(op.prox_tv(z, 0.0, 10), z)


def _tiny_measurements(g, s, K, seed=0):
    c_true = synth.tube_phantom(g, TINY.tubes, seed=seed, per_species=True)
    clean = oracle.forward(g, s, K, c_true)
    sigma = synth.noise_sigma(clean, TINY.snr_db)
    return clean + sigma * synth.gaussian(g.y_shape(), seed + 100)


@pytest.mark.parametrize("momentum", ["beck_teboulle", "paper_printed"])
def test_fista_tiny_workload_matches_oracle(cases, momentum):
    """The tiny workload's plain solve: 20 iterations, lambda_l1 = lambda_TV =
    1e-3, 10 inner iterations, the same alpha on both sides."""
    g, s, K, op = cases["tiny"]
    y = _tiny_measurements(g, s, K)
    L = oracle.power(g, s, K, synth.gaussian(g.c_shape(), 1), 100)
    alpha = 1.0 / L
    params = sw.SolveParams(step=alpha, lambda_l1=TINY.lam_l1, lambda_tv=TINY.lam_tv,
                            inner_iters=TINY.inner, max_iters=TINY.iters, momentum=momentum,
                            inner_momentum=momentum)
    got, stats = op.solve(dev(y), params)
    ref = oracle.fista(g, s, K, y, alpha, TINY.iters, TINY.lam_l1, TINY.lam_tv, TINY.inner,
                       momentum=momentum, inner_momentum=momentum)
    assert stats["iters"] == TINY.iters
    assert rel(host(got), ref) <= 1e-4
    F_ref, fit_ref = oracle.objective(g, s, K, ref, y, TINY.lam_l1, TINY.lam_tv)
    assert stats["objective"] == pytest.approx(F_ref, rel=1e-4)


def test_fista_ragged_matches_oracle(cases):
    g, s, K, op = cases["ragged"]
    rng = np.random.default_rng(18)
    y = oracle.forward(g, s, K, np.maximum(rng.standard_normal(g.c_shape()), 0))
    L = oracle.power(g, s, K, synth.gaussian(g.c_shape(), 2), 60)
    params = sw.SolveParams(step=1.0 / L, lambda_l1=0.01, lambda_tv=0.02, inner_iters=5,
                            max_iters=8)
    got, _ = op.solve(dev(y), params)
    ref = oracle.fista(g, s, K, y, 1.0 / L, 8, 0.01, 0.02, 5)
    assert rel(host(got), ref) <= 1e-4


def test_fista_steps_equal_solve(cases):
    g, s, K, op = cases["tiny"]
    y = dev(_tiny_measurements(g, s, K, 3))
    params = sw.SolveParams(step=0.5 / oracle.power(g, s, K, synth.gaussian(g.c_shape(), 1), 50),
                            max_iters=6)
    a, _ = op.solve(y, params)
    op.fista_init(y, params)
    op.fista_step(2)
    op.fista_step(4)
    b = op.fista_get()
    assert torch.equal(a, b)


def test_lipschitz_matches_dense_eigenvalue():
    g = Geometry(X=5, Y=4, Z=4, T=20, N=4, P=2, k=3, pulses_per_cycle=2)
    s = Switching((0.5, 0.0), (1.0, 0.0), (0.0, 1.0), 2.0)
    K = np.random.default_rng(19).standard_normal(g.k_shape())
    nc = int(np.prod(g.c_shape()))
    H = np.stack([oracle.forward(g, s, K, e.reshape(g.c_shape())).ravel()
                  for e in np.eye(nc)], axis=1)
    lam = np.linalg.eigvalsh(H.T @ H)[-1]
    op = sw.Operator(g, K, s)
    v0 = synth.gaussian(g.c_shape(), 4)
    L_gpu = op.lipschitz(500, dev(v0))
    assert L_gpu == pytest.approx(lam, rel=1e-4)
    assert op.lipschitz(500) == pytest.approx(lam, rel=1e-4)  # built-in start vector
    assert L_gpu == pytest.approx(oracle.power(g, s, K, v0, 500), rel=1e-5)
    op.close()


def test_objective_matches_oracle(cases):
    g, s, K, op = cases["ragged"]
    rng = np.random.default_rng(20)
    c = np.maximum(rng.standard_normal(g.c_shape()), 0)
    y = rng.standard_normal(g.y_shape())
    F, fit = op.objective(dev(c), dev(y), 0.05, 0.07)
    F_ref, fit_ref = oracle.objective(g, s, K, c, y, 0.05, 0.07)
    assert F == pytest.approx(F_ref, rel=1e-6)
    assert fit == pytest.approx(fit_ref, rel=1e-6)


def test_param_grad_matches_oracle(cases):
    g, s, K, op = cases["ragged"]
    rng = np.random.default_rng(21)
    c = np.maximum(rng.standard_normal(g.c_shape()), 0)
    y = oracle.forward(g, s, K, c * 1.1) + 0.01 * rng.standard_normal(g.y_shape())
    dk, dmu = op.param_grad(dev(c), dev(y))
    dk_ref, dmu_ref = oracle.param_grad(g, s, K, c, y)
    for p in range(g.P):
        if dk_ref[p] != 0:
            assert dk[p] == pytest.approx(dk_ref[p], rel=1e-4)
    assert dmu == pytest.approx(dmu_ref, rel=1e-4)


def test_solve_stops_on_eps2(cases):
    g, s, K, op = cases["tiny"]
    y = dev(_tiny_measurements(g, s, K, 5))
    params = sw.SolveParams(step=0.0, power_iters=50, max_iters=300, eps2=0.05)
    _, stats = op.solve(y, params, history=True)
    assert 1 < stats["iters"] < 300
    assert len(stats["history"]) == stats["iters"]
    assert np.all(np.isfinite(stats["history"]))
    params = sw.SolveParams(step=0.0, power_iters=50, max_iters=300, eps1=1e-3)
    _, stats = op.solve(y, params, history=True)
    assert 1 < stats["iters"] < 300
    h = stats["history"]
    assert abs(h[-1] - h[-2]) < 1e-3 * abs(h[-2])


def test_invalid_arguments_raise(cases):
    g, s, K, op = cases["tiny"]
    with pytest.raises(ValueError):
        op.forward(torch.zeros((1, 2, 3), device="cuda"))
    with pytest.raises(sw.SwoptError):
        sw._check(sw.lib().swopt_prox_l1(op._h, None, 0.1, 1, None))
    with pytest.raises(sw.SwoptError):
        op.prox_l1(dev(np.zeros(g.c_shape())), -1.0)


# ---------------------------------------------------------------------------
# Full size: the medium workload (64x64 scan, 64 depths, T=256, 15x15 support,
# 40 pulses in 4 cycles, 2 species) in the launch configuration the benchmark
# times, checked on sampled outputs that the oracle evaluates one by one.
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def medium():
    g, s = MEDIUM.geom, MEDIUM.sw
    K = synth.transducer_kernel(g, seed=0)
    op = sw.Operator(g, K, s)
    yield g, s, K, op
    op.close()


def test_medium_forward_sampled(medium):
    g, s, K, op = medium
    c = synth.tube_phantom(g, MEDIUM.tubes, seed=0)
    y = host(op.forward(dev(c)))
    rng = np.random.default_rng(22)
    idx = np.stack([rng.integers(0, g.N, 48), rng.integers(0, g.Y, 48), rng.integers(0, g.X, 48)], 1)
    idx[:4] = [[0, 0, 0], [g.N - 1, g.Y - 1, g.X - 1], [5, 0, g.X - 1], [39, g.Y - 1, 7]]
    ref = oracle.forward_at(g, s, K, c, idx)
    got = y[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert rel(got, ref) <= 1e-5


def test_medium_adjoint_sampled(medium):
    g, s, K, op = medium
    yv = synth.gaussian(g.y_shape(), 23)
    c = host(op.adjoint(dev(yv)))
    rng = np.random.default_rng(24)
    idx = np.stack([rng.integers(0, g.P, 48), rng.integers(0, g.Y, 48), rng.integers(0, g.X, 48),
                    rng.integers(0, g.Z, 48)], 1)
    idx[:2] = [[0, 0, 0, 0], [g.P - 1, g.Y - 1, g.X - 1, g.Z - 1]]
    ref = oracle.adjoint_at(g, s, K, yv, idx)
    got = c[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]]
    assert rel(got, ref) <= 1e-5


def test_medium_adjoint_identity_and_descent(medium):
    g, s, K, op = medium
    rng = np.random.default_rng(25)
    x = dev(rng.standard_normal(g.c_shape()))
    y = dev(rng.standard_normal(g.y_shape()))
    hx = op.forward(x)
    lhs = float(torch.sum(hx.double() * y.double()))
    rhs = float(torch.sum(x.double() * op.adjoint(y).double()))
    assert abs(lhs - rhs) <= 1e-6 * float(hx.double().norm() * y.double().norm())
    # a few FISTA iterations on a noisy phantom lower the objective
    c_true = dev(synth.tube_phantom(g, MEDIUM.tubes, seed=0))
    ym = op.forward(c_true)
    params = sw.SolveParams(step=0.0, power_iters=30, lambda_l1=MEDIUM.lam_l1,
                            lambda_tv=MEDIUM.lam_tv, inner_iters=MEDIUM.inner, max_iters=5)
    _, stats = op.solve(ym, params, history=True)
    h = stats["history"]
    F0 = 0.5 * float(ym.double().pow(2).sum())
    assert h[-1] < h[0] < F0


# ---------------------------------------------------------------------------
# Tensor-core precisions.  Tolerances (relative L2).  BF16 keeps 8
# significant bits (unit roundoff u = 2^-8).  The split mode writes each
# operand as v = hi + lo with |v - hi - lo| <= u^2 |v| = 2^-16 |v| and
# accumulates hi*hi + hi*lo + lo*hi in FP32, so each product carries at most
# about 3 * 2^-16 = 4.6e-5 relative error (two representation errors and the
# dropped lo*lo, each <= 2^-16): held to 4e-5 (measured 0.4-1.0e-5 with the
# corrections accumulated apart).  The three-term split keeps each product to
# about 3 * 2^-24; the FP32 accumulation is then what is left, as on the CUDA
# cores: held to the FP32 operator bound, 1e-5.  Plain BF16: two roundings of <= 2^-8 per
# product (7.8e-3 worst, about 0.9-3.3e-3 measured): held to 5e-3.  FP8 E4M3
# (3 mantissa bits, u = 2^-4) with per-channel equilibration: two roundings
# of <= 2^-4 per product (0.125 worst): held to 0.1 (measured 0.8-4e-2).
# ---------------------------------------------------------------------------
TC_TOL = {"bf16x6": 1e-5, "bf16x3": 4e-5, "bf16": 5e-3, "fp8": 1e-1}


@pytest.fixture(scope="module")
def tc_cases():
    out = {}
    for name in ("tiny", "ragged", "k1_one_pulse", "pulses_below_cycle", "single_column",
                 "support_wider_than_grid", "support_31"):
        g, s, seed = CASES[name]
        K = _kernel(g, seed)
        out[name] = (g, s, K)
    return out


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16", "fp8"])
@pytest.mark.parametrize("name", ["tiny", "ragged", "k1_one_pulse", "pulses_below_cycle",
                                  "single_column", "support_wider_than_grid", "support_31"])
def test_tensor_core_operator_matches_oracle(tc_cases, name, prec):
    g, s, K = tc_cases[name]
    if prec == "bf16x6" and g.k > 27:
        # three image terms of a 31-wide halo leave no shared memory for the
        # kernel stages: refused on the host, before any GPU work
        with pytest.raises(sw.SwoptError, match="no tensor-core configuration fits"):
            sw.Operator(g, K, s, precision=prec)
        return
    op = sw.Operator(g, K, s, precision=prec)
    c = np.random.default_rng(30).standard_normal(g.c_shape())
    yv = np.random.default_rng(31).standard_normal(g.y_shape())
    f = host(op.forward(dev(c)))
    a = host(op.adjoint(dev(yv)))
    op.check_device()
    assert rel(f, oracle.forward(g, s, K, c)) <= TC_TOL[prec]
    assert rel(a, oracle.adjoint(g, s, K, yv)) <= TC_TOL[prec]
    op.close()


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16"])
def test_tensor_core_medium_sampled(medium, prec):
    g, s, K, op = medium
    op.set_precision(prec)
    try:
        c = synth.tube_phantom(g, MEDIUM.tubes, seed=1)
        y = host(op.forward(dev(c)))
        rng = np.random.default_rng(32)
        idx = np.stack([rng.integers(0, g.N, 32), rng.integers(0, g.Y, 32),
                        rng.integers(0, g.X, 32)], 1)
        assert rel(y[idx[:, 0], idx[:, 1], idx[:, 2]], oracle.forward_at(g, s, K, c, idx)) \
            <= TC_TOL[prec]
        yv = synth.gaussian(g.y_shape(), 33)
        cg = host(op.adjoint(dev(yv)))
        idx4 = np.stack([rng.integers(0, g.P, 32), rng.integers(0, g.Y, 32),
                         rng.integers(0, g.X, 32), rng.integers(0, g.Z, 32)], 1)
        assert rel(cg[idx4[:, 0], idx4[:, 1], idx4[:, 2], idx4[:, 3]],
                   oracle.adjoint_at(g, s, K, yv, idx4)) <= TC_TOL[prec]
        op.check_device()
    finally:
        op.set_precision("fp32")


def test_tensor_core_fista_split_matches_oracle(tc_cases):
    g, s, K = tc_cases["tiny"]
    op = sw.Operator(g, K, s, precision="bf16x3")
    y = _tiny_measurements(g, s, K)
    alpha = 1.0 / oracle.power(g, s, K, synth.gaussian(g.c_shape(), 1), 100)
    params = sw.SolveParams(step=alpha, lambda_l1=TINY.lam_l1, lambda_tv=TINY.lam_tv,
                            inner_iters=TINY.inner, max_iters=TINY.iters)
    got, stats = op.solve(dev(y), params)
    ref = oracle.fista(g, s, K, y, alpha, TINY.iters, TINY.lam_l1, TINY.lam_tv, TINY.inner)
    assert rel(host(got), ref) <= 1e-4
    op.close()


def test_tensor_core_lipschitz_and_param_grad(tc_cases):
    g, s, K = tc_cases["ragged"]
    op = sw.Operator(g, K, s, precision="bf16x3")
    v0 = synth.gaussian(g.c_shape(), 5)
    assert op.lipschitz(50, dev(v0)) == pytest.approx(oracle.power(g, s, K, v0, 50), rel=1e-5)
    rng = np.random.default_rng(34)
    c = np.maximum(rng.standard_normal(g.c_shape()), 0)
    y = oracle.forward(g, s, K, c * 1.1) + 0.01 * rng.standard_normal(g.y_shape())
    dk, dmu = op.param_grad(dev(c), dev(y))
    dk_ref, dmu_ref = oracle.param_grad(g, s, K, c, y)
    assert dmu == pytest.approx(dmu_ref, rel=1e-4)
    for p in range(g.P):
        if dk_ref[p] != 0:
            assert dk[p] == pytest.approx(dk_ref[p], rel=1e-4)
    op.close()


def test_tensor_core_operator_is_deterministic(tc_cases):
    g, s, K = tc_cases["tiny"]
    op = sw.Operator(g, K, s, precision="bf16")
    c = dev(np.random.default_rng(35).standard_normal(g.c_shape()))
    assert torch.equal(op.forward(c), op.forward(c))
    y = dev(np.random.default_rng(36).standard_normal(g.y_shape()))
    assert torch.equal(op.adjoint(y), op.adjoint(y))
    op.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_graph_replay_equals_direct_launches(tc_cases, prec):
    """A FISTA iteration replayed from its CUDA graph gives bitwise the
    iterate of the same kernels launched one by one."""
    g, s, K = tc_cases["tiny"]
    y = dev(_tiny_measurements(g, s, K, 7))
    params = sw.SolveParams(step=0.5 / oracle.power(g, s, K, synth.gaussian(g.c_shape(), 1), 50),
                            max_iters=5)
    op = sw.Operator(g, K, s, precision=prec)
    op.fista_init(y, params)
    op.fista_step(5)
    a = op.fista_get().clone()
    op.use_graphs(False)
    op.fista_init(y, params)
    op.fista_step(5)
    b = op.fista_get()
    assert torch.equal(a, b)
    # profiling through the graph's event-record nodes
    op.use_graphs(True)
    op.fista_init(y, params)
    op.profile(True)
    op.fista_step(3)
    f = op.profile_read(0)
    adj = op.profile_read(1)
    assert f["launches"] == 3 and adj["launches"] == 3
    assert f["total_ms"] > 0 and adj["total_ms"] > 0
    op.close()


# ---------------------------------------------------------------------------
# Refined solve (incremental gradient).  In exact arithmetic it gives the
# iterates of Algorithm 1, so with FP32 throughout it is held to the plain
# solve's bound.  With BF16 increments the error of an increment scales with
# ||c_{k+1} - c_k||, which is largest in the first iterations: resyncing
# every iteration (R = 1) leaves only the resync precision's error; larger R
# must still beat plain BF16 (the same kernels without refinement).
# ---------------------------------------------------------------------------
def _tiny_solve(g, s, K, prec, **kw):
    y = _tiny_measurements(g, s, K)
    L = oracle.power(g, s, K, synth.gaussian(g.c_shape(), 1), 100)
    params = sw.SolveParams(step=1.0 / L, lambda_l1=TINY.lam_l1, lambda_tv=TINY.lam_tv,
                            inner_iters=TINY.inner, max_iters=TINY.iters, **kw)
    op = sw.Operator(g, K, s, precision=prec)
    got, stats = op.solve(dev(y), params)
    op.check_device()
    op.close()
    ref = oracle.fista(g, s, K, y, 1.0 / L, TINY.iters, TINY.lam_l1, TINY.lam_tv, TINY.inner)
    return rel(host(got), ref), stats


@pytest.mark.parametrize("R", [1, 3, 1000])
def test_refined_fp32_matches_oracle(tc_cases, R):
    g, s, K = tc_cases["tiny"]
    e, stats = _tiny_solve(g, s, K, "fp32", refine_every=R, refine_precision="fp32")
    assert stats["iters"] == TINY.iters
    assert e <= 1e-4


def test_refined_bf16_matches_oracle(tc_cases):
    g, s, K = tc_cases["tiny"]
    e1, _ = _tiny_solve(g, s, K, "bf16", refine_every=1, refine_precision="bf16x3")
    assert e1 <= 1e-4
    e1f, _ = _tiny_solve(g, s, K, "bf16", refine_every=1, refine_precision="fp32")
    assert e1f <= 1e-4
    plain, _ = _tiny_solve(g, s, K, "bf16")
    for R in (2, 5):
        eR, _ = _tiny_solve(g, s, K, "bf16", refine_every=R, refine_precision="bf16x3")
        assert eR < plain


def test_refined_graph_replay_equals_direct_launches(tc_cases):
    g, s, K = tc_cases["tiny"]
    y = dev(_tiny_measurements(g, s, K, 7))
    params = sw.SolveParams(step=0.5 / oracle.power(g, s, K, synth.gaussian(g.c_shape(), 1), 50),
                            max_iters=9, refine_every=4, refine_precision="bf16x3")
    op = sw.Operator(g, K, s, precision="bf16")
    op.fista_init(y, params)
    op.fista_step(9)
    a = op.fista_get().clone()
    op.use_graphs(False)
    op.fista_init(y, params)
    op.fista_step(9)
    b = op.fista_get()
    assert torch.equal(a, b)
    # the solve entry point runs the same iterations
    op.use_graphs(True)
    c, stats = op.solve(y, params)
    assert stats["iters"] == 9 and torch.equal(a, c)
    op.close()


def test_refined_medium_tracks_fp32_objective(medium):
    """Medium workload: over 150 iterations the objective of the refined BF16
    solve stays within 1e-5 (relative; 3e-6 measured) of the plain FP32
    solve's, where plain BF16 drifts further."""
    g, s, K, op = medium
    prob = MEDIUM
    c = synth.tube_phantom(g, prob.tubes, seed=1)
    op.set_precision("fp32")
    y = op.forward(dev(c))
    L = op.lipschitz(30)
    base = dict(step=1.0 / L, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                inner_iters=prob.inner, max_iters=150)
    cf, _ = op.solve(y, sw.SolveParams(**base))
    Ff, _ = op.objective(cf, y, prob.lam_l1, prob.lam_tv)
    ev = sw.Operator(g, K, s)
    try:
        op.set_precision("bf16")
        cr, _ = op.solve(y, sw.SolveParams(refine_every=10, refine_precision="bf16x3", **base))
        cp, _ = op.solve(y, sw.SolveParams(**base))
        op.check_device()
        Fr, _ = ev.objective(cr, y, prob.lam_l1, prob.lam_tv)
        Fp, _ = ev.objective(cp, y, prob.lam_l1, prob.lam_tv)
        assert abs(Fr - Ff) <= 1e-5 * Ff
        assert abs(Fr - Ff) < abs(Fp - Ff)
    finally:
        op.set_precision("fp32")
        ev.close()


@pytest.mark.parametrize("split,buffers", [(1, 1), (1, 2), (2, 1), (2, 2)])
@pytest.mark.parametrize("name", ["tiny", "ragged", "support_31"])
def test_tensor_core_schedules_match_oracle(tc_cases, name, split, buffers):
    """Every work split (whole (state, tile) pairs per CTA, or equal shares of
    all runs, where a pair cut between CTAs is summed by the last to finish)
    and either accumulator buffering gives the oracle's A and A^T, and the
    split-precision results of one handle are bitwise repeatable."""
    g, s, K = tc_cases[name]
    c = np.random.default_rng(41).standard_normal(g.c_shape())
    yv = np.random.default_rng(42).standard_normal(g.y_shape())
    op = sw.Operator(g, K, s)
    try:
        for kid in (0, 1):
            op.tc_schedule(kid, split=split, buffers=buffers)
        op.set_precision("bf16x3")
        for kid in (0, 1):
            info = op.tc_schedule_info(kid)
            assert info["split"] == split and info["buffers"] == buffers
            assert info["grid"] >= 1
            if split == 1:
                assert info["max_pieces"] == 1
        f = host(op.forward(dev(c)))
        a = host(op.adjoint(dev(yv)))
        assert np.array_equal(f, host(op.forward(dev(c))))
        assert np.array_equal(a, host(op.adjoint(dev(yv))))
        op.check_device()
        assert rel(f, oracle.forward(g, s, K, c)) <= TC_TOL["bf16x3"]
        assert rel(a, oracle.adjoint(g, s, K, yv)) <= TC_TOL["bf16x3"]
    finally:
        op.close()


def test_tensor_core_stream_k_sums_many_pieces(tc_cases):
    """On the tiny workload the equal-share split cuts every (state, tile)
    pair among many CTAs (more than two pieces: summed in piece order)."""
    g, s, K = tc_cases["tiny"]
    op = sw.Operator(g, K, s)
    try:
        op.tc_schedule(0, split=2)
        op.tc_schedule(1, split=2)
        op.set_precision("bf16")
        assert op.tc_schedule_info(0)["max_pieces"] > 2
        assert op.tc_schedule_info(1)["max_pieces"] > 2
        c = np.random.default_rng(43).standard_normal(g.c_shape())
        yv = np.random.default_rng(44).standard_normal(g.y_shape())
        f = host(op.forward(dev(c)))
        a = host(op.adjoint(dev(yv)))
        op.check_device()
        assert rel(f, oracle.forward(g, s, K, c)) <= TC_TOL["bf16"]
        assert rel(a, oracle.adjoint(g, s, K, yv)) <= TC_TOL["bf16"]
    finally:
        op.close()


def test_tensor_core_schedule_rejects_bad_values(tc_cases):
    g, s, K = tc_cases["tiny"]
    op = sw.Operator(g, K, s)
    try:
        for bad in ((0, 3, 0), (0, 0, 3), (2, 1, 1), (0, -1, 0)):
            with pytest.raises(Exception):
                op.tc_schedule(*bad)
        with pytest.raises(Exception):
            op.tc_schedule_info(0)  # no tensor-core precision selected
    finally:
        op.close()


def _semicircle_problem(Y, dims):
    """A small scan with the paper-literal kernel (SPR on discrete half
    spheres, matched time grid).  The library's host builder makes the
    kernel the GPU uses; the oracle builds its own for the expected values."""
    g = synth.matched_time_grid(Geometry(X=13, Y=Y, Z=18, T=48, N=5, P=2, k=9,
                                         pulses_per_cycle=4))
    s = Switching((0.08, 0.0), (1.0, 0.0), (0.05, 1.0), 2.0)
    args = (g.Z, g.k, g.T, dims, g.dx_mm / g.dz_mm, (g.Z - 1) / 2.0, g.T // 2,
            synth.spr_image(g, seed=9), synth.eir_taps(g))
    return g, s, sw.semicircle_kernel(*args), oracle.semicircle_kernel(*args)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
@pytest.mark.parametrize("Y,dims", [(11, 3), (1, 2)])
def test_semicircle_kernel_operator_matches_oracle(Y, dims, prec):
    """H and H^T with the paper-literal kernel (a thin shell per depth, the
    very sparse kernel of Eqs. q-above-final / q-below-final), in 3D and on
    a 2D scan (Y = 1), against the oracle."""
    g, s, K, K_or = _semicircle_problem(Y, dims)
    tol = {"fp32": 1e-5, **TC_TOL}[prec]
    op = sw.Operator(g, K, s, precision=prec)
    try:
        c = np.random.default_rng(50).standard_normal(g.c_shape())
        yv = np.random.default_rng(51).standard_normal(g.y_shape())
        f = host(op.forward(dev(c)))
        a = host(op.adjoint(dev(yv)))
        op.check_device()
        assert rel(f, oracle.forward(g, s, K_or, c)) <= tol
        assert rel(a, oracle.adjoint(g, s, K_or, yv)) <= tol
    finally:
        op.close()


def test_two_step_matches_oracle():
    """The two-step approach (per-pulse acoustic inversion with TV, then
    unmixing with l1 + TV) against the oracle's, with the same steps: the
    acoustic images b and the concentrations c within the FISTA tolerance."""
    from dataclasses import replace
    g, s = TINY.geom, TINY.sw
    K = synth.transducer_kernel(g, seed=0)
    c_true = synth.tube_phantom(g, 4, seed=3)
    y = oracle.forward(g, s, K, c_true)
    y = y + 0.02 * np.abs(y).max() * synth.gaussian(g.y_shape(), 11)
    g1 = replace(g, N=1, P=1, pulses_per_cycle=1)
    s1 = Switching((0.0,), (0.0,), (1.0,), 0.0)
    L1 = oracle.power(g1, s1, K, synth.gaussian(g1.c_shape(), 12), 60)
    S = oracle.switch_matrix(g, s)
    L2 = max(np.linalg.norm(S[:, :, j], 2) ** 2 for j in range(g.Z))
    a1, a2 = 0.9 / L1, 0.9 / L2
    acoustic = sw.SolveParams(step=a1, lambda_l1=0.0, lambda_tv=2e-3, inner_iters=10,
                              max_iters=20)
    unmixing = sw.SolveParams(step=a2, lambda_l1=1e-3, lambda_tv=1e-3, inner_iters=10,
                              max_iters=20)
    c, b = sw.two_step(g, K, s, dev(y), acoustic, unmixing)
    torch.cuda.synchronize()
    c_or, b_or = oracle.two_step(g, s, K, y, a1, 20, 0.0, 2e-3, 10, a2, 20, 1e-3, 1e-3, 10)
    assert rel(host(b), b_or) <= 1e-4
    assert rel(host(c), c_or) <= 1e-4


def _joint_step2(g, s, lam_tv, lam_l1, lam_b):
    """1 / a bound of eig_max(L L^T): 12 lam_tv^2 + lam_l1^2 + 12 lam_b^2 sum_n
    max_j sum_p S[n][p][j]^2 (the oracle's S)."""
    S = oracle.switch_matrix(g, s)
    return 1.0 / (12 * lam_tv ** 2 + lam_l1 ** 2 +
                  12 * lam_b ** 2 * float(np.sum(np.max(np.sum(S ** 2, axis=1), axis=1))))


@pytest.mark.parametrize("lams,shift,inplace", [((0.3, 0.1, 0.2), 0.5, False),
                                                ((0.0, 0.0, 0.4), 0.5, False),
                                                ((0.25, 0.15, 0.0), 0.5, False),
                                                ((0.2, 0.05, 0.5), -0.2, False),
                                                ((0.2, 0.05, 0.5), -0.2, True)])
def test_prox_joint_matches_oracle(lams, shift, inplace):
    """The prox of the full R3 with its lambda_3 term (TV of every pulse
    image) and the nonnegativity constraint, Algorithm 2 on the constrained
    dual with a fixed iteration count, against the oracle's iterates: pulses
    fold onto 3 switching states on the GPU (one dual per state) and keep one
    dual each in the oracle; outputs clip at zero (many of them with the
    negative shift); in place (x = z) gives the same result."""
    g = Geometry(X=7, Y=5, Z=6, T=8, N=5, P=2, k=3, pulses_per_cycle=3)
    s = Switching((0.2, 0.0), (1.0, 0.0), (0.05, 1.0), 3.0)
    K = np.random.default_rng(60).standard_normal(g.k_shape())
    lam_tv, lam_l1, lam_b = lams
    step2 = _joint_step2(g, s, lam_tv, lam_l1, lam_b)
    z = np.random.default_rng(61).standard_normal(g.c_shape()) + shift
    op = sw.Operator(g, K, s)
    try:
        assert op.prox_joint_step_bound(lam_tv, lam_l1, lam_b) == pytest.approx(1 / step2,
                                                                                 rel=1e-12)
        zt = dev(z)
        got = op.prox_joint(zt, 0.6, lam_tv, lam_l1, lam_b, 40, step2,
                            out=zt if inplace else None)
        if inplace:
            assert got.data_ptr() == zt.data_ptr()
        got = host(got)
        op.check_device()
    finally:
        op.close()
    want = oracle.prox_joint(g, s, z, 0.6, lam_tv, lam_l1, lam_b, 40, step2)
    assert (want == 0).any() and (want > 0).any()
    if shift < 0:
        assert (want == 0).mean() > 0.3
    assert rel(got, want) <= 1e-5


@pytest.mark.parametrize("mode", ["fp32", "refined_bf16"])
def test_fista_with_lambda3_matches_oracle(cases, mode):
    """Algorithm 1 with all three terms of R3 on the tiny workload: 20
    iterations, lambda_3 = 2e-3 with the workload's other weights, the joint
    prox with the workload's inner iteration count, the same alpha and dual
    step on both sides; FP32, and the refined BF16 schedule."""
    g, s, K, _ = cases["tiny"]
    y = _tiny_measurements(g, s, K)
    L = oracle.power(g, s, K, synth.gaussian(g.c_shape(), 1), 100)
    alpha = 1.0 / L
    lam_3 = 2e-3
    step2 = _joint_step2(g, s, TINY.lam_tv, TINY.lam_l1, lam_3)
    extra = sw.REFINED_DEFAULTS if mode == "refined_bf16" else {}
    op = sw.Operator(g, K, s, precision="bf16" if mode == "refined_bf16" else "fp32")
    try:
        params = sw.SolveParams(step=alpha, lambda_l1=TINY.lam_l1, lambda_tv=TINY.lam_tv,
                                inner_iters=TINY.inner, max_iters=TINY.iters, lambda_3=lam_3,
                                joint_step2=step2, **extra)
        got, stats = op.solve(dev(y), params)
        op.check_device()
    finally:
        op.close()
    ref = oracle.fista(g, s, K, y, alpha, TINY.iters, TINY.lam_l1, TINY.lam_tv, TINY.inner,
                       lam_3=lam_3, joint_step2=step2)
    assert stats["iters"] == TINY.iters
    assert rel(host(got), ref) <= 1e-4
    F_ref, _ = oracle.objective(g, s, K, ref, y, TINY.lam_l1, TINY.lam_tv, lam_3)
    assert stats["objective"] == pytest.approx(F_ref, rel=1e-4)
    # the lambda_3 term matters at this weight
    plain = oracle.fista(g, s, K, y, alpha, TINY.iters, TINY.lam_l1, TINY.lam_tv, TINY.inner)
    assert rel(plain, ref) > 1e-3


def test_objective_with_lambda3_matches_oracle(cases):
    g, s, K, op = cases["tiny"]
    rng = np.random.default_rng(62)
    c = np.maximum(rng.standard_normal(g.c_shape()), 0)
    y = rng.standard_normal(g.y_shape())
    F, fit = op.objective(dev(c), dev(y), 0.05, 0.07, 0.09)
    F_ref, fit_ref = oracle.objective(g, s, K, c, y, 0.05, 0.07, 0.09)
    assert F == pytest.approx(F_ref, rel=1e-5)
    assert fit == pytest.approx(fit_ref, rel=1e-5)


def test_tensor_core_accumulators_option(tc_cases):
    """One accumulator per tile (corrections summed with the main products)
    stays within the split tolerance; two is the default of the split mode."""
    g, s, K = tc_cases["ragged"]
    c = np.random.default_rng(40).standard_normal(g.c_shape())
    want = oracle.forward(g, s, K, c)
    for acc in (1, 2):
        op = sw.Operator(g, K, s)
        op.tc_configure(0, accumulators=acc)
        op.tc_configure(1, accumulators=acc)
        op.set_precision("bf16x3")
        assert op.tc_config(0)["accumulators"] == acc
        assert rel(host(op.forward(dev(c))), want) <= TC_TOL["bf16x3"]
        op.close()
    op = sw.Operator(g, K, s, precision="bf16x3")
    assert op.tc_config(0)["accumulators"] == 2 and op.tc_config(1)["accumulators"] == 2
    op.close()


# ---------------------------------------------------------------------------
# Differentiation (tiny workload's shapes, FP32 on the GPU against FP64 on the
# CPU): the autograd function around H gives the gradient of
# 1/2 ||H(kappa, mu) c - y||^2 with respect to c, kappa and mu.  References:
# the oracle's adjoint and parameter gradient, and central differences of the
# oracle's data fit (h = 1e-4, FP64).
# ---------------------------------------------------------------------------
def test_hfunction_gradients_match_oracle_and_central_differences():
    g, s = TINY.geom, TINY.sw
    K = synth.transducer_kernel(g, seed=0)
    op = sw.Operator(g, K, s)
    rng = np.random.default_rng(50)
    c = synth.tube_phantom(g, TINY.tubes, seed=3, per_species=True) + 0.05
    y = oracle.forward(g, s, K, c * 1.05) + 0.02 * rng.standard_normal(g.y_shape())
    kappa = torch.tensor(s.kappa, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(s.mu_per_mm, dtype=torch.float64, requires_grad=True)
    ct = dev(c).requires_grad_(True)
    yt = dev(y)
    H = sw.HFunction
    assert H is sw.HFunction  # one class, created once
    loss = 0.5 * (H.apply(ct, kappa, mu, op).double() - yt.double()).pow(2).sum()
    loss.backward()
    # c: H^T (H c - y)
    gc_ref = oracle.adjoint(g, s, K, oracle.forward(g, s, K, c) - y)
    assert rel(host(ct.grad), gc_ref) <= 1e-5
    # kappa, mu: the oracle's gradient and central differences
    dk_ref, dmu_ref = oracle.param_grad(g, s, K, c, y)

    def fit(kap, m):
        s2 = synth.Switching(tuple(kap), s.eps_bar, s.eps_off, m)
        return 0.5 * np.sum((oracle.forward(g, s2, K, c) - y) ** 2)

    h = 1e-4
    kp = list(s.kappa)
    for p in range(g.P):
        a, b = list(kp), list(kp)
        a[p] += h
        b[p] -= h
        fd = (fit(a, s.mu_per_mm) - fit(b, s.mu_per_mm)) / (2 * h)
        if abs(dk_ref[p]) > 0:
            assert dk_ref[p] == pytest.approx(fd, rel=1e-5)  # O(h^2) truncation
            assert kappa.grad[p].item() == pytest.approx(dk_ref[p], rel=1e-4)
        else:
            assert abs(kappa.grad[p].item()) <= 1e-6 * max(abs(fd), 1.0)
    fd = (fit(kp, s.mu_per_mm + h) - fit(kp, s.mu_per_mm - h)) / (2 * h)
    assert dmu_ref == pytest.approx(fd, rel=1e-5)
    assert mu.grad.item() == pytest.approx(dmu_ref, rel=1e-4)
    # c along random directions: the data fit's central difference
    for seed in range(3):
        v = np.random.default_rng(60 + seed).standard_normal(g.c_shape())
        fdc = (0.5 * np.sum((oracle.forward(g, s, K, c + h * v) - y) ** 2) -
               0.5 * np.sum((oracle.forward(g, s, K, c - h * v) - y) ** 2)) / (2 * h)
        assert float(np.sum(host(ct.grad) * v)) == pytest.approx(fdc, rel=1e-4)
    op.close()


def test_param_vjp_and_set_switching(cases):
    """<w, dH/dtheta c> for an arbitrary cotangent equals param_grad with
    y = H c - w; a changed kappa / mu changes the operator like a new handle."""
    g, s, K, op = cases["ragged"]
    rng = np.random.default_rng(51)
    c = np.abs(rng.standard_normal(g.c_shape()))
    w = rng.standard_normal(g.y_shape())
    dk, dmu = op.param_vjp(dev(c), dev(w))
    dk2, dmu2 = op.param_grad(dev(c), dev(oracle.forward(g, s, K, c) - w))
    np.testing.assert_allclose(dk, dk2, rtol=1e-4, atol=1e-9 * np.abs(dk2).max())
    assert dmu == pytest.approx(dmu2, rel=1e-4)
    s2 = synth.Switching(tuple(k * 1.7 for k in s.kappa), s.eps_bar, s.eps_off, s.mu_per_mm * 0.6)
    fresh = sw.Operator(g, K, s2)
    ref = host(fresh.forward(dev(c)))
    fresh.close()
    try:
        op.set_switching(kappa=s2.kappa, mu=s2.mu_per_mm)
        assert np.array_equal(host(op.forward(dev(c))), ref)
        assert rel(ref, oracle.forward(g, s2, K, c)) <= 1e-5
    finally:
        op.set_switching(kappa=s.kappa, mu=s.mu_per_mm)
    assert rel(host(op.forward(dev(c))), oracle.forward(g, s, K, c)) <= 1e-5


# ---------------------------------------------------------------------------
# Batched uneven problems: one graph per iteration; the contractions of all
# problems run as persistent launches over every problem's tile-states
# (shared), or every problem's kernels on a stream of its own.  The iterates
# are those of each handle stepped alone (a stream per problem: bitwise, the
# same kernels in the same order; shared: to FP32 summation order) and match
# the oracle's.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec,refine,budget,shared", [("fp32", 0, 0.0, True),
                                                       ("bf16", 3, 0.0, True),
                                                       ("bf16", 3, 0.0, False),
                                                       ("bf16", 25, 0.1, True),
                                                       ("bf16x3", 0, 0.0, True)])
def test_batch_equals_separate_solves(prec, refine, budget, shared):
    names = ["tiny", "ragged", "pulses_below_cycle", "support_wider_than_grid"]
    ops, ys, prms, refs = [], [], [], []
    for i, name in enumerate(names):
        g, s, seed = CASES[name]
        K = _kernel(g, seed)
        op = sw.Operator(g, K, s, precision=prec)
        if prec != "fp32":
            for kid in (0, 1):
                op.tc_schedule(kid, split=1)
        yn = np.random.default_rng(70 + i).standard_normal(g.y_shape())
        y = dev(yn)
        alpha = 0.9 / op.lipschitz(20)
        prm = sw.SolveParams(step=alpha, max_iters=9, lambda_l1=0.01,
                             lambda_tv=0.01, inner_iters=4, refine_every=refine,
                             refine_precision="bf16x3", refine_budget=budget)
        op.fista_init(y, prm)
        ops.append(op)
        ys.append(y)
        prms.append(prm)
        refs.append(oracle.fista(g, s, K, yn, alpha, 9, 0.01, 0.01, 4))
    b = sw.Batch(ops, shared=shared)
    b.step(4)
    b.step(5)
    assert b.shared_in_use() == (shared and prec != "fp32")
    if b.shared_in_use():
        assert 2 <= b.contraction_launches() < 2 * len(ops)
    got = [op.fista_get().clone() for op in ops]
    for op in ops:
        op.check_device()
    # the oracle's iterates: FP32, bf16x3 and the budget schedule to 1e-4; a
    # fixed resync every third iteration leaves the BF16 increments of two
    # large early steps in between (1e-3)
    tol = 1e-3 if (prec == "bf16" and budget == 0.0) else 1e-4
    for c, ref in zip(got, refs):
        assert rel(host(c), ref) <= tol
    # stepping one handle alone desynchronises the batch
    ops[0].fista_step(1)
    with pytest.raises(sw.SwoptError):
        b.step(1)
    b.close()
    # the same handles (same tuned tile configurations, hence the same FP32
    # summation order on the tensor cores) stepped one by one
    # (a shared launch splits tile-states between CTAs where the handle's own
    # launches take them whole: the same sums in another FP32 order)
    for op, y, prm, c in zip(ops, ys, prms, got):
        op.fista_init(y, prm)
        op.fista_step(9)
        if shared and prec != "fp32":
            assert rel(host(op.fista_get()), host(c)) <= 1e-5
        else:
            assert torch.equal(op.fista_get(), c)
        op.close()


@pytest.mark.parametrize("shape", [(2, 48, 48, 256), (3, 45, 53, 203), (1, 1500, 1300, 1),
                                   (2, 1, 4000, 280)])
def test_prox_and_fista_on_a_volume_beyond_shared_memory(shape):
    """Volumes whose TV prox state (8 floats per entry) exceeds the shared
    memory of all SMs together (about 35 MB), so the prox runs as the
    cooperative kernel on global memory: 8 x 8 x 32 tiles that divide the
    volume, ragged ones in every axis, a single depth and a single row.
    Prox and a short FISTA solve match the oracle."""
    P, Y, X, Z = shape
    g = Geometry(X=X, Y=Y, Z=Z, T=32, N=2, P=P, k=3, pulses_per_cycle=2)
    sw_p = [0.2] + [0.0] * (P - 1)
    s = Switching(tuple(sw_p), tuple([1.0] + [0.0] * (P - 1)), tuple([0.0] + [1.0] * (P - 1)),
                  1.0)
    K = np.random.default_rng(80).standard_normal(g.k_shape())
    K[..., :8] = 0.0
    op = sw.Operator(g, K, s)
    z = np.random.default_rng(81).standard_normal(g.c_shape())
    got = host(op.prox_tv(dev(z), 0.15, 10))
    assert rel(got, oracle.prox_tv(z, 0.15, 10)) <= 1e-5
    if Y * X * Z > 600_000:
        op.close()
        return  # the solve's oracle would take minutes; the prox covers the kernel
    y = np.random.default_rng(82).standard_normal(g.y_shape())
    alpha = 0.5 / oracle.power(g, s, K, synth.gaussian(g.c_shape(), 83), 30)
    params = sw.SolveParams(step=alpha, lambda_l1=0.01, lambda_tv=0.05, inner_iters=6,
                            max_iters=4)
    c, _ = op.solve(dev(y), params)
    op.check_device()
    ref = oracle.fista(g, s, K, y, alpha, 4, 0.01, 0.05, 6)
    assert rel(host(c), ref) <= 1e-4
    op.close()
