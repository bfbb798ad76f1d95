"""Pins of the FP64 oracle to things other than itself.

Each test ties one oracle function to an independent fact: a library
routine (torch conv2d / conv_transpose2d, numpy eigvalsh, scipy's L-BFGS-B
on the exact convex problem), a mathematical identity (the adjoint
identity, optimality conditions), a closed form or a finite difference.
Chosen so that a dropped term, a wrong sign, a swapped index or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.optimize
import torch

import oracle
import synth
from synth import Geometry, Switching

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _geom(**kw):
    base = dict(X=7, Y=6, Z=5, T=12, N=4, P=2, k=3, pulses_per_cycle=3)
    base.update(kw)
    return Geometry(**base)


def _sw(P, kappa=None, mu=2.0):
    kap = list(kappa) if kappa is not None else [0.3 * (p + 1) for p in range(P - 1)] + [0.0]
    eb = [1.0] * (P - 1) + [0.0]
    eo = [0.05] * (P - 1) + [1.0]
    return Switching(kappa=tuple(kap), eps_bar=tuple(eb), eps_off=tuple(eo), mu_per_mm=mu)


def _rand_kernel(g, seed):
    # an asymmetric random kernel: catches dy/dx/t index swaps
    return np.random.default_rng(seed).standard_normal(g.k_shape())


def _dense_H(g, sw, K):
    nc = int(np.prod(g.c_shape()))
    cols = []
    for i in range(nc):
        e = np.zeros(nc)
        e[i] = 1.0
        cols.append(oracle.forward(g, sw, K, e.reshape(g.c_shape())).ravel())
    return np.stack(cols, axis=1)


# --------------------------------------------------------------------------
# Forward / adjoint (Sec. 2.3.3, Eq. acoustic-full-forward, Eq. full-forward)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 3, 5])
def test_forward_is_conv2d_for_one_pulse_background(k):
    """N=1, P=1 background, Phi=1: H is torch's conv2d (cross-correlation)
    with C_in = Z depths, C_out = T samples, a k x k filter and zero padding."""
    g = _geom(N=1, P=1, k=k, X=9, Y=8, Z=4, T=10, pulses_per_cycle=1)
    sw = Switching(kappa=(0.0,), eps_bar=(0.0,), eps_off=(1.0,), mu_per_mm=0.0)
    K = _rand_kernel(g, 1)
    c = np.random.default_rng(2).standard_normal(g.c_shape())
    y = oracle.forward(g, sw, K, c)
    w = torch.from_numpy(K).permute(3, 0, 1, 2).contiguous()  # [T][Z][ky][kx]
    inp = torch.from_numpy(c[0]).permute(2, 0, 1)[None]       # [1][Z][Y][X]
    ref = torch.nn.functional.conv2d(inp, w, padding=k // 2)[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(y[0], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_adjoint_is_conv_transpose2d_for_one_pulse_background(k):
    g = _geom(N=1, P=1, k=k, X=9, Y=8, Z=4, T=10, pulses_per_cycle=1)
    sw = Switching(kappa=(0.0,), eps_bar=(0.0,), eps_off=(1.0,), mu_per_mm=0.0)
    K = _rand_kernel(g, 3)
    yv = np.random.default_rng(4).standard_normal(g.y_shape())
    c = oracle.adjoint(g, sw, K, yv)
    w = torch.from_numpy(K).permute(3, 0, 1, 2).contiguous()
    inp = torch.from_numpy(yv[0]).permute(2, 0, 1)[None]      # [1][T][Y][X]
    ref = torch.nn.functional.conv_transpose2d(inp, w, padding=k // 2)[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(c[0], ref, rtol=1e-12, atol=1e-12)


def test_adjoint_identity_random_pairs():
    """<Hx, y> = <x, H^T y> for 100 seeded N(0,1) pairs (full switching)."""
    g = _geom()
    sw = _sw(g.P)
    K = _rand_kernel(g, 5)
    rng = np.random.default_rng(6)
    worst = 0.0
    for _ in range(100):
        x = rng.standard_normal(g.c_shape())
        yv = rng.standard_normal(g.y_shape())
        hx = oracle.forward(g, sw, K, x)
        lhs = float(np.vdot(hx, yv))
        rhs = float(np.vdot(x, oracle.adjoint(g, sw, K, yv)))
        # scale: the Cauchy-Schwarz bound of either side
        worst = max(worst, abs(lhs - rhs) / (np.linalg.norm(hx) * np.linalg.norm(yv)))
    assert worst < 1e-13


def test_adjoint_identity_tiny_workload_kernel():
    prob = synth.workload("tiny_16x16x24_T64_k7_N8_P2")
    g = prob.geom
    K = synth.transducer_kernel(g)
    rng = np.random.default_rng(7)
    for _ in range(3):
        x = rng.standard_normal(g.c_shape())
        yv = rng.standard_normal(g.y_shape())
        lhs = float(np.vdot(oracle.forward(g, prob.sw, K, x), yv))
        rhs = float(np.vdot(x, oracle.adjoint(g, prob.sw, K, yv)))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _dense_H_definition(g, sw, K):
    """H entry by entry from Eq. (final-H) and the per-depth lateral
    correlation (Eq. acoustic-full-forward): row (n, y, x, t), column
    (p, y', x', j) holds S[n][p][j] K[j][y' - y + r][x' - x + r][t] for
    |y' - y|, |x' - x| <= r (pulse n's image b^n = sum_p S[n][p] c_p, read at
    the scan position shifted by the tap), else 0."""
    S = oracle.switch_matrix(g, sw)
    r = g.k // 2
    H = np.zeros((int(np.prod(g.y_shape())), int(np.prod(g.c_shape()))))
    for n in range(g.N):
        for y in range(g.Y):
            for x in range(g.X):
                for t in range(g.T):
                    row = ((n * g.Y + y) * g.X + x) * g.T + t
                    for p in range(g.P):
                        for yy in range(max(0, y - r), min(g.Y, y + r + 1)):
                            for xx in range(max(0, x - r), min(g.X, x + r + 1)):
                                for j in range(g.Z):
                                    col = ((p * g.Y + yy) * g.X + xx) * g.Z + j
                                    H[row, col] = S[n, p, j] * K[j, yy - y + r, xx - x + r, t]
    return H


def test_dense_forward_matches_the_entrywise_definition():
    """The oracle's forward, column by column, equals H assembled entry by
    entry from its definition (a ragged grid, a support wider than it on one
    axis, an asymmetric kernel, several pulses on a partial cycle)."""
    g = _geom(X=4, Y=3, Z=3, T=5, N=4, P=2, k=5, pulses_per_cycle=3)
    sw = _sw(g.P)
    K = _rand_kernel(g, 9)
    np.testing.assert_allclose(_dense_H(g, sw, K), _dense_H_definition(g, sw, K), rtol=0,
                               atol=1e-13)


def test_dense_adjoint_is_transpose():
    g = _geom(X=4, Y=3, Z=3, T=6, N=3, P=2, k=3)
    sw = _sw(g.P)
    K = _rand_kernel(g, 8)
    H = _dense_H_definition(g, sw, K)
    ny = int(np.prod(g.y_shape()))
    rows = []
    for i in range(ny):
        e = np.zeros(ny)
        e[i] = 1.0
        rows.append(oracle.adjoint(g, sw, K, e.reshape(g.y_shape())).ravel())
    HT = np.stack(rows, axis=1)
    np.testing.assert_allclose(HT, H.T, rtol=0, atol=1e-13)


def test_point_absorber_reproduces_kernel_background():
    """A unit background absorber at (y0, x0, j) gives
    y[n, y0-dy, x0-dx, t] = Phi_j K[j, dy, dx, t] for every pulse, and zero
    elsewhere: pins the correlation sign and the fluence prefactor."""
    g = _geom(X=9, Y=9, Z=4, T=8, N=5, P=2, k=5, pulses_per_cycle=5)
    sw = _sw(g.P, mu=3.0)
    K = _rand_kernel(g, 9)
    y0, x0, j = 4, 3, 2
    c = np.zeros(g.c_shape())
    c[g.P - 1, y0, x0, j] = 1.0
    y = oracle.forward(g, sw, K, c)
    phi_j = math.exp(-sw.mu_per_mm * j * g.dz_mm)
    expect = np.zeros(g.y_shape())
    r = g.r
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            expect[:, y0 - dy, x0 - dx, :] = phi_j * K[j, dy + r, dx + r, :]
    np.testing.assert_allclose(y, expect, rtol=0, atol=1e-14)


def test_point_absorber_switching_decay():
    """A switchable absorber decays geometrically within each cycle by the
    factor exp(-kappa Phi_j) per pulse and restarts at each new cycle."""
    g = _geom(X=5, Y=5, Z=6, T=8, N=9, P=2, k=3, pulses_per_cycle=3)
    sw = Switching(kappa=(0.4, 0.0), eps_bar=(1.0, 0.0), eps_off=(0.0, 1.0), mu_per_mm=5.0)
    K = np.abs(_rand_kernel(g, 10)) + 0.1
    for j in (0, 3, 5):
        c = np.zeros(g.c_shape())
        c[0, 2, 2, j] = 1.0
        y = oracle.forward(g, sw, K, c)[:, 2, 2, :]
        phi = math.exp(-sw.mu_per_mm * j * g.dz_mm)
        for n in range(g.N - 1):
            ratio = y[n + 1] / y[n]
            if (n + 1) % g.pulses_per_cycle == 0:
                np.testing.assert_allclose(y[n + 1], y[n + 1 - g.pulses_per_cycle], rtol=1e-13)
            else:
                np.testing.assert_allclose(ratio, math.exp(-0.4 * phi), rtol=1e-12)
    # background: constant over pulses, decays with depth by exp(-mu dz) per layer
    ys = []
    for j in range(g.Z):
        c = np.zeros(g.c_shape())
        c[1, 2, 2, j] = 1.0
        y = oracle.forward(g, sw, K, c)[:, 2, 2, :]
        np.testing.assert_allclose(y, np.broadcast_to(y[0], y.shape), rtol=1e-14)
        ys.append(y[0] / K[j, 1, 1, :])
    for j in range(g.Z - 1):
        np.testing.assert_allclose(ys[j + 1] / ys[j], math.exp(-sw.mu_per_mm * g.dz_mm), rtol=1e-12)


def test_linearity_and_shift_invariance():
    g = _geom(X=10, Y=10, Z=3, T=6, N=3, P=2, k=3)
    sw = _sw(g.P)
    K = _rand_kernel(g, 11)
    rng = np.random.default_rng(12)
    a, b = 0.7, -1.3
    x1 = rng.standard_normal(g.c_shape())
    x2 = rng.standard_normal(g.c_shape())
    lhs = oracle.forward(g, sw, K, a * x1 + b * x2)
    rhs = a * oracle.forward(g, sw, K, x1) + b * oracle.forward(g, sw, K, x2)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    c = np.zeros(g.c_shape())
    c[0, 4, 4, 1] = 1.0
    c2 = np.zeros(g.c_shape())
    c2[0, 5, 3, 1] = 1.0
    y1 = oracle.forward(g, sw, K, c)
    y2 = oracle.forward(g, sw, K, c2)
    np.testing.assert_allclose(y2[:, 2:9, 0:7], y1[:, 1:8, 1:8], atol=1e-15)


def test_sampled_forward_and_adjoint_match_full():
    g = _geom(X=8, Y=7, Z=4, T=9, N=5, P=3, k=5, pulses_per_cycle=2)
    sw = _sw(g.P)
    K = _rand_kernel(g, 13)
    rng = np.random.default_rng(14)
    c = rng.standard_normal(g.c_shape())
    yv = rng.standard_normal(g.y_shape())
    y = oracle.forward(g, sw, K, c)
    idx = np.array([[n, yy, xx] for n in range(g.N) for yy in (0, 3, 6) for xx in (0, 7)])
    np.testing.assert_allclose(oracle.forward_at(g, sw, K, c, idx), y[idx[:, 0], idx[:, 1], idx[:, 2]],
                               rtol=1e-13, atol=1e-13)
    a = oracle.adjoint(g, sw, K, yv)
    idx4 = np.array([[p, yy, xx, j] for p in range(g.P) for yy in (0, 6) for xx in (1, 7) for j in (0, 3)])
    np.testing.assert_allclose(oracle.adjoint_at(g, sw, K, yv, idx4),
                               a[idx4[:, 0], idx4[:, 1], idx4[:, 2], idx4[:, 3]], rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------
# TV, proximal maps (Eq. prox, Eq. prox-dual, Algorithm 2)
# --------------------------------------------------------------------------

def test_grad3_transpose_and_ramp():
    rng = np.random.default_rng(15)
    v = rng.standard_normal((4, 5, 6))
    gg = rng.standard_normal((3, 4, 5, 6))
    assert abs(np.vdot(oracle.grad3(v), gg) - np.vdot(v, oracle.grad3T(gg))) < 1e-12
    yy, xx, zz = np.meshgrid(np.arange(4), np.arange(5), np.arange(6), indexing="ij")
    ramp = 2.0 * yy - 3.0 * xx + 0.5 * zz
    d = oracle.grad3(ramp)
    assert np.allclose(d[0, :-1], 2.0) and np.allclose(d[0, -1], 0.0)
    assert np.allclose(d[1, :, :-1], -3.0) and np.allclose(d[1, :, -1], 0.0)
    assert np.allclose(d[2, :, :, :-1], 0.5) and np.allclose(d[2, :, :, -1], 0.0)


def test_tv_of_step_is_jump_times_interface():
    c = np.zeros((1, 4, 6, 5))
    c[0, :, 3:, :] = 2.5
    assert oracle.tv(c) == pytest.approx(2.5 * 4 * 5, rel=1e-15)


def test_l1_prox_closed_form_against_scalar_minimiser():
    rng = np.random.default_rng(16)
    z = rng.standard_normal(40) * 2
    theta = 0.7
    for nonneg in (True, False):
        x = oracle.prox_l1(z, theta, nonneg)
        for zi, xi in zip(z, x):
            lo = 0.0 if nonneg else -10.0
            res = scipy.optimize.minimize_scalar(lambda t: 0.5 * (t - zi) ** 2 + theta * abs(t),
                                                 bounds=(lo, 10.0), method="bounded",
                                                 options={"xatol": 1e-12})
            assert abs(res.x - xi) < 1e-6


def _dual_tv_exact(z, tau, theta=None):
    """Exact prox via the dual, solved by scipy's L-BFGS-B with box bounds.

    TV only:         min_{|u|<=tau} 1/2 ||z - D^T u||^2,        x = z - D^T u
    TV + l1 + (>=0): min_{|u|<=tau} 1/2 ||max(z - theta - D^T u, 0)||^2,
                                                                  x = max(z - theta - D^T u, 0)
    D is assembled here as an explicit sparse difference matrix.
    """
    import scipy.sparse as sp
    Y, X, Z = z.shape
    L = Y * X * Z
    idx = np.arange(L).reshape(Y, X, Z)
    rows, cols, vals = [], [], []
    e = 0
    blocks = []
    for axis in range(3):
        a = np.moveaxis(idx, axis, 0)
        lo = a[:-1].ravel()
        hi = a[1:].ravel()
        m = lo.size
        blocks.append((lo, hi, m))
    # one dual entry per (axis, voxel); unused entries (last along the axis) have a zero row
    D = sp.lil_matrix((3 * L, L))
    for axis in range(3):
        a = np.moveaxis(idx, axis, 0)
        lo = a[:-1].ravel()
        hi = a[1:].ravel()
        for l_, h_ in zip(lo, hi):
            D[axis * L + l_, h_] = 1.0
            D[axis * L + l_, l_] = -1.0
    D = D.tocsr()
    zf = z.ravel()

    if theta is None:
        def fun(u):
            w = zf - D.T @ u
            return 0.5 * w @ w, -(D @ w)
    else:
        def fun(u):
            w = np.maximum(zf - theta - D.T @ u, 0.0)
            return 0.5 * w @ w, -(D @ w)
    res = scipy.optimize.minimize(fun, np.zeros(3 * L), jac=True, method="L-BFGS-B",
                                  bounds=[(-tau, tau)] * (3 * L),
                                  options={"maxiter": 20000, "ftol": 1e-16, "gtol": 1e-13,
                                           "maxcor": 50})
    u = res.x
    if theta is None:
        return (zf - D.T @ u).reshape(z.shape)
    return np.maximum(zf - theta - D.T @ u, 0.0).reshape(z.shape)


def test_tv_prox_3d_matches_exact_dual_solution():
    rng = np.random.default_rng(17)
    z = rng.standard_normal((3, 4, 5))
    tau = 0.3
    exact = _dual_tv_exact(z, tau)
    fgp = oracle.prox_tv(z[None], tau, 4000)[0]
    np.testing.assert_allclose(fgp, exact, atol=2e-6)


def test_tv_prox_1d_optimality_conditions():
    """1D lines: x = prox_TV(z) iff z - x = tau D^T u with |u| <= 1 and
    u_i = sign(x_{i+1} - x_i) wherever the jump is nonzero."""
    rng = np.random.default_rng(18)
    for trial in range(4):
        Z = 14
        z = np.cumsum(rng.standard_normal(Z)) + rng.standard_normal(Z)
        tau = 0.4 + 0.3 * trial
        x = oracle.prox_tv(z.reshape(1, 1, 1, Z), tau, 30000)[0, 0, 0]
        w = (z - x) / tau
        assert abs(w.sum()) < 1e-8
        u = -np.cumsum(w)[:-1]  # (D^T u)_i = u_{i-1} - u_i
        assert np.all(np.abs(u) <= 1 + 1e-6)
        jump = np.diff(x)
        big = np.abs(jump) > 1e-5
        np.testing.assert_allclose(u[big], np.sign(jump[big]), atol=1e-5)


def test_tv_prox_special_cases():
    rng = np.random.default_rng(19)
    z = rng.standard_normal((2, 3, 4, 5))
    np.testing.assert_array_equal(oracle.prox_tv(z, 0.0, 10), z)  # tau = 0: identity
    const = np.full((1, 3, 4, 5), 1.7)
    np.testing.assert_array_equal(oracle.prox_tv(const, 0.5, 10), const)  # constant in, constant out
    big = oracle.prox_tv(z, 1e3, 6000)  # large tau: the per-species mean
    for p in range(2):
        np.testing.assert_allclose(big[p], z[p].mean(), atol=1e-6)


def test_composite_prox_equals_joint_prox():
    """max(prox_TV(z) - theta, 0) is the exact prox of TV + l1 + indicator(>= 0)
    (the joint dual of Eq. prox-dual solved to optimality)."""
    rng = np.random.default_rng(20)
    for trial in range(3):
        z = rng.standard_normal((3, 3, 4)) + 0.3
        tau, theta = 0.25 + 0.1 * trial, 0.2
        joint = _dual_tv_exact(z, tau, theta)
        comp = oracle.prox(z[None], 1.0, theta, tau, 4000)[0]
        np.testing.assert_allclose(comp, joint, atol=2e-6)


# --------------------------------------------------------------------------
# FISTA (Algorithm 1), power iteration, objective, parameter gradient
# --------------------------------------------------------------------------

def _small_problem(seed=21):
    """A small, reasonably conditioned problem (condition number ~1e3): a
    dominant on-axis tap at a distinct time per depth plus a random blur."""
    g = _geom(X=5, Y=4, Z=4, T=10, N=4, P=2, k=3, pulses_per_cycle=4)
    sw = Switching(kappa=(1.5, 0.0), eps_bar=(1.0, 0.0), eps_off=(0.0, 1.0), mu_per_mm=2.0)
    rng = np.random.default_rng(seed)
    K = 0.2 * np.abs(rng.standard_normal(g.k_shape()))
    for j in range(g.Z):
        K[j, 1, 1, 2 * j] += 1.0
    c_true = np.maximum(rng.standard_normal(g.c_shape()), 0)
    y = oracle.forward(g, sw, K, c_true) + 0.05 * rng.standard_normal(g.y_shape())
    return g, sw, K, y


def test_power_iteration_matches_dense_eigenvalue():
    g, sw, K, _ = _small_problem()
    H = _dense_H(g, sw, K)
    lam = np.linalg.eigvalsh(H.T @ H)[-1]
    v0 = synth.gaussian(g.c_shape(), 3)
    L = oracle.power(g, sw, K, v0, 3000)
    assert abs(L - lam) <= 1e-10 * lam


def test_objective_at_zero_and_components():
    g, sw, K, y = _small_problem()
    F, fit = oracle.objective(g, sw, K, np.zeros(g.c_shape()), y, 0.1, 0.2)
    assert F == pytest.approx(0.5 * float(np.sum(y * y)), rel=1e-14)
    c = np.zeros(g.c_shape())
    c[1, :, 2:, :] = 1.5  # TV = 1.5 * Y * Z, l1 = 1.5 * count
    F, fit = oracle.objective(g, sw, K, c, y, 0.1, 0.2)
    hc = oracle.forward(g, sw, K, c)
    exp_fit = 0.5 * float(np.sum((hc - y) ** 2))
    assert fit == pytest.approx(exp_fit, rel=1e-13)
    assert F - fit == pytest.approx(0.1 * 1.5 * c[1, :, 2:, :].size + 0.2 * 1.5 * g.Y * g.Z, rel=1e-13)


def test_fista_reaches_bound_constrained_qp_optimum():
    """lambda_TV = 0: min 1/2||Hc - y||^2 + lam sum(c), c >= 0 is a smooth
    bound-constrained QP; L-BFGS-B on the explicit matrix gives its optimum."""
    g, sw, K, y = _small_problem()
    H = _dense_H(g, sw, K)
    lam = 0.05
    yf = y.ravel()

    def fun(c):
        r = H @ c - yf
        return 0.5 * r @ r + lam * c.sum(), H.T @ r + lam

    res = scipy.optimize.minimize(fun, np.zeros(H.shape[1]), jac=True, method="L-BFGS-B",
                                  bounds=[(0, None)] * H.shape[1],
                                  options={"maxiter": 50000, "ftol": 1e-16, "gtol": 1e-12})
    Fstar = res.fun
    L = np.linalg.eigvalsh(H.T @ H)[-1]
    c = oracle.fista(g, sw, K, y, 1.0 / L, 3000, lam, 0.0, 0)
    F, _ = oracle.objective(g, sw, K, c, y, lam, 0.0)
    assert F - Fstar <= 1e-9 * abs(Fstar)
    assert np.linalg.norm(c.ravel() - res.x) <= 1e-4 * np.linalg.norm(res.x)


def test_ista_objective_is_monotone():
    g, sw, K, y = _small_problem()
    H = _dense_H(g, sw, K)
    L = np.linalg.eigvalsh(H.T @ H)[-1]
    _, hist = oracle.fista(g, sw, K, y, 1.0 / L, 60, 0.05, 0.0, 0, momentum="none", history=True)
    assert np.all(np.diff(hist) <= 1e-12 * np.abs(hist[:-1]))
    # with TV and a near-exact inner solve
    _, hist = oracle.fista(g, sw, K, y, 1.0 / L, 25, 0.05, 0.05, 600, momentum="none", history=True)
    assert np.all(np.diff(hist) <= 1e-7 * np.abs(hist[:-1]))


def test_fista_momentum_modes_differ_and_first_step_is_prox_gradient():
    g, sw, K, y = _small_problem()
    alpha = 0.01
    c1 = oracle.fista(g, sw, K, y, alpha, 1, 0.05, 0.02, 10)
    # one step from zero: c_1 = prox(alpha H^T y)
    z = alpha * oracle.adjoint(g, sw, K, y)
    np.testing.assert_allclose(c1, oracle.prox(z, alpha, 0.05, 0.02, 10), atol=1e-15)
    a = oracle.fista(g, sw, K, y, alpha, 5, 0.05, 0.02, 10, momentum="beck_teboulle")
    b = oracle.fista(g, sw, K, y, alpha, 5, 0.05, 0.02, 10, momentum="paper_printed")
    assert np.abs(a - b).max() > 0


def test_param_grad_matches_central_differences():
    g, sw, K, y = _small_problem(31)
    c = np.maximum(np.random.default_rng(32).standard_normal(g.c_shape()), 0) + 0.1
    dk, dmu = oracle.param_grad(g, sw, K, c, y)

    def f(sw_):
        _, fit = oracle.objective(g, sw_, K, c, y, 0.0, 0.0)
        return fit

    h = 1e-4
    for p in range(g.P - 1):
        kp = list(sw.kappa)
        kp[p] += h
        km = list(sw.kappa)
        km[p] -= h
        fd = (f(Switching(tuple(kp), sw.eps_bar, sw.eps_off, sw.mu_per_mm))
              - f(Switching(tuple(km), sw.eps_bar, sw.eps_off, sw.mu_per_mm))) / (2 * h)
        assert dk[p] == pytest.approx(fd, rel=1e-6)
    fd = (f(Switching(sw.kappa, sw.eps_bar, sw.eps_off, sw.mu_per_mm + h))
          - f(Switching(sw.kappa, sw.eps_bar, sw.eps_off, sw.mu_per_mm - h))) / (2 * h)
    assert dmu == pytest.approx(fd, rel=1e-6)


def test_incremental_gradient_fista_equals_algorithm_1():
    """The refined solve's recursion, written out in FP64 with the oracle's
    operators: the gradient at c_k kept and updated by H^T H (c_{k+1} - c_k),
    recomputed every R iterations, and the gradient at the momentum point
    taken as (1 + beta) G_{k+1} - beta G_k.  In exact arithmetic this is
    Algorithm 1, so it must reproduce the oracle's FISTA iterates."""
    g, sw, K, y = _small_problem()
    alpha, lam1, lamtv, inner, iters = 0.01, 0.05, 0.02, 10, 12

    def grad(c):
        return oracle.adjoint(g, sw, K, oracle.forward(g, sw, K, c) - y)

    for R in (1, 3, 1000):
        c = np.zeros(g.c_shape())
        G = grad(c)
        z = -alpha * G
        t = 1.0
        for k in range(iters):
            cn = oracle.prox(z, alpha, lam1, lamtv, inner)
            t1 = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            beta = (t - 1.0) / t1
            t = t1
            d = cn - c
            xi = cn + beta * d
            Gn = grad(cn) if (k + 1) % R == 0 else G + oracle.adjoint(
                g, sw, K, oracle.forward(g, sw, K, d))
            z = xi - alpha * ((1.0 + beta) * Gn - beta * G)
            c, G = cn, Gn
        ref = oracle.fista(g, sw, K, y, alpha, iters, lam1, lamtv, inner)
        assert np.linalg.norm(c - ref) <= 1e-12 * np.linalg.norm(ref), R


# --------------------------------------------------------------------------
# Paper-literal acoustic kernel (Sec. 2.3.1 "Acoustic Model", Eqs.
# q-above-final / q-below-final, discrete semicircles)
# --------------------------------------------------------------------------

def _shell_mask(Z, k, T, dims, rho, kf, tf):
    """The oracle's mask: eta = 1 and a unit impulse response."""
    return oracle.semicircle_kernel(Z, k, T, dims, rho, kf, tf, np.ones((Z, k, k)),
                                    np.array([1.0])) != 0.0


def _brute_meets(lo, hi, n):
    """Does the closed box [lo, hi] hold a point at distance exactly n from 0?
    |p|^2 - n^2 evaluated on a grid of each box: every corner, a 9-point
    subdivision of each edge, and 0 on every axis the box spans (where the
    minimum of |p| lies); continuity on the connected box does the rest."""
    axes = []
    for a in range(3):
        pts = set(np.linspace(lo[a], hi[a], 9).tolist())
        if lo[a] <= 0.0 <= hi[a]:
            pts.add(0.0)
        axes.append(np.array(sorted(pts)))
    f = (axes[0][:, None, None] ** 2 + axes[1][None, :, None] ** 2
         + axes[2][None, None, :] ** 2 - n * n)
    return f.min() <= 0.0 <= f.max()


@pytest.mark.parametrize("dims,rho,kf", [(2, 1.0, 4.0), (2, 2.0, 3.5), (3, 1.0, 3.5),
                                          (3, 2.0, 4.0)])
def test_semicircle_mask_matches_brute_force(dims, rho, kf):
    """Voxel by voxel and sample by sample against the definition, evaluated
    by brute force on each (clipped) box."""
    Z, k, T, tf = 9, 7, 20, 10
    M = _shell_mask(Z, k, T, dims, rho, kf, tf)
    r = k // 2
    for j in range(Z):
        for iy in range(k):
            for ix in range(k):
                dy, dx = iy - r, ix - r
                for t in range(T):
                    want = False
                    if dims == 3 or dy == 0:
                        lo = [(dx - 0.5) * rho, (dy - 0.5) * rho if dims == 3 else 0.0,
                              j - kf - 0.5]
                        hi = [(dx + 0.5) * rho, (dy + 0.5) * rho if dims == 3 else 0.0,
                              j - kf + 0.5]
                        if t < tf:
                            hi[2] = min(hi[2], 0.0)
                        if t > tf:
                            lo[2] = max(lo[2], 0.0)
                        want = lo[2] <= hi[2] and _brute_meets(lo, hi, float(abs(t - tf)))
                    assert M[j, iy, ix, t] == want, (j, dy, dx, t)


def test_semicircle_points_on_the_sphere_lie_in_the_mask():
    """Random points exactly on the half sphere of sample t (away from voxel
    faces) fall in voxels of the mask, on the side of the focus that the
    sample sees: above the focus before the focal sample, below after."""
    Z, k, T, tf, kf, rho = 13, 11, 26, 13, 6.0, 1.0
    M = _shell_mask(Z, k, T, 3, rho, kf, tf)
    r = k // 2
    rng = np.random.default_rng(5)
    hits = 0
    for t in range(T):
        n = abs(t - tf)
        if n == 0 or n > 5:
            continue
        u = rng.standard_normal((400, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        p = n * u
        p[:, 2] = -np.abs(p[:, 2]) if t < tf else np.abs(p[:, 2])
        cell = p / np.array([rho, rho, 1.0])
        idx = np.rint(cell)
        away = np.all(np.abs(np.abs(cell - idx) - 0.5) > 1e-6, axis=1)
        for (x, y, z), ok in zip(idx.astype(int), away):
            if not ok:
                continue
            j = z + int(kf)
            assert M[j, y + r, x + r, t], (t, x, y, z)
            hits += 1
    assert hits > 1000


def test_semicircle_sources_above_focus_arrive_before_it():
    """One source voxel at depth offset -d (above the focus) on the axis is
    heard only at sample t_F - d, one at +d only at t_F + d (Eqs.
    q-above-2d / q-below-2d: the upper semicircle before the focal time,
    the lower after); the focal voxel only at t_F."""
    Z, k, T, tf, kf = 11, 5, 24, 12, 5.0
    M = _shell_mask(Z, k, T, 2, 1.0, kf, tf)
    r = k // 2
    for d in range(0, 5):
        up = np.nonzero(M[int(kf) - d, r, r])[0].tolist()
        down = np.nonzero(M[int(kf) + d, r, r])[0].tolist()
        assert up == [tf - d] and down == [tf + d], (d, up, down)
    # a half-integer focus: the two voxels around it both hold it
    Mh = _shell_mask(6, 3, 10, 3, 1.0, 2.5, 5)
    assert sorted(zip(*np.nonzero(Mh[..., 5]))) == [(2, 1, 1), (3, 1, 1)]


def test_semicircle_kernel_weights_and_impulse_response():
    """K = eta on the mask, convolved along t with the centred impulse
    response: a response with a single tap at s = +1 delays every column by
    one sample; a symmetric three-tap response is the sum of shifts; in 2D
    only dy = 0 carries weight, and the mask is even in dx."""
    Z, k, T, tf, kf = 7, 5, 16, 8, 3.0
    rng = np.random.default_rng(7)
    eta = rng.random((Z, k, k)) + 0.5
    M = _shell_mask(Z, k, T, 3, 2.0, kf, tf)
    K0 = oracle.semicircle_kernel(Z, k, T, 3, 2.0, kf, tf, eta, np.array([1.0]))
    assert np.array_equal(K0, np.where(M, eta[..., None], 0.0))
    K1 = oracle.semicircle_kernel(Z, k, T, 3, 2.0, kf, tf, eta, np.array([0.0, 0.0, 1.0]))
    assert np.array_equal(K1[..., 1:], K0[..., :-1]) and not K1[..., 0].any()
    v = np.array([0.25, 0.5, -0.75])
    K3 = oracle.semicircle_kernel(Z, k, T, 3, 2.0, kf, tf, eta, v)
    want = 0.5 * K0
    want[..., 1:] += -0.75 * K0[..., :-1]
    want[..., :-1] += 0.25 * K0[..., 1:]
    assert np.allclose(K3, want, rtol=0, atol=1e-15)
    M2 = _shell_mask(Z, k, T, 2, 2.0, kf, tf)
    assert not M2[:, [0, 1, 3, 4]].any() and M2[:, 2].any()
    assert np.array_equal(M2, M2[:, :, ::-1]) and np.array_equal(M, M[:, ::-1, ::-1])


# --------------------------------------------------------------------------
# Two-step approach (Eqs. acoustic-inverse and unmixing)
# --------------------------------------------------------------------------

def test_two_step_acoustic_part_equals_the_joint_block_diagonal_solve():
    """The acoustic problem over all pulses at once (W_tot block diagonal:
    the pulses as N 'species' with the identity switching matrix, TV summed
    over them) gives, with the same step, the per-pulse solves' iterates:
    the separation the two-step oracle relies on."""
    g, sw, K, y = _small_problem()
    alpha, iters, lam_tv, inner = 0.02, 15, 0.03, 8
    _, b = oracle.two_step(g, sw, K, y, alpha, iters, 0.0, lam_tv, inner,
                           0.01, 1, 0.0, 0.0, 0)
    S_id = np.zeros((g.N, g.N, g.Z))
    for n in range(g.N):
        S_id[n, n, :] = 1.0
    joint = np.empty((g.N, g.Y, g.X, g.Z))
    oracle.lib().oracle_fista(*[ctypes_int(v) for v in (g.N, g.N, g.Y, g.X, g.Z, g.T, g.k)],
                              oracle._p(S_id), oracle._p(np.ascontiguousarray(K)),
                              oracle._p(np.ascontiguousarray(y)), ctypes_double(alpha),
                              ctypes_int(iters), ctypes_double(0.0), ctypes_double(lam_tv),
                              ctypes_int(inner), ctypes_int(0), ctypes_int(0), oracle._p(joint),
                              ctypes_void(0))
    assert np.abs(b - joint).max() <= 1e-12 * np.abs(joint).max()


def test_two_step_unmixing_recovers_exact_concentrations():
    """Unmixing exact data b = S c_true (no regularisation, a well-posed S:
    N = 4 pulses over 2 species) converges to c_true, the per-voxel least
    squares solution of numpy's lstsq; the acoustic step with an identity
    acoustic kernel and exact data returns that data."""
    g = _geom(X=3, Y=2, Z=3, T=3, N=4, P=2, k=1, pulses_per_cycle=4)
    sw = Switching(kappa=(1.2, 0.0), eps_bar=(1.0, 0.0), eps_off=(0.1, 1.0), mu_per_mm=2.0)
    rng = np.random.default_rng(4)
    c_true = rng.random(g.c_shape()) + 0.2
    S = oracle.switch_matrix(g, sw)
    b_true = np.einsum("npj,pyxj->nyxj", S, c_true)
    eye = np.zeros(g.k_shape())
    for j in range(g.Z):
        eye[j, 0, 0, j] = 1.0
    lip = max(np.linalg.norm(S[:, :, j], 2) ** 2 for j in range(g.Z))
    c, b = oracle.two_step(g, sw, eye, b_true, 1.0, 60, 0.0, 0.0, 0,
                           1.0 / lip, 6000, 0.0, 0.0, 0)
    assert np.abs(b - b_true).max() <= 1e-10
    for j in range(g.Z):
        sol = np.linalg.lstsq(S[:, :, j], b_true[:, :, :, j].reshape(g.N, -1), rcond=None)[0]
        assert np.abs(sol.reshape(g.P, g.Y, g.X) - c_true[..., j]).max() <= 1e-10
    assert np.abs(c - c_true).max() <= 1e-6 * np.abs(c_true).max()


def ctypes_int(v):
    import ctypes
    return ctypes.c_int(int(v))


def ctypes_double(v):
    import ctypes
    return ctypes.c_double(float(v))


def ctypes_void(v):
    import ctypes
    return ctypes.c_void_p(v)


# --------------------------------------------------------------------------
# Full R3 with its lambda_3 term (Eq. reg-tv-l1-one): Algorithm 2 on the
# stacked L
# --------------------------------------------------------------------------

def _diff_matrix(Y, X, Z):
    """3D forward differences as a dense (3L x L) matrix, one row per
    (axis, voxel); rows of the last voxel along an axis are zero."""
    L = Y * X * Z
    idx = np.arange(L).reshape(Y, X, Z)
    D = np.zeros((3 * L, L))
    for axis in range(3):
        a = np.moveaxis(idx, axis, 0)
        for lo, hi in zip(a[:-1].ravel(), a[1:].ravel()):
            D[axis * L + lo, hi] = 1.0
            D[axis * L + lo, lo] = -1.0
    return D


def _stacked_L(g, sw, lam_tv, lam_l1, lam_b):
    """R3 = ||L c||_1: TV of each species, l1, TV of each pulse image (S c)^n."""
    L = g.Y * g.X * g.Z
    D = _diff_matrix(g.Y, g.X, g.Z)
    S = oracle.switch_matrix(g, sw)                      # [N][P][Z], pinned elsewhere
    depth = np.tile(np.arange(g.Z), g.Y * g.X)           # depth of each voxel
    blocks = []
    for p in range(g.P):
        row = np.zeros((3 * L, g.P * L))
        row[:, p * L:(p + 1) * L] = lam_tv * D
        blocks.append(row)
    blocks.append(lam_l1 * np.eye(g.P * L))
    for n in range(g.N):
        Sn = np.concatenate([np.diag(S[n, p, depth]) for p in range(g.P)], axis=1)
        blocks.append(lam_b * D @ Sn)
    return np.concatenate(blocks, axis=0)


def _box_dual_prox(Lmat, z, alpha):
    """argmin_x 1/2||x - z||^2 + alpha ||L x||_1 through its dual, min over
    |u| <= alpha of 1/2 ||z - L^T u||^2, by scipy's L-BFGS-B."""
    def fun(u):
        w = z - Lmat.T @ u
        return 0.5 * w @ w, -(Lmat @ w)
    res = scipy.optimize.minimize(fun, np.zeros(Lmat.shape[0]), jac=True, method="L-BFGS-B",
                                  bounds=[(-alpha, alpha)] * Lmat.shape[0],
                                  options={"maxiter": 20000, "ftol": 1e-15, "gtol": 1e-12})
    return z - Lmat.T @ res.x


def _joint_case(N=3, P=2):
    g = _geom(X=3, Y=2, Z=3, T=3, N=N, P=P, k=1, pulses_per_cycle=3)
    sw = _sw(P, mu=3.0)
    return g, sw


@pytest.mark.parametrize("lams", [(0.3, 0.1, 0.2), (0.0, 0.0, 0.4), (0.25, 0.15, 0.0)])
def test_joint_prox_matches_the_dual_solution(lams):
    """Algorithm 2 on the stacked L of R3 (all three terms) converges to the
    prox computed from its dual by an independent solver; the inputs keep the
    result positive, so Algorithm 2's final clip is inactive."""
    g, sw = _joint_case()
    lam_tv, lam_l1, lam_b = lams
    rng = np.random.default_rng(31)
    z = rng.standard_normal(g.c_shape()) + 4.0
    alpha = 0.7
    Lmat = _stacked_L(g, sw, lam_tv, lam_l1, lam_b)
    want = _box_dual_prox(Lmat, z.ravel(), alpha)
    assert want.min() > 0
    step2 = 1.0 / np.linalg.norm(Lmat, 2) ** 2
    got = oracle.prox_joint(g, sw, z, alpha, lam_tv, lam_l1, lam_b, 20000, step2)
    # both sides iterate to a tolerance: ~4e-6 is where L-BFGS-B stops
    np.testing.assert_allclose(got.ravel(), want, atol=1e-5)


def _constrained_dual_prox(Lmat, z, alpha):
    """argmin over x >= 0 of 1/2||x - z||^2 + alpha ||L x||_1 through its dual:
    for fixed u the inner minimum over x >= 0 is at x = max(z - L^T u, 0), and
    the dual is min over |u| <= alpha of 1/2 ||max(z - L^T u, 0)||^2 (gradient
    -L max(z - L^T u, 0)), solved by scipy's L-BFGS-B."""
    def fun(u):
        w = np.maximum(z - Lmat.T @ u, 0.0)
        return 0.5 * w @ w, -(Lmat @ w)
    res = scipy.optimize.minimize(fun, np.zeros(Lmat.shape[0]), jac=True, method="L-BFGS-B",
                                  bounds=[(-alpha, alpha)] * Lmat.shape[0],
                                  options={"maxiter": 50000, "ftol": 1e-16, "gtol": 1e-13})
    return np.maximum(z - Lmat.T @ res.x, 0.0)


def test_joint_prox_with_an_active_clip_is_the_constrained_prox():
    """Inputs with negative parts, the lambda_3 term coupling the species:
    the joint prox is the prox of R3 plus the nonnegativity indicator (Eq.
    prox), checked against its constrained dual solved by L-BFGS-B, and it
    differs from clipping the unconstrained prox (which the printed form of
    Algorithm 2 would give) by far more than the solvers' tolerance."""
    g, sw = _joint_case()
    lam_tv, lam_l1, lam_b = 0.2, 0.05, 0.5
    rng = np.random.default_rng(34)
    z = rng.standard_normal(g.c_shape()) * 1.5 - 0.2
    alpha = 0.7
    Lmat = _stacked_L(g, sw, lam_tv, lam_l1, lam_b)
    want = _constrained_dual_prox(Lmat, z.ravel(), alpha)
    assert (want == 0).sum() > 3  # the constraint is active
    step2 = 1.0 / np.linalg.norm(Lmat, 2) ** 2
    got = oracle.prox_joint(g, sw, z, alpha, lam_tv, lam_l1, lam_b, 40000, step2)
    np.testing.assert_allclose(got.ravel(), want, atol=1e-5)
    clipped = np.maximum(_box_dual_prox(Lmat, z.ravel(), alpha), 0.0)
    assert np.abs(clipped - want).max() > 1e-2


def test_joint_prox_without_lambda3_is_the_composite_prox():
    """With lambda_3 = 0 the joint dual gives max(prox_TV(z) - alpha lambda_l1, 0),
    the composition the solver uses (reading O8)."""
    g, sw = _joint_case()
    rng = np.random.default_rng(32)
    z = rng.standard_normal(g.c_shape()) + 1.0
    alpha, lam_tv, lam_l1 = 0.8, 0.3, 0.1
    Lmat = _stacked_L(g, sw, lam_tv, lam_l1, 0.0)
    step2 = 1.0 / np.linalg.norm(Lmat, 2) ** 2
    got = oracle.prox_joint(g, sw, z, alpha, lam_tv, lam_l1, 0.0, 8000, step2)
    comp = oracle.prox(z, alpha, lam_l1, lam_tv, 8000)
    np.testing.assert_allclose(got, comp, atol=2e-6)


def test_joint_prox_lambda3_on_identical_pulse_images_is_a_tv_prox():
    """One species with weight 1 at every depth (no switching, no fluence
    decay): every pulse image is c itself, so lambda_3 sum_n TV((S c)^n) =
    N lambda_3 TV(c) and the prox is the TV prox with threshold alpha N lambda_3."""
    g = _geom(X=3, Y=2, Z=4, T=4, N=3, P=1, k=1, pulses_per_cycle=3)
    sw = Switching(kappa=(0.0,), eps_bar=(0.0,), eps_off=(1.0,), mu_per_mm=0.0)
    rng = np.random.default_rng(33)
    z = rng.standard_normal(g.c_shape()) + 3.0
    alpha, lam_b = 0.5, 0.2
    step2 = 1.0 / (12.0 * (g.N * lam_b) ** 2)
    got = oracle.prox_joint(g, sw, z, alpha, 0.0, 0.0, lam_b, 8000, step2)
    want = oracle.prox_tv(z, alpha * g.N * lam_b, 8000)
    np.testing.assert_allclose(got, want, atol=2e-6)


# --------------------------------------------------------------------------
# Differentiating through the unrolled solve (forward mode)
# --------------------------------------------------------------------------

def test_switch_matrix_derivative_matches_central_differences():
    g = _geom(Z=6, N=7, P=3, pulses_per_cycle=4)
    sw = _sw(3, kappa=[0.8, 1.7, 0.0], mu=2.5)
    h = 1e-6
    for which in range(g.P + 1):
        dS = oracle.switch_matrix_derivative(g, sw, which)
        if which < g.P:
            kp, km = list(sw.kappa), list(sw.kappa)
            kp[which] += h
            km[which] -= h
            sp, sm = (Switching(tuple(kp), sw.eps_bar, sw.eps_off, sw.mu_per_mm),
                      Switching(tuple(km), sw.eps_bar, sw.eps_off, sw.mu_per_mm))
        else:
            sp = Switching(sw.kappa, sw.eps_bar, sw.eps_off, sw.mu_per_mm + h)
            sm = Switching(sw.kappa, sw.eps_bar, sw.eps_off, sw.mu_per_mm - h)
        fd = (oracle.switch_matrix(g, sp) - oracle.switch_matrix(g, sm)) / (2 * h)
        assert np.abs(dS - fd).max() <= 1e-8 * max(1.0, np.abs(fd).max()), which


@pytest.mark.parametrize("which", [0, 2])
def test_unrolled_solve_tangent_matches_central_differences(which):
    """dc_K/dtheta carried through every step of Algorithm 1 (and the
    Algorithm 2 iterations inside its prox) equals the central difference of
    the oracle's own solve at theta +- h (kappa_0, or mu), FP64."""
    g, sw, K, y = _small_problem()
    lip = oracle.power(g, sw, K, np.random.default_rng(0).standard_normal(g.c_shape()), 200)
    alpha, iters, lam1, lamtv, inner = 0.9 / lip, 16, 0.05, 0.02, 10
    c, dc = oracle.fista_tangent(g, sw, K, y, alpha, iters, lam1, lamtv, inner, which)
    ref = oracle.fista(g, sw, K, y, alpha, iters, lam1, lamtv, inner)
    assert np.array_equal(c, ref)
    h = 1e-6

    def at(delta):
        if which < g.P:
            kap = list(sw.kappa)
            kap[which] += delta
            s2 = Switching(tuple(kap), sw.eps_bar, sw.eps_off, sw.mu_per_mm)
        else:
            s2 = Switching(sw.kappa, sw.eps_bar, sw.eps_off, sw.mu_per_mm + delta)
        return oracle.fista(g, s2, K, y, alpha, iters, lam1, lamtv, inner)

    fd = (at(h) - at(-h)) / (2 * h)
    assert 0 < (c > 0).mean() < 1 and np.abs(dc).max() > 1e-2   # some outputs clipped, some not
    assert np.linalg.norm(dc - fd) <= 1e-5 * np.linalg.norm(fd)


def test_pulse_image_tv_is_the_dense_sum():
    """sum_n TV((S c)^n) against ||D S_n c||_1 with explicit matrices, and
    N TV(c) when every pulse image is c itself."""
    g, sw = _joint_case(N=4, P=2)
    rng = np.random.default_rng(35)
    c = rng.standard_normal(g.c_shape())
    D = _diff_matrix(g.Y, g.X, g.Z)
    S = oracle.switch_matrix(g, sw)
    depth = np.tile(np.arange(g.Z), g.Y * g.X)
    want = 0.0
    for n in range(g.N):
        Sn = np.concatenate([np.diag(S[n, p, depth]) for p in range(g.P)], axis=1)
        want += np.abs(D @ Sn @ c.ravel()).sum()
    assert oracle.tv_pulses(g, sw, c) == pytest.approx(want, rel=1e-13)
    g1 = _geom(X=3, Y=2, Z=4, T=4, N=3, P=1, k=1, pulses_per_cycle=3)
    sw1 = Switching(kappa=(0.0,), eps_bar=(0.0,), eps_off=(1.0,), mu_per_mm=0.0)
    c1 = rng.standard_normal(g1.c_shape())
    assert oracle.tv_pulses(g1, sw1, c1) == pytest.approx(g1.N * oracle.tv(c1), rel=1e-13)
    F0, _ = oracle.objective(g1, sw1, np.ones(g1.k_shape()), c1, np.zeros(g1.y_shape()), 0, 0)
    F3, _ = oracle.objective(g1, sw1, np.ones(g1.k_shape()), c1, np.zeros(g1.y_shape()), 0, 0,
                             lam_3=0.3)
    assert F3 - F0 == pytest.approx(0.3 * g1.N * oracle.tv(c1), rel=1e-12)


def test_fista_with_lambda3_reaches_a_fixed_point_of_the_exact_prox_gradient_map():
    """Algorithm 1 with all three terms of R3: after enough iterations c is a
    fixed point of c -> prox(c - alpha H^T (H c - y)), the prox computed from
    its constrained dual by L-BFGS-B with the explicit H and L matrices, and
    no feasible perturbation lowers F (with the lambda_3 term)."""
    g, sw, K, y = _small_problem()
    H = _dense_H(g, sw, K)
    lam_l1, lam_tv, lam_3 = 0.02, 0.03, 0.04
    alpha = 1.0 / np.linalg.eigvalsh(H.T @ H)[-1]
    Lmat = _stacked_L(g, sw, lam_tv, lam_l1, lam_3)
    step2 = 1.0 / np.linalg.norm(Lmat, 2) ** 2
    c, hist = oracle.fista(g, sw, K, y, alpha, 1500, lam_l1, lam_tv, 300, lam_3=lam_3,
                           joint_step2=step2, history=True)
    cf = c.ravel()
    zf = cf - alpha * (H.T @ (H @ cf - y.ravel()))
    fixed = _constrained_dual_prox(Lmat, zf, alpha)
    assert np.linalg.norm(fixed - cf) <= 1e-5 * np.linalg.norm(cf)

    def F(v):
        r = H @ v - y.ravel()
        return 0.5 * r @ r + np.abs(Lmat @ v).sum()

    assert F(cf) == pytest.approx(hist[-1], rel=1e-12)
    assert hist[-1] == pytest.approx(oracle.objective(g, sw, K, c, y, lam_l1, lam_tv, lam_3)[0],
                                     rel=1e-12)
    rng = np.random.default_rng(36)
    for _ in range(50):
        d = 1e-3 * rng.standard_normal(cf.size)
        assert F(np.maximum(cf + d, 0.0)) >= F(cf) - 1e-10
    # the lambda_3 term changes the solution
    c0 = oracle.fista(g, sw, K, y, alpha, 300, lam_l1, lam_tv, 300)
    assert np.linalg.norm(c0 - c) > 1e-3 * np.linalg.norm(c)


# --------------------------------------------------------------------------
# Fluence from the diffusion equation, Eqs. (de)/(bc), finite volumes
# --------------------------------------------------------------------------

def _slab_closed_form(Z, dz, mu_a, D, q):
    """The laterally uniform discrete solution phi_j = A r^j + B r^-j of the
    finite-volume rows (interior: (mu_a + 2w) phi_j = w (phi_{j-1} + phi_{j+1}),
    w = D/dz^2; the two end rows carry the boundary loss b = 2D/(4D + dz)/dz
    and the top one the source q/dz), A and B from the end rows."""
    w = D / dz ** 2
    b = 2 * D / (4 * D + dz) / dz
    c = 2 + mu_a / w
    r = (c - np.sqrt(c * c - 4)) / 2
    d = mu_a + w + b
    j = np.arange(Z, dtype=np.float64)
    M = np.array([[d - w * r, d - w / r],
                  [d * r ** (Z - 1) - w * r ** (Z - 2), d * r ** -(Z - 1) - w * r ** -(Z - 2)]])
    A, B = np.linalg.solve(M, [q / dz, 0.0])
    return A * r ** j + B * r ** -j


def test_diffusion_slab_matches_the_closed_form_of_its_recurrence():
    Y, X, Z, dx, dz = 3, 4, 20, 0.02, 0.05
    mu_a, mu_s, g, q = 0.5, 10.0, 0.9, 2.0
    phi = oracle.diffusion_fluence(Y, X, Z, dx, dz, mu_a, mu_s, g, q, lateral_robin=False)
    D = 1 / (3 * (mu_a + (1 - g) * mu_s))
    want = _slab_closed_form(Z, dz, mu_a, D, q)
    for y in range(Y):
        for x in range(X):
            np.testing.assert_allclose(phi[y, x], want, rtol=1e-11)


def test_diffusion_slab_converges_to_the_continuum_solution():
    """-D phi'' + mu_a phi = 0 on (0, H) with -D phi'(0) = q - phi(0)/2
    (illumination in, the Robin loss out) and -D phi'(H) = phi(H)/2: the
    finite-volume values at the cell centres converge as dz halves."""
    H, mu_a, mu_s, g, q = 1.0, 0.3, 8.0, 0.9, 1.0
    D = 1 / (3 * (mu_a + (1 - g) * mu_s))
    k = np.sqrt(mu_a / D)
    # phi = a exp(-k z) + b exp(k z); rows: top -D phi'(0) + phi(0)/2 = q,
    # bottom -D phi'(H) - phi(H)/2 = 0
    M = np.array([[D * k + 0.5, -D * k + 0.5],
                  [(D * k - 0.5) * np.exp(-k * H), (-D * k - 0.5) * np.exp(k * H)]])
    a, b = np.linalg.solve(M, [q, 0.0])
    errs = []
    for Z in (20, 40, 80):
        dz = H / Z
        z = (np.arange(Z) + 0.5) * dz
        exact = a * np.exp(-k * z) + b * np.exp(k * z)
        phi = oracle.diffusion_fluence(1, 1, Z, 0.1, dz, mu_a, mu_s, g, q, lateral_robin=False)
        errs.append(np.abs(phi[0, 0] - exact).max() / exact.max())
    assert errs[0] < 0.05
    assert errs[1] < errs[0] / 1.8 and errs[2] < errs[1] / 1.8


def test_diffusion_conserves_power_and_keeps_symmetry():
    """Summed over all voxels the rows state that the illumination entering
    the top equals the absorbed power plus the Robin losses; a source and an
    absorber map symmetric in x give a symmetric, positive fluence."""
    Y, X, Z, dx, dz, g = 5, 8, 12, 0.05, 0.04, 0.9
    rng = np.random.default_rng(37)
    half = 0.05 + rng.random((Y, X // 2, Z))
    mu_a = np.concatenate([half, half[:, ::-1]], axis=1)
    mu_s = np.full((Y, X, Z), 6.0)
    src = np.zeros((Y, X))
    src[:, 2:6] = 1.5
    phi = oracle.diffusion_fluence(Y, X, Z, dx, dz, mu_a, mu_s, g, src)
    assert phi.min() > 0
    np.testing.assert_allclose(phi, phi[:, ::-1], rtol=1e-10)
    D = 1 / (3 * (mu_a + (1 - g) * mu_s))
    area = {"y": dx * dz, "x": dx * dz, "z": dx * dx}
    pitch = {"y": dx, "x": dx, "z": dz}
    loss = 0.0
    for ax, sl in (("y", np.s_[[0, -1], :, :]), ("x", np.s_[:, [0, -1], :]),
                   ("z", np.s_[:, :, [0, -1]])):
        h = pitch[ax]
        loss += area[ax] * np.sum(2 * D[sl] * phi[sl] / (4 * D[sl] + h))
    absorbed = np.sum(mu_a * phi) * dx * dx * dz
    entering = np.sum(src) * dx * dx
    assert absorbed + loss == pytest.approx(entering, rel=1e-10)
