"""FP64 CPU oracle (test infrastructure).

Plain, slow, obviously-correct reference for the photo-switching
optoacoustic hot path (arXiv 2510.23739): the switching matrix of
Eq. (final-H)/(Sij-detailed), the forward H = W_tot S of Sec. 2.3 and
Eq. (full-forward), its exact adjoint, the l1 and TV proximal maps of
Eq. (prox)/(prox-dual) and Algorithm 2, FISTA (Algorithm 1), the power
iteration for the step size, the kappa/mu gradient of the data fit, and the
paper-literal semicircle kernel of Eqs. (q-above-final)/(q-below-final), and
the two-step approach (Eqs. (acoustic-inverse), (unmixing)), and the
proximal map of the full R3 with its lambda_3 term (Algorithm 2 on the
stacked L), and the derivative of the unrolled solve with respect to the
switching parameters (forward mode).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  It shares no code with the CUDA
library.  The arithmetic lives in ``swopt_oracle.c`` (plain C, FP64, optional
OpenMP over independent outputs); this file only compiles it and marshals
numpy arrays.

Every function is pinned by ``tests/test_oracle_pins.py``; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swopt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MOMENTUM = {"beck_teboulle": 0, "paper_printed": 1, "none": 2}


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.oracle_power.restype = ctypes.c_double
            L.oracle_objective.restype = ctypes.c_double
            L.oracle_tv.restype = ctypes.c_double
            L.oracle_tv_pulses.restype = ctypes.c_double
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_diffusion_system.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(geom):
    g = geom
    return [ctypes.c_int(v) for v in (g.N, g.P, g.Y, g.X, g.Z, g.T, g.k)]


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of later oracle calls (timing only)."""
    lib().oracle_set_threads(ctypes.c_int(int(n)))


def fluence(geom, sw):
    """Phi_j = exp(-mu j dz)."""
    out = np.empty(geom.Z)
    lib().oracle_fluence(ctypes.c_int(geom.Z), ctypes.c_double(sw.mu_per_mm),
                         ctypes.c_double(geom.dz_mm), _p(out))
    return out


def diffusion_system(Y, X, Z, dx, dz, mu_a, mu_s, g, src_top, lateral_robin=True):
    """The finite-volume system of Eqs. (de)/(bc) (see oracle_diffusion_system):
    a scipy CSR matrix and the right-hand side, unknowns Phi[Y][X][Z]."""
    import scipy.sparse as sp
    n = Y * X * Z
    mu_a = np.ascontiguousarray(np.broadcast_to(mu_a, (Y, X, Z)), dtype=np.float64)
    mu_s = np.ascontiguousarray(np.broadcast_to(mu_s, (Y, X, Z)), dtype=np.float64)
    src = np.ascontiguousarray(np.broadcast_to(src_top, (Y, X)), dtype=np.float64)
    rows = np.empty(7 * n, dtype=np.int32)
    cols = np.empty(7 * n, dtype=np.int32)
    vals = np.empty(7 * n)
    rhs = np.empty(n)
    cnt = lib().oracle_diffusion_system(
        ctypes.c_int(Y), ctypes.c_int(X), ctypes.c_int(Z), ctypes.c_double(dx),
        ctypes.c_double(dz), _p(mu_a), _p(mu_s), ctypes.c_double(g), _p(src),
        ctypes.c_int(1 if lateral_robin else 0), _p(rows), _p(cols), _p(vals), _p(rhs))
    A = sp.csr_matrix((vals[:cnt], (rows[:cnt], cols[:cnt])), shape=(n, n))
    return A, rhs


def diffusion_fluence(Y, X, Z, dx, dz, mu_a, mu_s, g, src_top, lateral_robin=True):
    """Phi[Y][X][Z] solving the finite-volume system of Eqs. (de)/(bc)
    (scipy's sparse direct solver)."""
    import scipy.sparse.linalg as spla
    A, rhs = diffusion_system(Y, X, Z, dx, dz, mu_a, mu_s, g, src_top, lateral_robin)
    return spla.spsolve(A.tocsc(), rhs).reshape(Y, X, Z)


def switch_matrix(geom, sw, phi=None):
    """S[n][p][j] of Eq. (final-H); phi (optional, [Z]) replaces exp(-mu j dz)."""
    phi = fluence(geom, sw) if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    kap = _f64(sw.kappa)
    eb = _f64(sw.eps_bar)
    eo = _f64(sw.eps_off)
    S = np.empty((geom.N, geom.P, geom.Z))
    lib().oracle_switch_matrix(ctypes.c_int(geom.N), ctypes.c_int(geom.P),
                               ctypes.c_int(geom.Z), ctypes.c_int(geom.pulses_per_cycle),
                               _p(phi), _p(kap), _p(eb), _p(eo), _p(S))
    return S


def forward(geom, sw, K, c, S=None):
    """y = H c, y[N][Y][X][T]."""
    S = switch_matrix(geom, sw) if S is None else _f64(S)
    K = _f64(K)
    c = _f64(c)
    y = np.empty(geom.y_shape())
    lib().oracle_forward(*_dims(geom), _p(S), _p(K), _p(c), _p(y))
    return y


def adjoint(geom, sw, K, y, S=None):
    """c = H^T y, c[P][Y][X][Z]."""
    S = switch_matrix(geom, sw) if S is None else _f64(S)
    K = _f64(K)
    y = _f64(y)
    c = np.empty(geom.c_shape())
    lib().oracle_adjoint(*_dims(geom), _p(S), _p(K), _p(y), _p(c))
    return c


def forward_at(geom, sw, K, c, nyx):
    """(H c)[n, y, x, :] for each row of the int array ``nyx`` (count x 3)."""
    S = switch_matrix(geom, sw)
    idx = np.ascontiguousarray(nyx, dtype=np.int32)
    out = np.empty((idx.shape[0], geom.T))
    lib().oracle_forward_at(*_dims(geom), _p(S), _p(_f64(K)), _p(_f64(c)),
                            ctypes.c_int(idx.shape[0]), _p(idx), _p(out))
    return out


def adjoint_at(geom, sw, K, y, pyxj):
    """(H^T y)[p, y, x, j] for each row of ``pyxj`` (count x 4)."""
    S = switch_matrix(geom, sw)
    idx = np.ascontiguousarray(pyxj, dtype=np.int32)
    out = np.empty(idx.shape[0])
    lib().oracle_adjoint_at(*_dims(geom), _p(S), _p(_f64(K)), _p(_f64(y)),
                            ctypes.c_int(idx.shape[0]), _p(idx), _p(out))
    return out


def grad3(v):
    v = _f64(v)
    Y, X, Z = v.shape
    g = np.empty((3, Y, X, Z))
    lib().oracle_grad3(ctypes.c_int(Y), ctypes.c_int(X), ctypes.c_int(Z), _p(v), _p(g))
    return g


def grad3T(g):
    g = _f64(g)
    _, Y, X, Z = g.shape
    v = np.empty((Y, X, Z))
    lib().oracle_grad3T(ctypes.c_int(Y), ctypes.c_int(X), ctypes.c_int(Z), _p(g), _p(v))
    return v


def tv(c):
    c = _f64(c)
    P, Y, X, Z = c.shape
    return float(lib().oracle_tv(ctypes.c_int(P), ctypes.c_int(Y), ctypes.c_int(X),
                                 ctypes.c_int(Z), _p(c)))


def prox_l1(x, theta, nonneg=True):
    x = _f64(x).copy()
    lib().oracle_prox_l1(ctypes.c_size_t(x.size), _p(x), ctypes.c_double(theta),
                         ctypes.c_int(1 if nonneg else 0))
    return x


def prox_tv(z, tau, iters, momentum="beck_teboulle"):
    z = _f64(z)
    P, Y, X, Z = z.shape
    x = np.empty_like(z)
    lib().oracle_prox_tv(ctypes.c_int(P), ctypes.c_int(Y), ctypes.c_int(X), ctypes.c_int(Z),
                         _p(z), _p(x), ctypes.c_double(tau), ctypes.c_int(iters),
                         ctypes.c_int(MOMENTUM[momentum]))
    return x


def prox(z, alpha, lam_l1, lam_tv, inner, momentum="beck_teboulle"):
    z = _f64(z)
    P, Y, X, Z = z.shape
    x = np.empty_like(z)
    lib().oracle_prox(ctypes.c_int(P), ctypes.c_int(Y), ctypes.c_int(X), ctypes.c_int(Z),
                      _p(z), _p(x), ctypes.c_double(alpha), ctypes.c_double(lam_l1),
                      ctypes.c_double(lam_tv), ctypes.c_int(inner),
                      ctypes.c_int(MOMENTUM[momentum]))
    return x


def prox_joint(geom, sw, z, alpha, lam_tv, lam_l1, lam_b, iters, step2,
               momentum="beck_teboulle", return_dual=False):
    """prox of alpha (R3 + delta_{>=0}) with the lambda_3 term (Eq.
    (reg-tv-l1-one)) by Algorithm 2 on the stacked L; returns x (and the
    dual u = [uc (P x 3L), ul (P L), ub (N x 3L)] if asked)."""
    S = switch_matrix(geom, sw)
    z = _f64(z).reshape(geom.c_shape())
    x = np.empty(geom.c_shape())
    L = geom.Y * geom.X * geom.Z
    u = np.empty(geom.P * 4 * L + geom.N * 3 * L) if return_dual else None
    lib().oracle_prox_joint(ctypes.c_int(geom.N), ctypes.c_int(geom.P), ctypes.c_int(geom.Y),
                            ctypes.c_int(geom.X), ctypes.c_int(geom.Z), _p(S), _p(z), _p(x),
                            ctypes.c_double(alpha), ctypes.c_double(lam_tv),
                            ctypes.c_double(lam_l1), ctypes.c_double(lam_b), ctypes.c_int(iters),
                            ctypes.c_double(step2), ctypes.c_int(MOMENTUM[momentum]),
                            _p(u) if return_dual else ctypes.c_void_p(0))
    return (x, u) if return_dual else x


def tv_pulses(geom, sw, c):
    """sum_n TV((S c)^n), the lambda_3 term of Eq. (reg-tv-l1-one)."""
    S = switch_matrix(geom, sw)
    c = _f64(c).reshape(geom.c_shape())
    return float(lib().oracle_tv_pulses(ctypes.c_int(geom.N), ctypes.c_int(geom.P),
                                        ctypes.c_int(geom.Y), ctypes.c_int(geom.X),
                                        ctypes.c_int(geom.Z), _p(S), _p(c)))


def objective(geom, sw, K, c, y, lam_l1, lam_tv, lam_3=0.0):
    """Returns (F(c), data-fit 1/2||Hc - y||^2); F includes lam_3 sum_n TV((S c)^n)."""
    S = switch_matrix(geom, sw)
    fit = ctypes.c_double(0.0)
    F = lib().oracle_objective(*_dims(geom), _p(S), _p(_f64(K)), _p(_f64(c)), _p(_f64(y)),
                               ctypes.c_double(lam_l1), ctypes.c_double(lam_tv),
                               ctypes.byref(fit))
    if lam_3 != 0.0:
        F += lam_3 * tv_pulses(geom, sw, c)
    return float(F), float(fit.value)


def fista(geom, sw, K, y, alpha, iters, lam_l1, lam_tv, inner,
          momentum="beck_teboulle", inner_momentum="beck_teboulle", history=False,
          lam_3=0.0, joint_step2=None):
    """Algorithm 1 with a fixed iteration count; returns c (and F per iteration).
    lam_3 > 0 takes the prox of all three terms of R3 (prox_joint, ``inner``
    dual iterations with dual step ``joint_step2``)."""
    S = switch_matrix(geom, sw)
    c = np.empty(geom.c_shape())
    hist = np.empty(iters) if history else None
    if lam_3 > 0:
        if joint_step2 is None:
            raise ValueError("lam_3 > 0 needs the joint prox's dual step")
        lib().oracle_fista_joint(*_dims(geom), _p(S), _p(_f64(K)), _p(_f64(y)),
                                 ctypes.c_double(alpha), ctypes.c_int(iters),
                                 ctypes.c_double(lam_l1), ctypes.c_double(lam_tv),
                                 ctypes.c_double(lam_3), ctypes.c_int(inner),
                                 ctypes.c_double(joint_step2), ctypes.c_int(MOMENTUM[momentum]),
                                 ctypes.c_int(MOMENTUM[inner_momentum]), _p(c),
                                 _p(hist) if history else ctypes.c_void_p(0))
        return (c, hist) if history else c
    lib().oracle_fista(*_dims(geom), _p(S), _p(_f64(K)), _p(_f64(y)),
                       ctypes.c_double(alpha), ctypes.c_int(iters),
                       ctypes.c_double(lam_l1), ctypes.c_double(lam_tv), ctypes.c_int(inner),
                       ctypes.c_int(MOMENTUM[momentum]), ctypes.c_int(MOMENTUM[inner_momentum]),
                       _p(c), _p(hist) if history else ctypes.c_void_p(0))
    return (c, hist) if history else c


def power(geom, sw, K, v0, iters):
    """Rayleigh-quotient estimate of eig_max(H^T H) after ``iters`` steps."""
    S = switch_matrix(geom, sw)
    return float(lib().oracle_power(*_dims(geom), _p(S), _p(_f64(K)), _p(_f64(v0)),
                                    ctypes.c_int(iters)))


def two_step(geom, sw, K, y, alpha1, iters1, lam_l1_1, lam_tv_1, inner1,
             alpha2, iters2, lam_l1_2, lam_tv_2, inner2):
    """The two-step approach: per-pulse acoustic inversion (Eq.
    (acoustic-inverse)) into b[N][Y][X][Z], then unmixing (Eq. (unmixing))
    into c[P][Y][X][Z]; returns (c, b)."""
    S = switch_matrix(geom, sw)
    b = np.empty((geom.N, geom.Y, geom.X, geom.Z))
    c = np.empty(geom.c_shape())
    lib().oracle_two_step(*_dims(geom), _p(S), _p(_f64(K)), _p(_f64(y)),
                          ctypes.c_double(alpha1), ctypes.c_int(iters1),
                          ctypes.c_double(lam_l1_1), ctypes.c_double(lam_tv_1), ctypes.c_int(inner1),
                          ctypes.c_double(alpha2), ctypes.c_int(iters2),
                          ctypes.c_double(lam_l1_2), ctypes.c_double(lam_tv_2), ctypes.c_int(inner2),
                          _p(b), _p(c))
    return c, b


def semicircle_kernel(Z, k, T, dims, rho, focal_depth, focal_sample, eta, eir):
    """K[Z][k][k][T]: the paper-literal kernel of Eqs. (q-above-final) /
    (q-below-final), the spatial response on the discrete half spheres of
    each time sample, convolved along t with the centred impulse response."""
    eta = _f64(eta).reshape(Z, k, k)
    eir = _f64(eir).ravel()
    K = np.empty((Z, k, k, T))
    lib().oracle_semicircle_kernel(ctypes.c_int(Z), ctypes.c_int(k), ctypes.c_int(T),
                                   ctypes.c_int(dims), ctypes.c_double(rho),
                                   ctypes.c_double(focal_depth), ctypes.c_int(focal_sample),
                                   _p(eta), _p(eir), ctypes.c_int(eir.size), _p(K))
    return K


def switch_matrix_derivative(geom, sw, which):
    """dS/dkappa_p (which = p < P) or dS/dmu (which = P) of Eq. (final-H)."""
    dS = np.empty((geom.N, geom.P, geom.Z))
    lib().oracle_switch_matrix_derivative(
        ctypes.c_int(geom.N), ctypes.c_int(geom.P), ctypes.c_int(geom.Z),
        ctypes.c_int(geom.pulses_per_cycle), ctypes.c_double(sw.mu_per_mm),
        ctypes.c_double(geom.dz_mm), _p(_f64(sw.kappa)), _p(_f64(sw.eps_bar)),
        _p(_f64(sw.eps_off)), ctypes.c_int(which), _p(dS))
    return dS


def fista_tangent(geom, sw, K, y, alpha, iters, lam_l1, lam_tv, inner, which,
                  momentum="beck_teboulle", inner_momentum="beck_teboulle"):
    """Algorithm 1's output c_K and its derivative dc_K/dtheta through the
    unrolled solve (forward mode), theta = kappa_p (which = p) or mu (which = P),
    with the step, weights and counts held fixed."""
    S = switch_matrix(geom, sw)
    dS = switch_matrix_derivative(geom, sw, which)
    c = np.empty(geom.c_shape())
    dc = np.empty(geom.c_shape())
    lib().oracle_fista_tangent(*_dims(geom), _p(S), _p(dS), _p(_f64(K)), _p(_f64(y)),
                               ctypes.c_double(alpha), ctypes.c_int(iters),
                               ctypes.c_double(lam_l1), ctypes.c_double(lam_tv),
                               ctypes.c_int(inner), ctypes.c_int(MOMENTUM[momentum]),
                               ctypes.c_int(MOMENTUM[inner_momentum]), _p(c), _p(dc))
    return c, dc


def param_grad(geom, sw, K, c, y):
    """(d/dkappa[P], d/dmu) of 1/2 ||H c - y||^2."""
    dk = np.empty(geom.P)
    dmu = ctypes.c_double(0.0)
    lib().oracle_param_grad(*_dims(geom), ctypes.c_int(geom.pulses_per_cycle),
                            ctypes.c_double(sw.mu_per_mm), ctypes.c_double(geom.dz_mm),
                            _p(_f64(sw.kappa)), _p(_f64(sw.eps_bar)), _p(_f64(sw.eps_off)),
                            _p(_f64(K)), _p(_f64(c)), _p(_f64(y)), _p(dk), ctypes.byref(dmu))
    return dk, float(dmu.value)
