"""The C-ABI library: it builds for sm_103a, loads, exports every entry point
declared in include/swopt.h, and rejects bad arguments on the host before
any GPU work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2510_23739_gb300 as sw
from paper_2510_23739_gb300 import build as swbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "swopt.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|swopt_status|double)\s+(swopt_\w+)\s*\(",
                                 text, re.M)))


def test_library_targets_sm_103a_and_loads():
    path = swbuild.build()
    assert os.path.exists(path)
    assert any("arch=compute_103a,code=sm_103a" in a for a in swbuild.ARCH)
    sw.lib()


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 20
    L = ctypes.CDLL(swbuild.build())
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(names) <= set(sw._SIGS)


def test_binding_enums_match_the_header():
    """The binding's precision and momentum names carry the header's values."""
    text = open(os.path.join(ROOT, "include", "swopt.h")).read()
    prec = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"SWOPT_PREC_(\w+)\s*=\s*(\d+)", text)}
    assert prec == sw.PRECISION
    mom = {m.group(1).lower(): int(m.group(2))
           for m in re.finditer(r"SWOPT_MOMENTUM_(\w+)\s*=\s*(\d+)", text)}
    assert mom == sw.MOMENTUM


def _geom(**kw):
    g = sw._Geometry(8, 8, 4, 16, 4, 2, 3, 2, 0.01)
    for k, v in kw.items():
        setattr(g, k, v)
    return g


def _switching(P=2):
    arrs = [np.array([0.1, 0.0][:P]), np.array([1.0, 0.0][:P]), np.array([0.0, 1.0][:P])]
    dp = ctypes.POINTER(ctypes.c_double)
    return sw._Switching(*(a.ctypes.data_as(dp) for a in arrs), 2.0), arrs


def _create(g, K, s):
    h = ctypes.c_void_p()
    st = sw.lib().swopt_create(ctypes.byref(g) if g is not None else None,
                               K.ctypes.data_as(ctypes.c_void_p) if K is not None else None,
                               ctypes.byref(s) if s is not None else None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("field,value", [("k", 4), ("k", 0), ("X", 0), ("P", 9), ("T", 0),
                                         ("pulses_per_cycle", 0), ("N", 0)])
def test_create_rejects_bad_shapes(field, value):
    s, keep = _switching()
    g = _geom(**{field: value})
    K = np.ones((max(g.Z, 1), max(g.k, 1), max(g.k, 1), max(g.T, 1)))
    st, h = _create(g, K, s)
    assert st == 2 and not h.value  # SWOPT_ERR_SHAPE
    assert b"range" in sw.lib().swopt_last_error()


def test_create_rejects_null_and_nonfinite():
    s, keep = _switching()
    g = _geom()
    K = np.ones((4, 3, 3, 16))
    assert _create(None, K, s)[0] == 1
    assert _create(g, None, s)[0] == 1
    assert _create(g, K, None)[0] == 1
    K2 = K.copy()
    K2[1, 1, 1, 3] = np.nan
    assert _create(g, K2, s)[0] == 1
    assert _create(_geom(dz_mm=-1.0), K, s)[0] == 1
    # an all-zero kernel has no time window
    st, _ = _create(g, np.zeros_like(K), s)
    assert st == 2 and b"zero" in sw.lib().swopt_last_error()


def test_null_handle_calls_fail_cleanly():
    L = sw.lib()
    assert L.swopt_destroy(None) == 0
    assert L.swopt_forward(None, None, None, None) == 1
    assert L.swopt_adjoint(None, None, None, None) == 1
    assert L.swopt_set_precision(None, 0) == 1
    assert L.swopt_fista_step(None, 1, None) == 1
    assert b"null handle" in L.swopt_last_error()
    assert L.swopt_tc_schedule(None, 0, 1, 1) == 1
    i = ctypes.c_int()
    assert L.swopt_tc_schedule_info(None, 0, *[ctypes.byref(i)] * 4) == 1
    assert L.swopt_two_step(None, None, None, None, None, None, None, None, None) == 1
    assert L.swopt_prox_joint(None, None, None, 1.0, 0.1, 0.1, 0.1, 1, 0.1, None) == 1
    assert L.swopt_prox_joint_step_bound(None, 0.1, 0.1, 0.1) == 0.0
    assert L.swopt_set_state_offset(None, 0) == 1
    assert L.swopt_fista_gradient(None, None, None, None) == 1
    assert L.swopt_fista_step_external(None, None, None) == 1
    assert L.swopt_set_fluence(None, None) == 1
    assert L.swopt_unrolled_vjp(None, None, None, None, None, None, None, None) == 1
    i = ctypes.c_int()
    assert L.swopt_batch_configure(None, 1) == 1
    assert L.swopt_batch_query(None, ctypes.byref(i), None) == 1
    assert b"null" in L.swopt_last_error()
    assert L.swopt_version().decode().count(".") == 2


def test_diffusion_fluence_rejects_bad_arguments_before_gpu_work():
    L = sw.lib()
    n = 2 * 2 * 3
    ok = np.ones(n)
    src = np.ones(4)
    out = np.zeros(n)
    dp = ctypes.c_void_p
    args = lambda mu_a, g, tol: (2, 2, 3, 0.02, 0.01, mu_a.ctypes.data_as(dp),
                                 ok.ctypes.data_as(dp), g, src.ctypes.data_as(dp), 1, tol, 100,
                                 out.ctypes.data_as(dp), None, None)
    assert L.swopt_diffusion_fluence(*args(ok, 1.0, 1e-8)) == 1       # g must be < 1
    assert L.swopt_diffusion_fluence(*args(ok, 0.9, 0.0)) == 1        # tol must be > 0
    bad = ok.copy()
    bad[3] = -1.0
    assert L.swopt_diffusion_fluence(*args(bad, 0.9, 1e-8)) == 1      # negative absorption
    bad[3] = np.nan
    assert L.swopt_diffusion_fluence(*args(bad, 0.9, 1e-8)) == 1
    assert b"absorption" in L.swopt_last_error()


@pytest.mark.parametrize("dims,rho,kf", [(2, 2.0, 3.5), (3, 2.0, 3.5), (3, 1.0, 4.0)])
def test_semicircle_kernel_builder_matches_oracle(dims, rho, kf):
    """The library's host builder of the paper-literal kernel against the
    oracle's: the masks bit-exact (their decisions are exact in FP64 here),
    the weighted and convolved kernel to FP64 rounding."""
    import oracle
    Z, k, T, tf = 10, 9, 30, 15
    ones = np.ones((Z, k, k))
    a = sw.semicircle_kernel(Z, k, T, dims, rho, kf, tf, ones, np.array([1.0]))
    b = oracle.semicircle_kernel(Z, k, T, dims, rho, kf, tf, ones, np.array([1.0]))
    assert np.array_equal(a, b) and a.any()
    rng = np.random.default_rng(3)
    eta = rng.random((Z, k, k))
    eir = rng.standard_normal(7)
    a = sw.semicircle_kernel(Z, k, T, dims, rho, kf, tf, eta, eir)
    b = oracle.semicircle_kernel(Z, k, T, dims, rho, kf, tf, eta, eir)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_semicircle_kernel_builder_rejects_bad_arguments():
    ones = np.ones((4, 3, 3))
    good = dict(Z=4, k=3, T=8, dims=3, lateral_ratio=1.0, focal_depth=1.5, focal_sample=4,
                eta=ones, eir=np.array([1.0]))
    sw.semicircle_kernel(**good)
    for bad in (dict(dims=1), dict(lateral_ratio=0.0), dict(lateral_ratio=float("nan")),
                dict(focal_sample=8), dict(focal_sample=-1), dict(eir=np.array([1.0, 2.0])),
                dict(focal_depth=float("inf"))):
        with pytest.raises(sw.SwoptError):
            sw.semicircle_kernel(**{**good, **bad})
    with pytest.raises(sw.SwoptError):
        sw.semicircle_kernel(**{**good, "k": 4, "eta": np.ones((4, 4, 4))})
