"""Python binding of the swopt C-ABI (argument marshalling only).

Every operation runs in the CUDA library ``_build/libswopt.so`` (built from
``csrc/`` by ``build.py``); this module only converts PyTorch CUDA tensors to
device pointers and the current CUDA stream to a ``cudaStream_t``.  There is
no CPU path: if the library cannot be built or loaded, the import of
:func:`lib` raises.

The operator is H = A o P of arXiv 2510.23739 (Sec. 2.3, Eq. full-forward):
P maps concentrations c[P][Y][X][Z] to per-pulse initial pressure through the
switching law of Eq. (final-H), A is the lateral-shift-invariant per-depth
acoustic kernel K[Z][k][k][T] that maps each pulse's pressure to
measurements y[N][Y][X][T].
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["lib", "Operator", "SolveParams", "SwoptError", "PRECISION", "MOMENTUM",
           "HFunction", "Batch", "REFINED_DEFAULTS"]

PRECISION = {"fp32": 0, "bf16": 1, "bf16x3": 2, "fp8": 3, "bf16x6": 4}
MOMENTUM = {"beck_teboulle": 0, "paper_printed": 1, "none": 2}
# The refined solve's recommended schedule for BF16 contractions: an exact
# (two-term BF16) gradient every 25 iterations, and sooner whenever the
# relative steps ||c_{k+1} - c_k|| / ||c_{k+1}|| taken on BF16 increments since
# the last exact gradient add up to more than 0.1 (see refine_budget in
# swopt_solve_params).
REFINED_DEFAULTS = {"refine_every": 25, "refine_precision": "bf16x3", "refine_budget": 0.1}

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "SHAPE", 3: "CUDA", 4: "OOM", 5: "TIMEOUT",
           6: "DEVICE_CHECK", 7: "UNSUPPORTED"}


class SwoptError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"swopt error {_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Geometry(ctypes.Structure):
    _fields_ = [("X", ctypes.c_int), ("Y", ctypes.c_int), ("Z", ctypes.c_int),
                ("T", ctypes.c_int), ("N", ctypes.c_int), ("P", ctypes.c_int),
                ("k", ctypes.c_int), ("pulses_per_cycle", ctypes.c_int),
                ("dz_mm", ctypes.c_double)]


class _Switching(ctypes.Structure):
    _fields_ = [("kappa_host", ctypes.POINTER(ctypes.c_double)),
                ("eps_bar_host", ctypes.POINTER(ctypes.c_double)),
                ("eps_off_host", ctypes.POINTER(ctypes.c_double)),
                ("mu_per_mm", ctypes.c_double)]


class _SolveParams(ctypes.Structure):
    _fields_ = [("step", ctypes.c_double), ("lambda_l1", ctypes.c_double),
                ("lambda_tv", ctypes.c_double), ("inner_iters", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("eps1", ctypes.c_double),
                ("eps2", ctypes.c_double), ("momentum", ctypes.c_int),
                ("inner_momentum", ctypes.c_int), ("power_iters", ctypes.c_int),
                ("refine_every", ctypes.c_int), ("refine_precision", ctypes.c_int),
                ("history_host", ctypes.POINTER(ctypes.c_double)),
                ("refine_budget", ctypes.c_double), ("lambda_3", ctypes.c_double),
                ("joint_step2", ctypes.c_double)]


class _SolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("step", ctypes.c_double),
                ("objective", ctypes.c_double), ("data_fit", ctypes.c_double)]


_lock = threading.Lock()
_lib = None

# exported symbol -> argtypes (restype is swopt_status = int unless listed)
_SIGS = {
    "swopt_last_error": ([], ctypes.c_char_p),
    "swopt_version": ([], ctypes.c_char_p),
    "swopt_create": ([ctypes.POINTER(_Geometry), ctypes.c_void_p, ctypes.POINTER(_Switching),
                      ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "swopt_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "swopt_set_precision": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "swopt_forward": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                      ctypes.c_int),
    "swopt_adjoint": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                      ctypes.c_int),
    "swopt_prox_l1": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int,
                       ctypes.c_void_p], ctypes.c_int),
    "swopt_prox_tv": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                       ctypes.c_int, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "swopt_lipschitz": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p], ctypes.c_int),
    "swopt_fista_init": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_SolveParams),
                          ctypes.c_void_p], ctypes.c_int),
    "swopt_fista_step": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "swopt_fista_get": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "swopt_solve": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                     ctypes.POINTER(_SolveParams), ctypes.POINTER(_SolveStats), ctypes.c_void_p],
                    ctypes.c_int),
    "swopt_objective": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                         ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p], ctypes.c_int),
    "swopt_param_grad": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.c_void_p], ctypes.c_int),
    "swopt_param_vjp": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                         ctypes.c_void_p], ctypes.c_int),
    "swopt_set_switching": ([ctypes.c_void_p, ctypes.POINTER(_Switching)], ctypes.c_int),
    "swopt_batch_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                            ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "swopt_batch_step": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "swopt_batch_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "swopt_batch_configure": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "swopt_batch_query": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "swopt_profile_enable": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "swopt_use_graphs": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "swopt_profile_read": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)],
                           ctypes.c_int),
    "swopt_launch_count": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "swopt_info": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "swopt_check_device": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "swopt_issued_flops": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
                           ctypes.c_int),
    "swopt_tc_configure": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_int], ctypes.c_int),
    "swopt_tc_config": ([ctypes.c_void_p, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 5,
                        ctypes.c_int),
    "swopt_prox_joint": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                          ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                          ctypes.c_double, ctypes.c_void_p], ctypes.c_int),
    "swopt_unrolled_vjp": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_SolveParams),
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.c_void_p], ctypes.c_int),
    "swopt_diffusion_fluence": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "swopt_set_fluence": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "swopt_set_state_offset": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "swopt_fista_gradient": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p], ctypes.c_int),
    "swopt_fista_step_external": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                                  ctypes.c_int),
    "swopt_prox_joint_step_bound": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double], ctypes.c_double),
    "swopt_two_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.c_void_p], ctypes.c_int),
    "swopt_semicircle_kernel": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "swopt_tc_schedule": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "swopt_tc_schedule_info": ([ctypes.c_void_p, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4,
                               ctypes.c_int),
    "swopt_prox_tv_static": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int,
                              ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "swopt_refine_stats": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p], ctypes.c_int),
    "swopt_fista_state_bytes": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "swopt_fista_save": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p],
                         ctypes.c_int),
    "swopt_fista_restore": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p],
                            ctypes.c_int),
    "swopt_debug_barrier": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_uint], ctypes.c_int),
}


def lib():
    """Load (building first if needed) the CUDA library.  Raises on failure."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def diffusion_fluence(Y, X, Z, dx_mm, dz_mm, mu_a, mu_s, g, src_top, lateral_robin=True,
                      tol=1e-10, max_iters=100000):
    """Fluence Phi [Y][X][Z] from the diffusion equation (see
    swopt_diffusion_fluence); mu_a, mu_s broadcast to [Y][X][Z], src_top to
    [Y][X].  Returns (phi, iterations, relative residual)."""
    mu_a = np.ascontiguousarray(np.broadcast_to(mu_a, (Y, X, Z)), dtype=np.float64)
    mu_s = np.ascontiguousarray(np.broadcast_to(mu_s, (Y, X, Z)), dtype=np.float64)
    src = np.ascontiguousarray(np.broadcast_to(src_top, (Y, X)), dtype=np.float64)
    phi = np.empty((Y, X, Z))
    it, rel = ctypes.c_int(), ctypes.c_double()
    _check(lib().swopt_diffusion_fluence(
        int(Y), int(X), int(Z), float(dx_mm), float(dz_mm),
        mu_a.ctypes.data_as(ctypes.c_void_p), mu_s.ctypes.data_as(ctypes.c_void_p), float(g),
        src.ctypes.data_as(ctypes.c_void_p), 1 if lateral_robin else 0, float(tol),
        int(max_iters), phi.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it),
        ctypes.byref(rel)))
    return phi, it.value, rel.value


def semicircle_kernel(Z, k, T, dims, lateral_ratio, focal_depth, focal_sample, eta, eir):
    """The paper-literal per-depth kernel K[Z][k][k][T] (FP64 numpy array):
    the spatial response eta [Z][k][k] on the discrete half spheres of each
    time sample (Eqs. q-above-final / q-below-final), convolved along t with
    the centred impulse response eir.  Host only (no GPU); see
    swopt_semicircle_kernel in include/swopt.h."""
    import numpy as np
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    eir = np.ascontiguousarray(eir, dtype=np.float64)
    if eta.shape != (Z, k, k) or eir.ndim != 1:
        raise ValueError("eta must be [Z][k][k] and eir one-dimensional")
    out = np.empty((Z, k, k, T), dtype=np.float64)
    _check(lib().swopt_semicircle_kernel(int(Z), int(k), int(T), int(dims), float(lateral_ratio),
                                         float(focal_depth), int(focal_sample),
                                         eta.ctypes.data, eir.ctypes.data, int(eir.size),
                                         out.ctypes.data))
    return out


def _check(status: int):
    if status != 0:
        msg = lib().swopt_last_error().decode(errors="replace")
        raise SwoptError(status, msg)


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class SolveParams:
    """Settings of Algorithm 1 (see ``swopt_solve_params``)."""

    def __init__(self, step=0.0, lambda_l1=1e-3, lambda_tv=1e-3, inner_iters=10, max_iters=100,
                 eps1=0.0, eps2=0.0, momentum="beck_teboulle", inner_momentum="beck_teboulle",
                 power_iters=100, refine_every=0, refine_precision="bf16x3", refine_budget=0.0,
                 lambda_3=0.0, joint_step2=0.0):
        self.step = step
        self.lambda_l1 = lambda_l1
        self.lambda_tv = lambda_tv
        self.inner_iters = inner_iters
        self.max_iters = max_iters
        self.eps1 = eps1
        self.eps2 = eps2
        self.momentum = momentum
        self.inner_momentum = inner_momentum
        self.power_iters = power_iters
        self.refine_every = refine_every
        self.refine_precision = refine_precision
        self.refine_budget = refine_budget
        self.lambda_3 = lambda_3
        self.joint_step2 = joint_step2

    def _c(self, history=None):
        p = _SolveParams()
        p.step = float(self.step)
        p.lambda_l1 = float(self.lambda_l1)
        p.lambda_tv = float(self.lambda_tv)
        p.inner_iters = int(self.inner_iters)
        p.max_iters = int(self.max_iters)
        p.eps1 = float(self.eps1)
        p.eps2 = float(self.eps2)
        p.momentum = MOMENTUM[self.momentum] if isinstance(self.momentum, str) else int(self.momentum)
        p.inner_momentum = (MOMENTUM[self.inner_momentum] if isinstance(self.inner_momentum, str)
                            else int(self.inner_momentum))
        p.power_iters = int(self.power_iters)
        p.refine_every = int(self.refine_every)
        p.refine_precision = (PRECISION[self.refine_precision]
                              if isinstance(self.refine_precision, str)
                              else int(self.refine_precision))
        p.history_host = (history.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                          if history is not None else ctypes.POINTER(ctypes.c_double)())
        p.refine_budget = float(self.refine_budget)
        p.lambda_3 = float(self.lambda_3)
        p.joint_step2 = float(self.joint_step2)
        return p


class Operator:
    """A handle: geometry, FP64 kernel and switching parameters on one GPU.

    ``geom`` and ``sw`` are objects with the fields of ``synth.Geometry`` /
    ``synth.Switching`` (X, Y, Z, T, N, P, k, pulses_per_cycle, dz_mm;
    kappa, eps_bar, eps_off, mu_per_mm).  ``K`` is the FP64 kernel
    [Z][k][k][T] (numpy), copied at creation.
    """

    def __init__(self, geom, K, sw, precision: str = "fp32"):
        L = lib()
        self.geom = geom
        self.sw = sw
        g = _Geometry(int(geom.X), int(geom.Y), int(geom.Z), int(geom.T), int(geom.N),
                      int(geom.P), int(geom.k), int(geom.pulses_per_cycle), float(geom.dz_mm))
        K = np.ascontiguousarray(K, dtype=np.float64)
        if K.shape != (geom.Z, geom.k, geom.k, geom.T):
            raise ValueError(f"kernel shape {K.shape} does not match the geometry")
        s = self._switching_struct(sw.kappa, sw.eps_bar, sw.eps_off, sw.mu_per_mm)
        h = ctypes.c_void_p()
        _check(L.swopt_create(ctypes.byref(g), K.ctypes.data_as(ctypes.c_void_p), ctypes.byref(s),
                              ctypes.byref(h)))
        self._h = h
        self.precision = "fp32"
        if precision != "fp32":
            try:
                self.set_precision(precision)
            except SwoptError:
                self.close()  # a precision the geometry does not support: no handle leaks
                raise
        self.precision = precision

    def _switching_struct(self, kappa, eps_bar, eps_off, mu):
        self._kap = np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
        self._eb = np.ascontiguousarray(eps_bar, dtype=np.float64).reshape(-1)
        self._eo = np.ascontiguousarray(eps_off, dtype=np.float64).reshape(-1)
        for a in (self._kap, self._eb, self._eo):
            if a.shape != (self.geom.P,):
                raise ValueError("switching parameters must have one entry per species")
        self._mu = float(mu)
        dp = ctypes.POINTER(ctypes.c_double)
        return _Switching(self._kap.ctypes.data_as(dp), self._eb.ctypes.data_as(dp),
                          self._eo.ctypes.data_as(dp), self._mu)

    def set_switching(self, kappa=None, mu=None, eps_bar=None, eps_off=None):
        """Replace (some of) the switching parameters of Eq. (final-H)."""
        s = self._switching_struct(self._kap if kappa is None else kappa,
                                   self._eb if eps_bar is None else eps_bar,
                                   self._eo if eps_off is None else eps_off,
                                   self._mu if mu is None else mu)
        _check(lib().swopt_set_switching(self._h, ctypes.byref(s)))

    @property
    def switching(self):
        """(kappa, mu, eps_bar, eps_off) in use (FP64 copies)."""
        return self._kap.copy(), self._mu, self._eb.copy(), self._eo.copy()

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().swopt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: str):
        _check(lib().swopt_set_precision(self._h, PRECISION[precision]))
        self.precision = precision

    @property
    def c_shape(self):
        g = self.geom
        return (g.P, g.Y, g.X, g.Z)

    @property
    def y_shape(self):
        g = self.geom
        return (g.N, g.Y, g.X, g.T)

    def info(self):
        t0, tw, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nnz = ctypes.c_int64()
        _check(lib().swopt_info(self._h, ctypes.byref(t0), ctypes.byref(tw), ctypes.byref(q),
                                ctypes.byref(nnz)))
        return {"t0": t0.value, "tw": tw.value, "states": q.value, "kernel_nnz": nnz.value}

    # -- operators --------------------------------------------------------
    def forward(self, c, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.y_shape, device=c.device, dtype=torch.float32)
        _check(lib().swopt_forward(self._h, _ptr(c, self.c_shape, "c"),
                                   _ptr(out, self.y_shape, "y"), _stream(stream)))
        return out

    def adjoint(self, y, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.c_shape, device=y.device, dtype=torch.float32)
        _check(lib().swopt_adjoint(self._h, _ptr(y, self.y_shape, "y"),
                                   _ptr(out, self.c_shape, "c"), _stream(stream)))
        return out

    def prox_l1(self, x, thresh, nonneg=True, stream=None):
        _check(lib().swopt_prox_l1(self._h, _ptr(x, self.c_shape, "x"), float(thresh),
                                   1 if nonneg else 0, _stream(stream)))
        return x

    def prox_tv(self, z, tau, inner_iters, momentum="beck_teboulle", out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(z)
        _check(lib().swopt_prox_tv(self._h, _ptr(z, self.c_shape, "z"),
                                   _ptr(out, self.c_shape, "x"), float(tau), int(inner_iters),
                                   MOMENTUM[momentum], _stream(stream)))
        return out

    def lipschitz(self, iters=100, v0=None, stream=None):
        L = ctypes.c_double()
        v = _ptr(v0, self.c_shape, "v0") if v0 is not None else ctypes.c_void_p(0)
        _check(lib().swopt_lipschitz(self._h, v, int(iters), ctypes.byref(L), _stream(stream)))
        return L.value

    # -- Algorithm 1 ------------------------------------------------------
    def fista_init(self, y, params: SolveParams, stream=None):
        p = params._c()
        _check(lib().swopt_fista_init(self._h, _ptr(y, self.y_shape, "y"), ctypes.byref(p),
                                      _stream(stream)))

    def fista_step(self, iters=1, stream=None):
        _check(lib().swopt_fista_step(self._h, int(iters), _stream(stream)))

    def fista_get(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.c_shape, device="cuda", dtype=torch.float32)
        _check(lib().swopt_fista_get(self._h, _ptr(out, self.c_shape, "c"), _stream(stream)))
        return out

    def unrolled_vjp(self, y, params: SolveParams, w, stream=None):
        """Gradient of <w, c_K> with respect to (kappa, mu) through the
        unrolled solve (see swopt_unrolled_vjp).  Returns (c_K, dkappa, dmu)."""
        import torch
        c = torch.empty(self.c_shape, device=y.device, dtype=torch.float32)
        dk = np.zeros(self.geom.P)
        dm = ctypes.c_double()
        p = params._c()
        _check(lib().swopt_unrolled_vjp(self._h, _ptr(y, self.y_shape, "y"), ctypes.byref(p),
                                        _ptr(w, self.c_shape, "w"), _ptr(c, self.c_shape, "c"),
                                        dk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.byref(dm), _stream(stream)))
        return c, dk, dm.value

    def set_fluence(self, phi=None):
        """Depth profile Phi_j [Z] used in Eq. (final-H) instead of
        exp(-mu j dz) (None restores it); see swopt_set_fluence."""
        if phi is None:
            _check(lib().swopt_set_fluence(self._h, None))
            return
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        if phi.shape != (self.geom.Z,):
            raise ValueError("the fluence profile needs one value per depth")
        _check(lib().swopt_set_fluence(self._h, phi.ctypes.data_as(ctypes.c_void_p)))

    def set_state_offset(self, offset):
        """First switching state of this handle's pulses (see swopt_set_state_offset)."""
        _check(lib().swopt_set_state_offset(self._h, int(offset)))

    def fista_gradient(self, carry=None, out=None, stream=None):
        """H^T (H xi - y) at the momentum iterate, the P^T sum continued from
        ``carry`` (see swopt_fista_gradient)."""
        import torch
        if out is None:
            out = torch.empty(self.c_shape, device="cuda", dtype=torch.float32)
        _check(lib().swopt_fista_gradient(
            self._h, _ptr(carry, self.c_shape, "carry") if carry is not None else None,
            _ptr(out, self.c_shape, "g"), _stream(stream)))
        return out

    def fista_step_external(self, g, stream=None):
        """One FISTA iteration with the supplied data-fit gradient."""
        _check(lib().swopt_fista_step_external(self._h, _ptr(g, self.c_shape, "g"),
                                               _stream(stream)))

    def refine_stats(self, stream=None):
        """(iterations, exact gradients) of the refined solve since fista_init."""
        it, rs = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().swopt_refine_stats(self._h, ctypes.byref(it), ctypes.byref(rs),
                                        _stream(stream)))
        return it.value, rs.value

    def fista_save(self, stream=None) -> bytes:
        """Checkpoint of the FISTA state (host bytes)."""
        n = ctypes.c_size_t()
        _check(lib().swopt_fista_state_bytes(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().swopt_fista_save(self._h, buf, n, _stream(stream)))
        return buf.raw

    def fista_restore(self, state: bytes, stream=None):
        """Load a checkpoint into this handle (after fista_init with the same
        measurements and settings)."""
        buf = ctypes.create_string_buffer(state, len(state))
        _check(lib().swopt_fista_restore(self._h, buf, len(state), _stream(stream)))

    def debug_barrier(self, phantom_arrivals=0, poll_limit=0):
        """Failure-detection test hook of the TV prox's grid barrier."""
        _check(lib().swopt_debug_barrier(self._h, int(phantom_arrivals), int(poll_limit)))

    def solve(self, y, params: SolveParams, history=False, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.c_shape, device=y.device, dtype=torch.float32)
        hist = np.zeros(params.max_iters) if history else None
        p = params._c(hist)
        st = _SolveStats()
        _check(lib().swopt_solve(self._h, _ptr(y, self.y_shape, "y"), _ptr(out, self.c_shape, "c"),
                                 ctypes.byref(p), ctypes.byref(st), _stream(stream)))
        stats = {"iters": st.iters, "step": st.step, "objective": st.objective,
                 "data_fit": st.data_fit}
        if history:
            stats["history"] = hist[: st.iters]
        return out, stats

    def prox_joint(self, z, alpha, lambda_tv, lambda_l1, lambda_b, iters, step2, out=None,
                   stream=None):
        """prox of alpha (R3 + delta_{>=0}) with the lambda_3 term (lambda_b),
        Algorithm 2 on the stacked L (see swopt_prox_joint)."""
        import torch
        if out is None:
            out = torch.empty(self.c_shape, device=z.device, dtype=torch.float32)
        _check(lib().swopt_prox_joint(self._h, _ptr(z, self.c_shape, "z"),
                                      _ptr(out, self.c_shape, "x"), float(alpha),
                                      float(lambda_tv), float(lambda_l1), float(lambda_b),
                                      int(iters), float(step2), _stream(stream)))
        return out

    def prox_joint_step_bound(self, lambda_tv, lambda_l1, lambda_b):
        """An upper bound of eig_max(L L^T) for prox_joint's stacked L."""
        return float(lib().swopt_prox_joint_step_bound(self._h, float(lambda_tv),
                                                       float(lambda_l1), float(lambda_b)))

    def objective(self, c, y, lambda_l1, lambda_tv, lambda_3=0.0, stream=None):
        F, fit = ctypes.c_double(), ctypes.c_double()
        _check(lib().swopt_objective(self._h, _ptr(c, self.c_shape, "c"),
                                     _ptr(y, self.y_shape, "y"), float(lambda_l1),
                                     float(lambda_tv), float(lambda_3), ctypes.byref(F),
                                     ctypes.byref(fit), _stream(stream)))
        return F.value, fit.value

    def param_grad(self, c, y, stream=None):
        dk = np.zeros(self.geom.P)
        dmu = ctypes.c_double()
        _check(lib().swopt_param_grad(self._h, _ptr(c, self.c_shape, "c"),
                                      _ptr(y, self.y_shape, "y"),
                                      dk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.byref(dmu), _stream(stream)))
        return dk, dmu.value

    def param_vjp(self, c, w, stream=None):
        """(dkappa [P], dmu) = <w, d(H c)/d(kappa, mu)> for a cotangent w [N][Y][X][T]."""
        dk = np.zeros(self.geom.P)
        dmu = ctypes.c_double()
        _check(lib().swopt_param_vjp(self._h, _ptr(c, self.c_shape, "c"),
                                     _ptr(w, self.y_shape, "w"),
                                     dk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     ctypes.byref(dmu), _stream(stream)))
        return dk, dmu.value

    # -- instrumentation --------------------------------------------------
    def use_graphs(self, on=True):
        _check(lib().swopt_use_graphs(self._h, 1 if on else 0))

    def profile(self, on=True):
        _check(lib().swopt_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, kernel_id):
        ms, n, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().swopt_profile_read(self._h, int(kernel_id), ctypes.byref(ms), ctypes.byref(n),
                                        ctypes.byref(fl)))
        return {"total_ms": ms.value, "launches": n.value, "flops_per_launch": fl.value}

    def check_device(self, stream=None):
        _check(lib().swopt_check_device(self._h, _stream(stream)))

    def issued_flops(self, kernel_id):
        f = ctypes.c_double()
        _check(lib().swopt_issued_flops(self._h, int(kernel_id), ctypes.byref(f)))
        return f.value

    def tc_configure(self, kernel_id, tiles_per_cta=0, ctas_per_sm=0, accumulators=0):
        _check(lib().swopt_tc_configure(self._h, int(kernel_id), int(tiles_per_cta),
                                        int(ctas_per_sm), int(accumulators)))

    def tc_config(self, kernel_id):
        v = [ctypes.c_int() for _ in range(5)]
        _check(lib().swopt_tc_config(self._h, int(kernel_id), *[ctypes.byref(x) for x in v]))
        return {"tiles_per_cta": v[0].value, "ctas_per_sm": v[1].value, "stages": v[2].value,
                "groups": v[3].value, "accumulators": v[4].value}

    def tc_schedule(self, kernel_id, split=0, buffers=0):
        """Pin the work split (1 whole pairs, 2 equal shares of all runs) and
        the accumulator buffers (1 or 2) of a contraction; 0 leaves the timed
        choice."""
        _check(lib().swopt_tc_schedule(self._h, int(kernel_id), int(split), int(buffers)))

    def tc_schedule_info(self, kernel_id):
        v = [ctypes.c_int() for _ in range(4)]
        _check(lib().swopt_tc_schedule_info(self._h, int(kernel_id),
                                            *[ctypes.byref(x) for x in v]))
        return {"split": v[0].value, "buffers": v[1].value, "grid": v[2].value,
                "max_pieces": v[3].value}

    def launch_count(self):
        n = ctypes.c_int64()
        _check(lib().swopt_launch_count(self._h, ctypes.byref(n)))
        return n.value


def two_step(geom, K, sw, y, acoustic: "SolveParams", unmixing: "SolveParams", b_out=None,
             c_out=None, stream=None):
    """The two-step approach: per-pulse acoustic inversion (TV) into b
    [N][Y][X][Z], then unmixing (l1 + TV) of b into c [P][Y][X][Z]; see
    swopt_two_step.  Returns (c, b)."""
    import torch
    g = _Geometry(int(geom.X), int(geom.Y), int(geom.Z), int(geom.T), int(geom.N),
                  int(geom.P), int(geom.k), int(geom.pulses_per_cycle), float(geom.dz_mm))
    K = np.ascontiguousarray(K, dtype=np.float64)
    if K.shape != (geom.Z, geom.k, geom.k, geom.T):
        raise ValueError(f"kernel shape {K.shape} does not match the geometry")
    arrs = [np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
            for v in (sw.kappa, sw.eps_bar, sw.eps_off)]
    if any(a.shape != (geom.P,) for a in arrs):
        raise ValueError("switching parameters must have one entry per species")
    dp = ctypes.POINTER(ctypes.c_double)
    s = _Switching(*(a.ctypes.data_as(dp) for a in arrs), float(sw.mu_per_mm))
    b_shape = (geom.N, geom.Y, geom.X, geom.Z)
    c_shape = (geom.P, geom.Y, geom.X, geom.Z)
    if b_out is None:
        b_out = torch.empty(b_shape, device=y.device, dtype=torch.float32)
    if c_out is None:
        c_out = torch.empty(c_shape, device=y.device, dtype=torch.float32)
    pa, pu = acoustic._c(None), unmixing._c(None)
    _check(lib().swopt_two_step(ctypes.byref(g), K.ctypes.data, ctypes.byref(s),
                                _ptr(y, (geom.N, geom.Y, geom.X, geom.T), "y"),
                                _ptr(b_out, b_shape, "b"), _ptr(c_out, c_shape, "c"),
                                ctypes.byref(pa), ctypes.byref(pu), _stream(stream)))
    return c_out, b_out


class Batch:
    """Independent problems stepped together (``swopt_batch_*``): every
    iteration of all of them is one CUDA graph with a stream per problem, or
    (``shared=True``) with the contractions as persistent launches over all
    problems' tile-states.  Each operator must have been ``fista_init``-ed
    (same refine_every)."""

    def __init__(self, ops, shared=False):
        self.ops = list(ops)
        arr = (ctypes.c_void_p * len(self.ops))(*[o._h.value for o in self.ops])
        b = ctypes.c_void_p()
        _check(lib().swopt_batch_create(arr, len(self.ops), ctypes.byref(b)))
        self._b = b
        if shared:
            _check(lib().swopt_batch_configure(self._b, 1))

    def shared_in_use(self):
        """True when every captured iteration graph uses shared launches."""
        v, n = ctypes.c_int(), ctypes.c_int()
        _check(lib().swopt_batch_query(self._b, ctypes.byref(v), ctypes.byref(n)))
        return bool(v.value)

    def contraction_launches(self):
        """Contraction kernels of one gradient path per iteration (see
        swopt_batch_query)."""
        v, n = ctypes.c_int(), ctypes.c_int()
        _check(lib().swopt_batch_query(self._b, ctypes.byref(v), ctypes.byref(n)))
        return n.value

    def step(self, iters=1, stream=None):
        _check(lib().swopt_batch_step(self._b, int(iters), _stream(stream)))

    def close(self):
        if getattr(self, "_b", None):
            lib().swopt_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_HFUNCTION = None


def _make_hfunction():
    import torch

    class HFunction(torch.autograd.Function):
        """y = H(kappa, mu) c on the GPU, differentiable in c, kappa and mu.

        ``HFunction.apply(c, kappa, mu, op)``: c [P][Y][X][Z] float32 on the
        GPU; kappa a tensor of P switching rates and mu a scalar tensor (any
        device and dtype; used in FP64); eps_bar / eps_off stay those of
        ``op``.  Forward sets the operator's switching parameters and applies
        H.  Backward: the hand-written adjoint H^T for c, and
        ``swopt_param_vjp`` (the cotangent contracted with dH/dkappa c and
        dH/dmu c) for kappa and mu.
        """

        @staticmethod
        def forward(ctx, c, kappa, mu, op):
            k = kappa.detach().double().cpu().numpy().reshape(-1)
            m = float(mu.detach().double().cpu())
            op.set_switching(kappa=k, mu=m)
            ctx.op, ctx.k, ctx.m = op, k, m
            ctx.kdev, ctx.kdtype = kappa.device, kappa.dtype
            ctx.mdev, ctx.mdtype = mu.device, mu.dtype
            ctx.save_for_backward(c)
            return op.forward(c.contiguous())

        @staticmethod
        def backward(ctx, gy):
            (c,) = ctx.saved_tensors
            op = ctx.op
            k0, m0 = op.switching[0], op.switching[1]
            if not (np.array_equal(k0, ctx.k) and m0 == ctx.m):
                op.set_switching(kappa=ctx.k, mu=ctx.m)
            gy = gy.contiguous()
            gc = op.adjoint(gy) if ctx.needs_input_grad[0] else None
            gk = gm = None
            if ctx.needs_input_grad[1] or ctx.needs_input_grad[2]:
                dk, dmu = op.param_vjp(c.contiguous(), gy)
                gk = torch.tensor(dk, dtype=ctx.kdtype, device=ctx.kdev)
                gm = torch.tensor(dmu, dtype=ctx.mdtype, device=ctx.mdev)
            return gc, gk, gm, None

    return HFunction


def __getattr__(name):
    # torch is imported only when the autograd function is first used
    global _HFUNCTION
    if name == "HFunction":
        if _HFUNCTION is None:
            _HFUNCTION = _make_hfunction()
        return _HFUNCTION
    raise AttributeError(name)
