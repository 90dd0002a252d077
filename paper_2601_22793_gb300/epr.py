"""Thin Python binding of libepr (the C ABI in include/epr.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libepr.so.  The functions carry the C names; arrays are torch
tensors (CUDA or CPU, float32, contiguous) or numpy arrays, passed by data
pointer.  The stream defaults to torch's current CUDA stream.

If libepr.so is missing or cannot be loaded, every call raises RuntimeError:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libepr.so")
_lock = threading.Lock()
_lib = None

EPR_OK = 0
EPR_ERR_INVALID_ARG = 1
EPR_ERR_UNSUPPORTED_SIZE = 2
EPR_ERR_OOM = 3
EPR_ERR_CUDA = 4
EPR_ERR_NONFINITE = 5
EPR_ERR_TIMEOUT = 6
EPR_ERR_NOT_CONVERGED = 7
EPR_ERR_SHIFT_OVERFLOW = 8

EPR_MODEL_NONLOCAL = 0
EPR_MODEL_LOCAL1 = 1
EPR_MODEL_LOCAL2 = 2
EPR_MODEL_NONLOCAL_WKB1 = 3

SYMBOLS = ("epr_plan_create", "epr_plan_destroy", "epr_forward", "epr_adjoint",
           "epr_precondition", "epr_solve_nonlocal", "epr_solve_nonlocal_wkb1", "epr_solve_local",
           "epr_check_device_status", "epr_status_string", "epr_launch_count",
           "epr_profile_enable", "epr_profile_read", "epr_precondition_noalloc", "epr_vjp",
           "epr_batch_create", "epr_batch_destroy", "epr_solve_nonlocal_batched",
           "epr_plan_set_xspec", "epr_solve_vjp", "epr_plan_set_params", "epr_plan_get_tuning",
           "epr_plan_set_tuning")

KERNEL_KINDS = ("splat", "row_fwd", "col", "row_inv", "local", "other")


class epr_options(ctypes.Structure):
    _fields_ = [("max_shift_px", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("overflow_capacity", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("serial_launches", ctypes.c_int),
                ("oversample", ctypes.c_int), ("fft_radix", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


class epr_batch_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("D", ctypes.c_void_p),
                ("T", ctypes.c_void_p)]


class epr_xspec(ctypes.Structure):
    _fields_ = [("n_knots", ctypes.c_int), ("x_knots", ctypes.POINTER(ctypes.c_double)),
                ("weights", ctypes.POINTER(ctypes.c_double)),
                ("delta", ctypes.POINTER(ctypes.c_double)),
                ("beta", ctypes.POINTER(ctypes.c_double))]


class epr_solve_opts(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int), ("omega", ctypes.c_double), ("tol", ctypes.c_double),
                ("eps_I", ctypes.c_double), ("init", ctypes.c_int)]


class epr_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.POINTER(ctypes.c_int)),
                ("rho", ctypes.POINTER(ctypes.c_double)),
                ("kappa", ctypes.POINTER(ctypes.c_double)),
                ("rho_hist", ctypes.POINTER(ctypes.c_double)),
                ("kappa_hist", ctypes.POINTER(ctypes.c_double)),
                ("overflow_sources", ctypes.c_longlong)]


class EprError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


def load(path: str | None = None):
    """Load libepr.so (raises RuntimeError if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libepr.so not found at {p}; build it with "
                               "`python -m paper_2601_22793_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(p)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        lib.epr_plan_create.argtypes = [ctypes.POINTER(vp), i, i, d, d, i, dp, dp, dp, dp,
                                        ctypes.POINTER(epr_options)]
        lib.epr_plan_create.restype = i
        lib.epr_plan_destroy.argtypes = [vp]
        lib.epr_plan_destroy.restype = None
        lib.epr_forward.argtypes = [vp, vp, vp, vp, i, i, vp]
        lib.epr_forward.restype = i
        lib.epr_adjoint.argtypes = [vp, vp, vp, vp, i, i, vp]
        lib.epr_adjoint.restype = i
        lib.epr_precondition.argtypes = [vp, vp, i, i, vp]
        lib.epr_precondition.restype = i
        lib.epr_solve_nonlocal.argtypes = [vp, vp, vp, i, ctypes.POINTER(epr_solve_opts),
                                           ctypes.POINTER(epr_solve_info), vp]
        lib.epr_solve_nonlocal.restype = i
        lib.epr_solve_nonlocal_wkb1.argtypes = [vp, vp, vp, i, ctypes.POINTER(epr_solve_opts),
                                                ctypes.POINTER(epr_solve_info), vp]
        lib.epr_solve_nonlocal_wkb1.restype = i
        lib.epr_solve_local.argtypes = [vp, vp, vp, i, i, ctypes.POINTER(epr_solve_opts),
                                        ctypes.POINTER(epr_solve_info), vp]
        lib.epr_solve_local.restype = i
        lib.epr_check_device_status.argtypes = [vp, vp]
        lib.epr_check_device_status.restype = i
        lib.epr_status_string.argtypes = [i]
        lib.epr_status_string.restype = ctypes.c_char_p
        lib.epr_profile_enable.argtypes = [vp, i]
        lib.epr_profile_enable.restype = i
        lib.epr_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp]
        lib.epr_profile_read.restype = i
        lib.epr_precondition_noalloc.argtypes = [vp, i, i, d, d, d, d, d, i, vp]
        lib.epr_precondition_noalloc.restype = i
        lib.epr_vjp.argtypes = [vp, vp, vp, vp, dp, dp, dp, i, vp]
        lib.epr_vjp.restype = i
        lib.epr_batch_create.argtypes = [ctypes.POINTER(vp), d, d, i, dp, dp, dp, dp,
                                         ctypes.POINTER(epr_options)]
        lib.epr_batch_create.restype = i
        lib.epr_batch_destroy.argtypes = [vp]
        lib.epr_batch_destroy.restype = None
        lib.epr_solve_nonlocal_batched.argtypes = [vp, ctypes.POINTER(epr_batch_desc), i,
                                                   ctypes.POINTER(epr_solve_opts),
                                                   ctypes.POINTER(epr_solve_info), vp]
        lib.epr_solve_nonlocal_batched.restype = i
        lib.epr_solve_vjp.argtypes = [vp, vp, vp, i, i, d, d, i, vp, vp, vp, vp, dp, dp, dp, vp]
        lib.epr_solve_vjp.restype = i
        lib.epr_plan_get_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.epr_plan_get_tuning.restype = i
        lib.epr_plan_set_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.epr_plan_set_tuning.restype = i
        lib.epr_plan_set_params.argtypes = [vp, d, dp, dp]
        lib.epr_plan_set_params.restype = i
        lib.epr_plan_set_xspec.argtypes = [vp, ctypes.POINTER(epr_xspec)]
        lib.epr_plan_set_xspec.restype = i
        lib.epr_launch_count.argtypes = []
        lib.epr_launch_count.restype = ctypes.c_longlong
        _lib = lib
        return lib


def status_string(status: int) -> str:
    try:
        return load().epr_status_string(int(status)).decode()
    except RuntimeError:
        return "libepr not loaded"


def epr_status_string(status: int) -> str:
    return load().epr_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != EPR_OK:
        raise EprError(status, what)


def _ptr(a):
    """Data pointer of a float32 contiguous torch tensor or numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be float32 and C-contiguous")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("tensors must be float32 and contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    import torch
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None


def _darr(x):
    a = np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64)))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _options(max_shift_px, deterministic, overflow_capacity, use_graphs, autotune,
             serial_launches=False, oversample=1, fft_radix=0):
    return epr_options(int(max_shift_px), int(bool(deterministic)), int(overflow_capacity),
                       int(bool(use_graphs)), int(bool(autotune)), int(bool(serial_launches)),
                       int(oversample), int(fft_radix), (ctypes.c_int * 4)())


def epr_plan_create(nx, ny, pixel_m, L_m, energy_keV, delta, beta, weights=None,
                    max_shift_px=4, deterministic=False, overflow_capacity=0, use_graphs=True,
                    autotune=False, serial_launches=False, oversample=1, fft_radix=0):
    """Returns an opaque plan handle (int).  With oversample = o > 1, nx, ny
    and pixel_m are the detector's and the solve runs on the o-times finer
    grid (see epr_options in the C header)."""
    lib = load()
    E, Ep = _darr(energy_keV)
    dl, dp_ = _darr(delta)
    bt, bp = _darr(beta)
    w, wp = _darr(np.ones(E.size) if weights is None else weights)
    opt = _options(max_shift_px, deterministic, overflow_capacity, use_graphs, autotune,
                   serial_launches, oversample, fft_radix)
    h = ctypes.c_void_p()
    _check(lib.epr_plan_create(ctypes.byref(h), int(nx), int(ny), float(pixel_m), float(L_m),
                               int(E.size), Ep, dp_, bp, wp, ctypes.byref(opt)), "epr_plan_create")
    return h.value


def epr_plan_get_tuning(plan) -> dict:
    """The plan's kernel choices (defaults, or the autotuner's)."""
    v = (ctypes.c_int * 9)()
    _check(load().epr_plan_get_tuning(plan, v), "epr_plan_get_tuning")
    return {"splat_tile": [v[0], v[1]], "splat_reach": v[2], "col_tile_width": v[3],
            "col_radix": v[4], "row_blocks_per_sm": v[5], "col_blocks_per_sm": v[6],
            "splat_blocks_per_sm": v[7], "tuned": bool(v[8])}


def epr_plan_set_tuning(plan, tuning: dict):
    """Apply kernel choices in the form epr_plan_get_tuning returns."""
    v = (ctypes.c_int * 9)(tuning["splat_tile"][0], tuning["splat_tile"][1], tuning["splat_reach"],
                           tuning["col_tile_width"], tuning["col_radix"],
                           tuning["row_blocks_per_sm"], tuning.get("col_blocks_per_sm", 4),
                           tuning.get("splat_blocks_per_sm", 5), 1)
    _check(load().epr_plan_set_tuning(plan, v), "epr_plan_set_tuning")


def epr_plan_set_params(plan, L_m, delta, beta):
    """New L, delta_s, beta_s for an existing plan (no reallocation)."""
    dl, dp_ = _darr(delta)
    bt, bp = _darr(beta)
    _check(load().epr_plan_set_params(plan, float(L_m), dp_, bp), "epr_plan_set_params")


def epr_plan_set_xspec(plan, x_knots=None, weights=None, delta=None, beta=None):
    """x-dependent spectrum: knot columns [K] and per-line tables [n_lines][K]
    of weights, delta, beta (see the C header).  x_knots None returns the plan
    to its uniform spectrum."""
    if x_knots is None:
        _check(load().epr_plan_set_xspec(plan, None), "epr_plan_set_xspec")
        return
    X, Xp = _darr(x_knots)
    w, wp = _darr(np.ravel(weights))
    d, dp_ = _darr(np.ravel(delta))
    b, bp = _darr(np.ravel(beta))
    tab = epr_xspec(int(X.size), Xp, wp, dp_, bp)
    _check(load().epr_plan_set_xspec(plan, ctypes.byref(tab)), "epr_plan_set_xspec")


def epr_plan_destroy(plan):
    load().epr_plan_destroy(plan)


def epr_forward(plan, T, P, Ps=None, batch=1, model=EPR_MODEL_NONLOCAL, stream=None):
    _check(load().epr_forward(plan, _ptr(T), _ptr(P), _ptr(Ps), int(batch), int(model),
                              _stream(stream)), "epr_forward")


def epr_adjoint(plan, T, r, g, line=0, batch=1, stream=None):
    _check(load().epr_adjoint(plan, _ptr(T), _ptr(r), _ptr(g), int(line), int(batch),
                              _stream(stream)), "epr_adjoint")


def epr_precondition(plan, g, line=0, batch=1, stream=None):
    _check(load().epr_precondition(plan, _ptr(g), int(line), int(batch), _stream(stream)),
           "epr_precondition")


def epr_precondition_noalloc(g, nx, ny, pixel_m, L_m, energy_keV, delta, beta, batch=1,
                             stream=None):
    """Plan-free preconditioner of one line that allocates no device memory
    (scratch in a static device array; batch * nx * ny <= 4 Mi pixels)."""
    _check(load().epr_precondition_noalloc(_ptr(g), int(nx), int(ny), float(pixel_m), float(L_m),
                                           float(energy_keV), float(delta), float(beta),
                                           int(batch), _stream(stream)),
           "epr_precondition_noalloc")


def epr_vjp(plan, T, gbar, Tbar, n_lines, batch=1, scalars=True, stream=None):
    """Tbar <- dF/dT for F = <gbar, P(T)>; returns (delta_bar [batch][n_lines],
    beta_bar [batch][n_lines], L_bar [batch]) when `scalars`, else None."""
    if scalars:
        db = np.zeros((batch, n_lines))
        bb = np.zeros((batch, n_lines))
        lb = np.zeros(batch)
        ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in (db, bb, lb)]
    else:
        ptrs = [None, None, None]
    _check(load().epr_vjp(plan, _ptr(T), _ptr(gbar), _ptr(Tbar), *ptrs, int(batch),
                          _stream(stream)), "epr_vjp")
    return (db, bb, lb) if scalars else None


def epr_solve_vjp(plan, D, Tbar, n_lines, n_iter, omega=1.0, T0=None, eps_I=1e-8,
                  checkpoint_every=0, batch=1, T_out=None, T0_bar=None, D_bar=None,
                  scalars=True, stream=None):
    """Reverse mode through n_iter iterations of the non-local solve (device
    tensors): fills T_out, T0_bar, D_bar when given and returns (delta_bar
    [batch][n_lines], beta_bar [batch][n_lines], L_bar [batch]) when
    `scalars`, else None."""
    if scalars:
        db = np.zeros((batch, n_lines))
        bb = np.zeros((batch, n_lines))
        lb = np.zeros(batch)
        ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in (db, bb, lb)]
    else:
        ptrs = [None, None, None]
    _check(load().epr_solve_vjp(plan, _ptr(D), _ptr(T0), int(batch), int(n_iter), float(omega),
                                float(eps_I), int(checkpoint_every), _ptr(Tbar), _ptr(T_out),
                                _ptr(T0_bar), _ptr(D_bar), *ptrs, _stream(stream)),
           "epr_solve_vjp")
    return (db, bb, lb) if scalars else None


def _solve_opts(n_iter, omega, tol, eps_I, init):
    return epr_solve_opts(int(n_iter), float(omega), float(tol), float(eps_I), int(init))


def _info(batch, n_iter):
    arrs = {"iters": np.zeros(batch, np.int32), "rho": np.zeros(batch), "kappa": np.zeros(batch),
            "rho_hist": np.zeros((batch, max(n_iter, 1))),
            "kappa_hist": np.zeros((batch, max(n_iter, 1)))}
    info = epr_solve_info(
        arrs["iters"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        arrs["rho"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        arrs["kappa"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        arrs["rho_hist"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        arrs["kappa_hist"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    return info, arrs


def epr_solve_nonlocal(plan, D, T, batch=1, n_iter=20, omega=1.0, tol=0.0, eps_I=1e-8,
                       init=0, want_info=True, stream=None):
    """Returns a dict of per-projection results (iters, rho, kappa, histories,
    overflow_sources) when want_info, else None (asynchronous)."""
    opts = _solve_opts(n_iter, omega, tol, eps_I, init)
    info, arrs = _info(batch, n_iter) if want_info else (None, None)
    st = load().epr_solve_nonlocal(plan, _ptr(D), _ptr(T), int(batch), ctypes.byref(opts),
                                   ctypes.byref(info) if info is not None else None,
                                   _stream(stream))
    _check(st, "epr_solve_nonlocal")
    if arrs is not None:
        arrs["overflow_sources"] = int(info.overflow_sources)
    return arrs


def epr_solve_nonlocal_wkb1(plan, D, T, batch=1, n_iter=20, omega=1.0, tol=0.0, eps_I=1e-8,
                            init=0, want_info=True, stream=None):
    """The non-local solve with the second-order forward model (see the C header)."""
    opts = _solve_opts(n_iter, omega, tol, eps_I, init)
    info, arrs = _info(batch, n_iter) if want_info else (None, None)
    st = load().epr_solve_nonlocal_wkb1(plan, _ptr(D), _ptr(T), int(batch), ctypes.byref(opts),
                                        ctypes.byref(info) if info is not None else None,
                                        _stream(stream))
    _check(st, "epr_solve_nonlocal_wkb1")
    if arrs is not None:
        arrs["overflow_sources"] = int(info.overflow_sources)
    return arrs


def epr_solve_local(plan, D, T, batch=1, order=2, n_iter=20, omega=1.0, tol=0.0, eps_I=1e-8,
                    init=0, want_info=True, stream=None):
    opts = _solve_opts(n_iter, omega, tol, eps_I, init)
    info, arrs = _info(batch, n_iter) if want_info else (None, None)
    st = load().epr_solve_local(plan, _ptr(D), _ptr(T), int(batch), int(order),
                                ctypes.byref(opts),
                                ctypes.byref(info) if info is not None else None,
                                _stream(stream))
    _check(st, "epr_solve_local")
    if arrs is not None:
        arrs["overflow_sources"] = int(info.overflow_sources)
    return arrs


def epr_batch_create(pixel_m, L_m, energy_keV, delta, beta, weights=None, max_shift_px=4,
                     deterministic=False, overflow_capacity=0, use_graphs=True, autotune=False,
                     serial_launches=False, oversample=1, fft_radix=0):
    """Returns an opaque batch handle (int) for epr_solve_nonlocal_batched
    (oversample > 1 is refused)."""
    lib = load()
    E, Ep = _darr(energy_keV)
    dl, dp_ = _darr(delta)
    bt, bp = _darr(beta)
    w, wp = _darr(np.ones(E.size) if weights is None else weights)
    opt = _options(max_shift_px, deterministic, overflow_capacity, use_graphs, autotune,
                   serial_launches, oversample, fft_radix)
    h = ctypes.c_void_p()
    _check(lib.epr_batch_create(ctypes.byref(h), float(pixel_m), float(L_m), int(E.size), Ep, dp_,
                                bp, wp, ctypes.byref(opt)), "epr_batch_create")
    return h.value


def epr_batch_destroy(batch):
    load().epr_batch_destroy(batch)


def epr_solve_nonlocal_batched(batch, Ds, Ts, n_iter=20, omega=1.0, tol=0.0, eps_I=1e-8,
                               init=0, want_info=True, stream=None):
    """Solve projections of uneven sizes: Ds[i], Ts[i] are [ny_i][nx_i] maps.
    Returns per-projection info (in the order given) when want_info."""
    n = len(Ds)
    descs = (epr_batch_desc * n)()
    for i, (D, T) in enumerate(zip(Ds, Ts)):
        ny, nx = D.shape[-2], D.shape[-1]
        descs[i] = epr_batch_desc(int(nx), int(ny), _ptr(D), _ptr(T))
    opts = _solve_opts(n_iter, omega, tol, eps_I, init)
    info, arrs = _info(n, n_iter) if want_info else (None, None)
    st = load().epr_solve_nonlocal_batched(batch, descs, n, ctypes.byref(opts),
                                           ctypes.byref(info) if info is not None else None,
                                           _stream(stream))
    _check(st, "epr_solve_nonlocal_batched")
    if arrs is not None:
        arrs["overflow_sources"] = int(info.overflow_sources)
    return arrs


def epr_check_device_status(plan, stream=None):
    _check(load().epr_check_device_status(plan, _stream(stream)), "epr_check_device_status")


def epr_profile_enable(plan, enable=True):
    _check(load().epr_profile_enable(plan, int(bool(enable))), "epr_profile_enable")


def epr_profile_read(plan):
    """{kind: (launches, total_ms)} since the last read (synchronises)."""
    n = len(KERNEL_KINDS)
    cnt = (ctypes.c_int * n)()
    ms = (ctypes.c_double * n)()
    _check(load().epr_profile_read(plan, cnt, ms), "epr_profile_read")
    return {k: (int(cnt[i]), float(ms[i])) for i, k in enumerate(KERNEL_KINDS)}


def epr_launch_count() -> int:
    return int(load().epr_launch_count())


class Plan:
    """Owning wrapper of a plan handle (destroyed with the object)."""

    def __init__(self, nx, ny, pixel_m, L_m, energy_keV, delta, beta, weights=None, **opts):
        self.nx, self.ny = int(nx), int(ny)
        self.n_lines = int(np.atleast_1d(energy_keV).size)
        self.handle = epr_plan_create(nx, ny, pixel_m, L_m, energy_keV, delta, beta, weights,
                                      **opts)

    def close(self):
        if getattr(self, "handle", None):
            epr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
