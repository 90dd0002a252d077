"""Python binding of the FP64 CPU oracle (``epr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
CPU-baseline leg of the benchmark are the only callers.  The product library
never imports this module, and this module imports nothing from the product.

Arrays are numpy float64, row-major ``[ny][nx]``.  Every function follows one
passage of arXiv 2601.22793; the C source gives the passage and the reading
taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libepr_oracle.so")
_lock = threading.Lock()
_lib = None

MODEL_NONLOCAL = 0
MODEL_LOCAL1 = 1
MODEL_LOCAL2 = 2
MODEL_NONLOCAL_WKB1 = 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE semantics, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fno-fast-math", "-ffp-contract=off",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            f = ctypes.c_double
            ip = ctypes.POINTER(ctypes.c_int)
            lib.orc_line_params.argtypes = [i, d, d, d, d, f, f, d, d, d, d, d]
            lib.orc_gradient.argtypes = [i, i, d, d, d]
            lib.orc_gradient.restype = None
            lib.orc_splat.argtypes = [i, i, d, d, d, d, d]
            lib.orc_splat.restype = None
            lib.orc_gather.argtypes = [i, i, d, d, d, d]
            lib.orc_gather.restype = None
            lib.orc_fft.argtypes = [i, d, d, i]
            lib.orc_dft_naive.argtypes = [i, d, d, d, d, i]
            lib.orc_dft_naive.restype = None
            lib.orc_fft2.argtypes = [i, i, d, d, i]
            lib.orc_paganin.argtypes = [i, i, f, f, f, d]
            lib.orc_forward.argtypes = [i, i, f, f, i, d, d, d, d, i, d, d, d, d]
            lib.orc_adjoint.argtypes = [i, i, f, f, i, d, d, d, d, i, d, d, d]
            lib.orc_precondition.argtypes = [i, i, f, f, i, d, d, d, d, i, d]
            lib.orc_vjp.argtypes = [i, i, f, f, i, d, d, d, d, d, d, d, d, d, d]
            lib.orc_solve.argtypes = [i, i, f, f, i, d, d, d, d, i, d, d, i, f, f, f,
                                      d, d, ip]
            lib.orc_solve_os.argtypes = [i, i, i, f, f, i, d, d, d, d, i, d, d, i, f, f, f,
                                         d, d, ip]
            lib.orc_bin.argtypes = [i, i, i, d, d]
            lib.orc_bin.restype = None
            lib.orc_solve_vjp.argtypes = [i, i, f, f, i, d, d, d, d, d, d, i, f, f, d, d, d, d,
                                          d, d]
            lib.orc_xspec_params.argtypes = [i, i, d, i, d, d, d, d, f, f, d, d, d, d, d]
            lib.orc_forward_x.argtypes = [i, i, i, d, d, d, d, d, d, d]
            lib.orc_solve_x.argtypes = [i, i, f, i, d, d, d, d, d, d, d, i, f, f, f, d, d, ip]
            lib.orc_forward_fields.argtypes = [i, i, f, f, i, d, d, d, d, d, d]
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


class Lines:
    """Spectrum description shared by the oracle calls: energies in keV,
    delta_s, beta_s and (unnormalised) weights; L and p in metres."""

    def __init__(self, energy_keV, delta, beta, weights=None, L=1.0, pixel=1e-6):
        self.E = _c(np.atleast_1d(energy_keV))
        self.delta = _c(np.atleast_1d(delta))
        self.beta = _c(np.atleast_1d(beta))
        n = self.E.size
        self.w = _c(np.ones(n) if weights is None else np.atleast_1d(weights))
        self.L = float(L)
        self.p = float(pixel)
        if not (self.delta.size == self.beta.size == self.w.size == n):
            raise ValueError("line arrays differ in length")

    @property
    def n(self):
        return int(self.E.size)

    def params(self):
        """(f, mu, k, c, eps) per line (orc_line_params)."""
        lib = _load()
        n = self.n
        out = [np.zeros(n) for _ in range(5)]
        st = lib.orc_line_params(n, _p(self.E), _p(self.delta), _p(self.beta), _p(self.w),
                                 self.L, self.p, *[_p(o) for o in out])
        _check(st, "line_params")
        return tuple(out)

    def _args(self):
        return (self.p, self.L, self.n, _p(self.E), _p(self.delta), _p(self.beta), _p(self.w))


def gradient(T):
    T = _c(T)
    gy = np.empty_like(T)
    gx = np.empty_like(T)
    _load().orc_gradient(T.shape[0], T.shape[1], _p(T), _p(gy), _p(gx))
    return gy, gx


def splat(I, uy, ux):
    """Returns (P, dropped) of the bilinear redistribution of I."""
    I, uy, ux = _c(I), _c(uy), _c(ux)
    P = np.zeros_like(I)
    dropped = np.zeros(1)
    _load().orc_splat(I.shape[0], I.shape[1], _p(I), _p(uy), _p(ux), _p(P), _p(dropped))
    return P, float(dropped[0])


def gather(e, uy, ux):
    e, uy, ux = _c(e), _c(uy), _c(ux)
    g = np.empty_like(e)
    _load().orc_gather(e.shape[0], e.shape[1], _p(e), _p(uy), _p(ux), _p(g))
    return g


def fft(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    re = _c(x.real)
    im = _c(x.imag)
    _check(_load().orc_fft(x.size, _p(re), _p(im), sign), "fft")
    return re + 1j * im


def dft_naive(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    re, im = _c(x.real), _c(x.imag)
    ore, oim = np.empty_like(re), np.empty_like(im)
    _load().orc_dft_naive(x.size, _p(re), _p(im), _p(ore), _p(oim), sign)
    return ore + 1j * oim


def fft2(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    re, im = _c(x.real), _c(x.imag)
    _check(_load().orc_fft2(x.shape[0], x.shape[1], _p(re), _p(im), sign), "fft2")
    return re + 1j * im


def paganin(g, pixel, mu, L_delta):
    g = _c(g).copy()
    _check(_load().orc_paganin(g.shape[0], g.shape[1], pixel, mu, L_delta, _p(g)), "paganin")
    return g


def forward(lines: Lines, T, model=MODEL_NONLOCAL, per_line=False):
    """P (and, with per_line, P_s [n_lines, ny, nx] and dropped [n_lines])."""
    T = _c(T)
    ny, nx = T.shape
    P = np.empty_like(T)
    Ps = np.empty((lines.n, ny, nx)) if per_line else None
    dropped = np.zeros(lines.n) if per_line else None
    st = _load().orc_forward(ny, nx, *lines._args(), model, _p(T), _p(P), _p(Ps), _p(dropped))
    _check(st, "forward")
    return (P, Ps, dropped) if per_line else P


def adjoint(lines: Lines, T, e, line=0):
    T, e = _c(T), _c(e)
    g = np.empty_like(T)
    st = _load().orc_adjoint(T.shape[0], T.shape[1], *lines._args(), line, _p(T), _p(e), _p(g))
    _check(st, "adjoint")
    return g


def precondition(lines: Lines, g, line=0):
    g = _c(g).copy()
    st = _load().orc_precondition(g.shape[0], g.shape[1], *lines._args(), line, _p(g))
    _check(st, "precondition")
    return g


def vjp(lines: Lines, T, gbar):
    """(Tbar, delta_bar[n], beta_bar[n], L_bar) of F = <gbar, P(T)> for the
    non-local forward."""
    T, gbar = _c(T), _c(gbar)
    Tbar = np.empty_like(T)
    db = np.zeros(lines.n)
    bb = np.zeros(lines.n)
    lb = np.zeros(1)
    st = _load().orc_vjp(T.shape[0], T.shape[1], *lines._args(), _p(T), _p(gbar), _p(Tbar),
                         _p(db), _p(bb), _p(lb))
    _check(st, "vjp")
    return Tbar, db, bb, float(lb[0])


def solve_vjp(lines: Lines, D, Tbar, n_iter, omega=1.0, T0=None, eps_I=1e-8):
    """Gradients of F = <Tbar, tau_N>, tau_N the thickness after n_iter
    non-local iterations from T0 (zeros when None), without early stop:
    returns (T0_bar, D_bar, delta_bar[n], beta_bar[n], L_bar)."""
    D, Tbar = _c(D), _c(Tbar)
    T0 = np.zeros_like(D) if T0 is None else _c(T0)
    t0b = np.empty_like(D)
    dbar = np.empty_like(D)
    db = np.zeros(lines.n)
    bb = np.zeros(lines.n)
    lb = np.zeros(1)
    st = _load().orc_solve_vjp(D.shape[0], D.shape[1], *lines._args(), _p(D), _p(T0),
                               int(n_iter), float(omega), float(eps_I), _p(Tbar), _p(t0b),
                               _p(dbar), _p(db), _p(bb), _p(lb))
    _check(st, "solve_vjp")
    return t0b, dbar, db, bb, float(lb[0])


def solve(lines: Lines, D, T0=None, n_iter=20, omega=1.0, tol=0.0, eps_I=1e-8,
          model=MODEL_NONLOCAL):
    """Returns (T, info) with info = {rho, kappa, iters}."""
    D = _c(D)
    T = np.zeros_like(D) if T0 is None else _c(T0).copy()
    rho = np.zeros(max(n_iter, 1))
    kappa = np.zeros(max(n_iter, 1))
    iters = ctypes.c_int(0)
    st = _load().orc_solve(D.shape[0], D.shape[1], *lines._args(), model, _p(D), _p(T),
                           int(n_iter), float(omega), float(tol), float(eps_I),
                           _p(rho), _p(kappa), ctypes.byref(iters))
    _check(st, "solve")
    k = iters.value
    return T, {"rho": rho[:k], "kappa": kappa[:k], "iters": k}


def bin_mean(fine, os_):
    """Detector image of a fine map: the mean of each os x os block."""
    fine = _c(fine)
    nyd, nxd = fine.shape[0] // os_, fine.shape[1] // os_
    det = np.empty((nyd, nxd))
    _load().orc_bin(nyd, nxd, int(os_), _p(fine), _p(det))
    return det


def solve_os(lines: Lines, D, os_, T0=None, n_iter=20, omega=1.0, tol=0.0, eps_I=1e-8,
             model=MODEL_NONLOCAL):
    """Solve on a grid oversampled by os_: D is the detector image (pixel
    lines.p), T the fine thickness [os_ ny][os_ nx].  Returns (T, info)."""
    D = _c(D)
    nyd, nxd = D.shape
    T = np.zeros((nyd * os_, nxd * os_)) if T0 is None else _c(T0).copy()
    rho = np.zeros(max(n_iter, 1))
    kappa = np.zeros(max(n_iter, 1))
    iters = ctypes.c_int(0)
    st = _load().orc_solve_os(nyd, nxd, int(os_), *lines._args(), model, _p(D), _p(T),
                              int(n_iter), float(omega), float(tol), float(eps_I),
                              _p(rho), _p(kappa), ctypes.byref(iters))
    _check(st, "solve_os")
    k = iters.value
    return T, {"rho": rho[:k], "kappa": kappa[:k], "iters": k}


class XSpec:
    """x-dependent spectrum (reading R13): energies E (keV) per line, knot
    columns X (ascending, pixel units) and per-line, per-knot weights, delta
    and beta ([n_lines][K] each); L and p in metres; nx columns."""

    def __init__(self, energy_keV, X, weights, delta, beta, L, pixel, nx):
        self.E = _c(np.atleast_1d(energy_keV))
        self.X = _c(np.atleast_1d(X))
        K = self.X.size
        self.w = _c(np.reshape(weights, (self.E.size, K)))
        self.delta = _c(np.reshape(delta, (self.E.size, K)))
        self.beta = _c(np.reshape(beta, (self.E.size, K)))
        self.L, self.p, self.nx = float(L), float(pixel), int(nx)
        n = self.E.size
        self.f = np.zeros((n, nx))
        self.mu = np.zeros((n, nx))
        self.c = np.zeros((n, nx))
        self.mu_h = np.zeros(n)
        self.Ld_h = np.zeros(n)
        st = _load().orc_xspec_params(nx, n, _p(self.E), K, _p(self.X), _p(self.w),
                                      _p(self.delta), _p(self.beta), self.L, self.p,
                                      _p(self.f), _p(self.mu), _p(self.c), _p(self.mu_h),
                                      _p(self.Ld_h))
        _check(st, "xspec_params")

    @property
    def n(self):
        return int(self.E.size)


def material_fields(lines: Lines, chords, delta_m, beta_m, e_ref_keV):
    """Per-line phase and attenuation line integrals of an object made of
    several materials (orc_forward_fields): ``chords`` [n_mat][ny][nx] are the
    chord lengths (metres) through each material, whose indices at the
    reference energy are ``delta_m``, ``beta_m``; at line s they scale as
    (e_ref / E_s)^2 and (e_ref / E_s)^4 (the away-from-edge scalings of the
    spectra here), mu_{m,s} = 2 k_s beta_{m,s}.  Returns (Phi, A), each
    [n_lines][ny][nx]."""
    chords = np.asarray(chords, dtype=np.float64)
    _, _, k, _, _ = lines.params()
    phi0 = np.tensordot(np.asarray(delta_m, dtype=np.float64), chords, axes=1)
    bet0 = np.tensordot(np.asarray(beta_m, dtype=np.float64), chords, axes=1)
    r = e_ref_keV / lines.E
    Phi = np.stack([phi0 * r[s] ** 2 for s in range(lines.n)])
    A = np.stack([2.0 * k[s] * bet0 * r[s] ** 4 for s in range(lines.n)])
    return Phi, A


def forward_fields(lines: Lines, Phi, A, per_line=False):
    """Non-local forward from per-line phase and attenuation line integrals
    (orc_forward_fields); the energies, delta and beta of ``lines`` are not
    used, only its weights, L and pixel."""
    Phi, A = _c(Phi), _c(A)
    ns, ny, nx = Phi.shape
    assert A.shape == Phi.shape and ns == lines.n
    P = np.empty((ny, nx))
    Ps = np.empty((ns, ny, nx)) if per_line else None
    dropped = np.zeros(ns) if per_line else None
    st = _load().orc_forward_fields(ny, nx, lines.p, lines.L, ns, _p(lines.w), _p(Phi), _p(A),
                                    _p(P), _p(Ps), _p(dropped))
    _check(st, "forward_fields")
    return (P, Ps, dropped) if per_line else P


def forward_x(xs: XSpec, T, per_line=False):
    T = _c(T)
    ny, nx = T.shape
    P = np.empty_like(T)
    Ps = np.empty((xs.n, ny, nx)) if per_line else None
    dropped = np.zeros(xs.n) if per_line else None
    st = _load().orc_forward_x(ny, nx, xs.n, _p(xs.f), _p(xs.mu), _p(xs.c), _p(T), _p(P),
                               _p(Ps), _p(dropped))
    _check(st, "forward_x")
    return (P, Ps, dropped) if per_line else P


def solve_x(xs: XSpec, D, T0=None, n_iter=20, omega=1.0, tol=0.0, eps_I=1e-8):
    D = _c(D)
    T = np.zeros_like(D) if T0 is None else _c(T0).copy()
    rho = np.zeros(max(n_iter, 1))
    kappa = np.zeros(max(n_iter, 1))
    iters = ctypes.c_int(0)
    st = _load().orc_solve_x(D.shape[0], D.shape[1], xs.p, xs.n, _p(xs.f), _p(xs.mu), _p(xs.c),
                             _p(xs.mu_h), _p(xs.Ld_h), _p(D), _p(T), int(n_iter), float(omega),
                             float(tol), float(eps_I), _p(rho), _p(kappa), ctypes.byref(iters))
    _check(st, "solve_x")
    k = iters.value
    return T, {"rho": rho[:k], "kappa": kappa[:k], "iters": k}
