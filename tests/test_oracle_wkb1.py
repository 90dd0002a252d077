"""Pins of the oracle's non-local model to second order (reading R12): the
WKB0 bilinear transport of Eq. 3 minus the diffraction-pressure (WKB1) term
of Eq. 1, eps^2/(4 p^4) D_i(I_s D_i Q_s), evaluated on the detector grid with
the object intensity.  CPU only."""
import math

import numpy as np

from paper_2601_22793_gb300 import phantoms as ph


def test_wkb1_term_closed_form_at_zero_shift(oracle):
    """delta = 0 (no shift): P = I - eps^2/(4 p^4) D_x(I D_x Q), whose
    first-order response to sqrt(I) = 1 + a cos(theta x) follows from the
    discrete symbols of the stencils: P - I = -eps^2/(4 p^4) a (2 - 2 cos
    theta) sin^2(theta) cos(theta x)."""
    nx, ny, p, L, E, beta = 96, 6, 1e-6, 1.0, 10.0, 1e-8
    a, m = 1e-5, 9
    theta = 2 * np.pi * m / nx
    ln = oracle.Lines([E], [0.0], [beta], [1.0], L=L, pixel=p)
    f, mu, k, c, eps = ln.params()
    xs = np.arange(nx, dtype=float)
    sq = 1 + a * np.cos(theta * xs)
    T = (-2.0 * np.log(sq) / mu[0])[None, :].repeat(ny, 0)
    P3 = oracle.forward(ln, T, model=oracle.MODEL_NONLOCAL_WKB1)[ny // 2]
    coef = eps[0] ** 2 / (4 * p ** 4)
    want = -coef * a * (2 - 2 * np.cos(theta)) * np.sin(theta) ** 2 * np.cos(theta * xs)
    sl = slice(4, -4)
    assert np.abs(want).max() > 1e-4
    assert np.allclose((P3 - sq ** 2)[sl], want[sl], rtol=0, atol=2e-4 * np.abs(want).max())


def test_wkb1_term_uses_the_object_intensity(oracle):
    """With multi-pixel shifts, model 3 minus the plain transport is the
    diffraction-pressure term of the unshifted object intensity, which is the
    local closure of order 2 at delta = 0 minus I; per line, two lines."""
    p, L = 20e-6, 30.0
    tau = ph.spheres(96, 80, 4, 6.0, 16.0, 10.0, p, seed=8)
    E, d, b, w = [70.0, 110.0], [2.6e-7, 1.06e-7], [1.7e-10, 2.8e-11], [0.6, 0.4]
    ln = oracle.Lines(E, d, b, w, L=L, pixel=p)
    l0 = oracle.Lines(E, [0.0, 0.0], b, w, L=L, pixel=p)
    P3, P3s, _ = oracle.forward(ln, tau, model=oracle.MODEL_NONLOCAL_WKB1, per_line=True)
    P0, P0s, _ = oracle.forward(ln, tau, model=oracle.MODEL_NONLOCAL, per_line=True)
    P2, P2s, _ = oracle.forward(l0, tau, model=oracle.MODEL_LOCAL2, per_line=True)
    f, mu, *_ = ln.params()
    # the shifts are several pixels, so transporting the term would differ
    gy, gx = oracle.gradient(tau)
    assert np.abs(ln.params()[3][0] * gx).max() > 2.0
    for s in range(2):
        I = f[s] * np.exp(-mu[s] * tau)
        term = P2s[s] - I
        assert np.abs(term).max() > 1e-6
        assert np.allclose(P3s[s] - P0s[s], term, rtol=0, atol=1e-12)
    assert np.allclose(P3, P3s.sum(0), rtol=0, atol=1e-14)


def test_wkb1_model_conserves_mass(oracle):
    p = 20e-6
    tau = ph.spheres(64, 64, 3, 5.0, 10.0, 10.0, p, seed=3)
    ln = oracle.Lines([80.0], [2e-7], [1e-10], [1.0], L=30.0, pixel=p)
    f, mu, *_ = ln.params()
    P, _, dropped = oracle.forward(ln, tau, model=oracle.MODEL_NONLOCAL_WKB1, per_line=True)
    I = np.exp(-mu[0] * tau)
    assert dropped[0] == 0.0
    assert math.isclose(P.sum(), I.sum(), rel_tol=1e-12)


def test_wkb1_solve_fixed_point_and_descent(oracle):
    """Exact model-3 data are a fixed point of the model-3 solve, and from the
    flat field the relative update falls."""
    p = 20e-6
    tau = ph.spheres(64, 64, 3, 6.0, 12.0, 10.0, p, seed=5) * 0.3
    ln = oracle.Lines([70.0, 110.0], [2.6e-7, 1.06e-7], [1.7e-10, 2.8e-11], [0.6, 0.4],
                      L=10.0, pixel=p)
    D = oracle.forward(ln, tau, model=oracle.MODEL_NONLOCAL_WKB1)
    T, info = oracle.solve(ln, D, T0=tau, n_iter=1, model=oracle.MODEL_NONLOCAL_WKB1)
    assert np.abs(T - tau).max() < 1e-11 * tau.max()
    assert info["rho"][0] < 1e-14
    T, info = oracle.solve(ln, D, n_iter=30, omega=0.5, model=oracle.MODEL_NONLOCAL_WKB1)
    k = info["kappa"]
    assert k[-1] < 0.05 * k[1]
    assert np.linalg.norm(T - tau) / np.linalg.norm(tau) < 0.2
