"""Pins of the oracle's vector-Jacobian product of the non-local forward
against central finite differences of F = <gbar, P(T; L, delta, beta)>.
The bilinear transport is only piecewise smooth (the derivative jumps where
a mapped point crosses a pixel boundary), so the phantom keeps every mapped
point at least 1e-2 px away from integer coordinates, and the test reports
that fraction.  CPU only."""
import numpy as np
import pytest


def _setup(oracle, ny=40, nx=48):
    E, delta, beta = [60.0, 90.0], [1.4e-7, 7e-8], [9e-11, 3e-11]
    p, L = 6.5e-6, 2.0
    ln = oracle.Lines(E, delta, beta, [0.6, 0.4], L=L, pixel=p)
    f, mu, k, c, eps = ln.params()
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    # ramps giving mapped offsets near (0.45, 0.35) px for line 0, smooth
    # variation on top, and an offset that keeps tau positive
    ax, ay = 0.45 / c[0], 0.35 / c[0]
    A = 0.08 * 40 / (2 * np.pi * abs(c[0]))
    tau = 3e-3 + ax * (xx - nx / 2) + ay * (yy - ny / 2) \
        + A * np.sin(2 * np.pi * xx / 40) * np.sin(2 * np.pi * yy / 50)
    return ln, tau, (E, delta, beta, p, L)


def _frac_near_crossing(oracle, ln, tau):
    f, mu, k, c, eps = ln.params()
    gy, gx = oracle.gradient(tau)
    worst = 1.0
    for s in range(ln.n):
        for u in (c[s] * gx, c[s] * gy):
            d = np.abs(u - np.round(u))
            worst = min(worst, d.min())
    return worst


def test_vjp_against_finite_differences(oracle):
    ln, tau, (E, delta, beta, p, L) = _setup(oracle)
    assert _frac_near_crossing(oracle, ln, tau) > 1e-2
    g = np.random.default_rng(1)
    gbar = g.normal(size=tau.shape)
    Tbar, dbar, bbar, Lbar = oracle.vjp(ln, tau, gbar)

    def F(T=tau, L_=L, d=delta, b=beta):
        l2 = oracle.Lines(E, d, b, [0.6, 0.4], L=L_, pixel=p)
        return float(np.sum(gbar * oracle.forward(l2, T)))

    # thickness: along a smooth direction and along a random one
    for v in (np.cos(np.arange(tau.size).reshape(tau.shape) * 0.01),
              g.normal(size=tau.shape)):
        h = 1e-9
        fd = (F(T=tau + h * v) - F(T=tau - h * v)) / (2 * h)
        an = float(np.sum(Tbar * v))
        assert abs(fd - an) <= 1e-6 * abs(an)
    # propagation distance
    h = 1e-6 * L
    fd = (F(L_=L + h) - F(L_=L - h)) / (2 * h)
    assert abs(fd - Lbar) <= 1e-6 * abs(Lbar)
    # per-line delta and beta
    for s in range(2):
        dd = list(delta); hd = 1e-6 * delta[s]
        dp, dm = dd.copy(), dd.copy(); dp[s] += hd; dm[s] -= hd
        fd = (F(d=dp) - F(d=dm)) / (2 * hd)
        assert abs(fd - dbar[s]) <= 1e-6 * abs(dbar[s])
        bb = list(beta); hb = 1e-6 * beta[s]
        bp, bm = bb.copy(), bb.copy(); bp[s] += hb; bm[s] -= hb
        fd = (F(b=bp) - F(b=bm)) / (2 * hb)
        assert abs(fd - bbar[s]) <= 1e-6 * abs(bbar[s])


def test_vjp_shift_free_case_is_the_adjoint_times_intensity_derivative(oracle):
    """delta = 0: no shift, so dF/dtau = -sum_s mu_s I_s gbar exactly."""
    ny, nx = 24, 30
    ln = oracle.Lines([60.0, 80.0], [0.0, 0.0], [9e-11, 5e-11], [1.0, 3.0], L=2.0, pixel=6.5e-6)
    f, mu, *_ = ln.params()
    g = np.random.default_rng(2)
    tau = g.uniform(0.0, 2e-3, size=(ny, nx))
    gbar = g.normal(size=(ny, nx))
    Tbar, dbar, bbar, Lbar = oracle.vjp(ln, tau, gbar)
    want = sum(-mu[s] * f[s] * np.exp(-mu[s] * tau) * gbar for s in range(2))
    assert np.allclose(Tbar, want, rtol=1e-13, atol=0)
