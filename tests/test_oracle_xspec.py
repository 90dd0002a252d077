"""Pins of the oracle's x-dependent effective spectrum (reading R13: the
paper's "Remark on spatially varying spectra", Eq. 6 with db_s(x) and Eq. 7
with f_s(x), gamma_s(x)).  A knot table gives per line and knot column the
weight, delta and beta; the oracle interpolates them linearly in the column,
normalises the weights per column, takes mu_s(x) = 2 k_s beta_s(x) and
c_s(x) = -L delta_s(x) / p^2, and runs the solve with per-column constants
(the preconditioner with each line's column means).  CPU only."""
import numpy as np

from paper_2601_22793_gb300 import phantoms as ph

E3 = [55.0, 85.0, 130.0]


def _table(nx, K=4, seed=1):
    g = np.random.default_rng(seed)
    X = np.sort(g.choice(np.arange(1, nx - 1), size=K, replace=False)).astype(float)
    w = g.uniform(0.2, 1.0, size=(3, K))
    d = np.array([2.4e-7, 1.0e-7, 4.5e-8])[:, None] * g.uniform(0.7, 1.3, size=(3, K))
    b = np.array([2.0e-10, 4.0e-11, 8.0e-12])[:, None] * g.uniform(0.7, 1.3, size=(3, K))
    return X, w, d, b


def test_table_interpolation_is_numpy_interp(oracle):
    nx, L, p = 50, 3.0, 5e-6
    X, w, d, b = _table(nx)
    xs = oracle.XSpec(E3, X, w, d, b, L, p, nx)
    cols = np.arange(nx, dtype=float)
    wi = np.stack([np.interp(cols, X, w[s]) for s in range(3)])
    di = np.stack([np.interp(cols, X, d[s]) for s in range(3)])
    bi = np.stack([np.interp(cols, X, b[s]) for s in range(3)])
    _, mu1, k1, *_ = oracle.Lines(E3, [1e-7] * 3, [1.0] * 3, L=L, pixel=p).params()
    assert np.allclose(xs.f, wi / wi.sum(0), rtol=1e-14, atol=0)
    assert np.allclose(xs.mu, 2 * k1[:, None] * bi, rtol=1e-14, atol=0)
    assert np.allclose(xs.c, -L * di / p ** 2, rtol=1e-14, atol=0)
    assert np.allclose(xs.mu_h, xs.mu.mean(1), rtol=1e-13)
    assert np.allclose(xs.Ld_h, L * di.mean(1), rtol=1e-13)


def test_uniform_table_is_the_plain_solve(oracle):
    wl, tau = ph.spheres_mono_256()
    tau = tau[:96, :128]
    ny, nx = tau.shape
    Es, d, b, w = ph.spectrum(3, 60.0, 140.0, 90.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, 3)
    ln = oracle.Lines(Es, d, b, w, L=wl.L, pixel=wl.pixel)
    xs = oracle.XSpec(Es, [10.0], w[:, None], d[:, None], b[:, None], wl.L, wl.pixel, nx)
    D = ph.poisson(oracle.forward(ln, tau), 1e4, 5)
    assert np.allclose(oracle.forward_x(xs, tau), oracle.forward(ln, tau), rtol=0, atol=1e-15)
    T1, i1 = oracle.solve(ln, D, n_iter=6, omega=0.6)
    T2, i2 = oracle.solve_x(xs, D, n_iter=6, omega=0.6)
    assert np.linalg.norm(T2 - T1) / np.linalg.norm(T1) < 1e-12
    assert np.allclose(i1["rho"], i2["rho"], rtol=1e-12)


def test_transport_free_update_closed_form(oracle):
    """L = 0 and omega = 1: every line is scaled by D / P, so per column
    tau' = tau - (sum_s f_s(x) mu_s(x) / sum_s f_s(x) mu_s(x)^2) ln(D / P)."""
    ny, nx, p = 20, 36, 1e-6
    X, w, d, b = _table(nx, seed=2)
    xs = oracle.XSpec(E3, X, w, d, b, 0.0, p, nx)
    g = np.random.default_rng(3)
    tau = 2e-3 * (1.0 + g.random((ny, nx)))
    I = xs.f[:, None, :] * np.exp(-xs.mu[:, None, :] * tau[None])
    P = I.sum(0)
    D = P * np.exp(g.normal(scale=1.0, size=(ny, nx)))
    T, _ = oracle.solve_x(xs, D, T0=tau, n_iter=1, omega=1.0)
    a = (xs.f * xs.mu).sum(0) / (xs.f * xs.mu ** 2).sum(0)
    ref = tau - a[None, :] * np.log(D / P)
    assert np.abs(T - ref).max() < 1e-12 * np.abs(ref).max()


def test_first_iteration_from_flat_field_closed_form(oracle):
    """From tau = 0 with omega = 1 the split residual of line s is
    (D - 1) f_s(x) and the transport is the identity, so the update is
    I'_s = f_s(x) + F^-1[Hbar_s F[(D - 1) f_s]] with the column-mean symbol
    Hbar_s = mu_h / (mu_h + Ld_h |q|^2), projected with per-column weights."""
    ny, nx, p, L = 48, 64, 4e-6, 1.5
    X, w, d, b = _table(nx, seed=4)
    xs = oracle.XSpec(E3, X, w, d, b, L, p, nx)
    g = np.random.default_rng(5)
    D = 1.0 + 0.05 * g.normal(size=(ny, nx))
    T, _ = oracle.solve_x(xs, D, n_iter=1, omega=1.0)
    fy = np.fft.fftfreq(ny, p)[:, None]
    fx = np.fft.fftfreq(nx, p)[None, :]
    q2 = 4 * np.pi ** 2 * (fx ** 2 + fy ** 2)
    num = np.zeros((ny, nx))
    for s in range(3):
        H = xs.mu_h[s] / (xs.mu_h[s] + xs.Ld_h[s] * q2)
        h = np.real(np.fft.ifft2(H * np.fft.fft2((D - 1.0) * xs.f[s][None, :])))
        In = np.maximum(xs.f[s][None, :] + h, 1e-8 * xs.f[s][None, :])
        num += xs.f[s][None, :] * xs.mu[s][None, :] * np.log(In / xs.f[s][None, :])
    ref = -num / (xs.f * xs.mu ** 2).sum(0)[None, :]
    assert np.abs(T - ref).max() < 1e-10 * np.abs(ref).max()


def test_shift_follows_the_source_column(oracle):
    """A thickness ramp along y with delta piecewise constant by column blocks
    (exact powers of two): every source moves down by the integer k(x) of its
    own column, P_s(y + k(x), x) = I_s(y, x) (to the last bit of exp)."""
    ny, nx = 40, 48
    a = p = 2.0 ** -20
    L = 1.0
    ks = [1, 3, 2]                                  # per block of 16 columns
    X = np.array([0, 15, 16, 31, 32, 47], float)
    dk = np.array([ks[0], ks[0], ks[1], ks[1], ks[2], ks[2]], float) * 2.0 ** -20
    xs = oracle.XSpec([80.0], X, np.ones((1, 6)), dk[None, :], np.full((1, 6), 1e-10), L, p, nx)
    assert np.array_equal(xs.c[0], -np.repeat(np.array(ks, float), 16) * 2.0 ** 20)
    tau = a * (ny - 1 - np.arange(ny, dtype=float))[:, None].repeat(nx, 1)
    P, Ps, _ = oracle.forward_x(xs, tau, per_line=True)
    I = xs.f[0][None, :] * np.exp(-xs.mu[0][None, :] * tau)
    for x in range(nx):
        k = ks[x // 16]
        assert np.allclose(Ps[0][k:ny, x], I[0:ny - k, x], rtol=1e-15, atol=0), x
        assert np.all(Ps[0][:k, x] == 0.0)
