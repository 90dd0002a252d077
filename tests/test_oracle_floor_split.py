"""Pins of two steps of the oracle's update that no other pin reaches.

The positivity floor of the update (reading R7, "Iterative inversion" with
Eq. 7): I'_s = max(I_s + omega h_s, eps_I f_s).  From the flat field with
omega = 1 the first update of line s is I'_s = f_s F^-1[H_s F[D]] (the split
residual of the flat field is (D - 1) f_s, the transport is the identity at
zero shift and H_s(0) = 1), so with a dark block in D the line intensity
falls to the floor inside the block.  The projection of Eq. 7 then gives the
closed form tau' = -sum_s f_s mu_s ln(max(F^-1[H_s F[D]], eps_I)) /
sum_s f_s mu_s^2, written here with numpy.fft.  A floor at eps_I instead of
eps_I f_s, or the floor taken after the logarithm, fails it.

The residual split (reading R5, "Iteration structure": the detector residual
is split across the lines "with positivity-weighted weights").  Without
transport and preconditioning (L = 0: zero shift, H_s = 1) and with omega = 1
the update of line s is I'_s = I_s + w_s (D - P).  A split that distributes
the residual (sum_s w_s = 1) and keeps every updated line positive for every
non-negative D must have w_s <= I_s / P for all s (take D -> 0), and since
both sides sum to one, w_s = I_s / P = P_s / P.  The update is then
I'_s = I_s D / P for every line, and the projection gives
tau' = tau - (sum_s f_s mu_s / sum_s f_s mu_s^2) ln(D / P), checked here in
closed form on data far from the model (where the equal-fraction split r f_s
would drive a line negative).  CPU only."""
import numpy as np
import pytest


def _lines(oracle, L, p):
    # two lines with unequal weights and attenuations; at L = 0.5 mm the
    # filter's length sqrt(L delta / mu) is about one pixel
    return oracle.Lines([55.0, 95.0], [2.4e-7, 8.0e-8], [2.0e-10, 2.6e-11], [0.35, 0.65],
                        L=L, pixel=p)


def _paganin_np(D, p, mu, Ld):
    ny, nx = D.shape
    fy = np.fft.fftfreq(ny, p)[:, None]
    fx = np.fft.fftfreq(nx, p)[None, :]
    H = mu / (mu + Ld * 4 * np.pi ** 2 * (fx ** 2 + fy ** 2))
    return np.real(np.fft.ifft2(H * np.fft.fft2(D)))


def _dark_block_data(ny=64, nx=72):
    g = np.random.default_rng(21)
    D = 1.0 + 0.02 * g.normal(size=(ny, nx))
    D[14:50, 14:58] = 0.0
    return D


@pytest.mark.parametrize("eps_I", [1e-3, 1e-6])
def test_floor_closed_form_on_a_dark_block(oracle, eps_I):
    p, L = 1.0e-6, 5e-4
    ln = _lines(oracle, L, p)
    f, mu, *_ = ln.params()
    D = _dark_block_data()
    T, _ = oracle.solve(ln, D, n_iter=1, omega=1.0, eps_I=eps_I)
    num = np.zeros_like(D)
    low = []
    for s in range(2):
        hD = _paganin_np(D, p, mu[s], L * ln.delta[s])
        low.append(hD < eps_I)
        num += f[s] * mu[s] * np.log(np.maximum(hD, eps_I))
    ref = -num / np.sum(f * mu ** 2)
    # two FP64 FFTs agree to ~1e-16 absolute; ln near the floor amplifies that
    # by 1 / eps_I
    assert np.abs(T - ref).max() < 1e-9 * np.abs(ref).max()
    # both branches of the floor are in play (at eps_I = 1e-6 mostly where
    # the periodic filter rings below zero)
    assert all(m.sum() < D.size - 50 for m in low)
    assert sum(m.sum() for m in low) > 40
    # the floor relative to f_s matters here: a floor at eps_I alone differs
    num_abs = np.zeros_like(D)
    for s in range(2):
        hD = _paganin_np(D, p, mu[s], L * ln.delta[s])
        num_abs += f[s] * mu[s] * np.log(np.maximum(f[s] * hD, eps_I) / f[s])
    alt = -num_abs / np.sum(f * mu ** 2)
    assert np.abs(alt - ref).max() > 1e-3 * np.abs(ref).max()


def test_floor_pixels_take_the_floored_thickness(oracle):
    """Mono: where the first update is floored the thickness is exactly
    -ln(eps_I) / mu."""
    p, L, eps_I = 1.0e-6, 5e-4, 1e-4
    ln = oracle.Lines([55.0], [2.4e-7], [2.0e-10], [1.0], L=L, pixel=p)
    _, mu, *_ = ln.params()
    D = _dark_block_data()
    T, _ = oracle.solve(ln, D, n_iter=1, omega=1.0, eps_I=eps_I)
    hD = _paganin_np(D, p, mu[0], L * 2.4e-7)
    m = hD < eps_I
    assert m.sum() > 100
    assert np.allclose(T[m], -np.log(eps_I) / mu[0], rtol=1e-13, atol=0)
    assert np.allclose(T[~m], -np.log(hD[~m]) / mu[0], rtol=1e-10, atol=1e-18)


def test_split_is_the_positivity_preserving_one(oracle):
    p = 1.0e-6
    ln = oracle.Lines([50.0, 80.0, 140.0], [3e-7, 1.2e-7, 4e-8], [4e-10, 1e-10, 1.5e-11],
                      [0.2, 0.5, 0.3], L=0.0, pixel=p)
    f, mu, *_ = ln.params()
    g = np.random.default_rng(31)
    ny, nx = 24, 40
    tau = 1e-3 * (1.0 + g.random((ny, nx)))
    I = f[:, None, None] * np.exp(-mu[:, None, None] * tau[None])
    P = I.sum(0)
    D = P * np.exp(g.normal(scale=1.5, size=(ny, nx)))   # far from the model, D > 0
    T, _ = oracle.solve(ln, D, T0=tau, n_iter=1, omega=1.0)
    ref = tau - np.sum(f * mu) / np.sum(f * mu ** 2) * np.log(D / P)
    assert np.abs(T - ref).max() < 1e-12 * np.abs(ref).max()
    # the data are far enough from the model that the split r f_s would push
    # some line below zero, so the case tells the two splits apart
    assert (I + f[:, None, None] * (D - P)[None] <= 0).any()
