"""Pins of the oracle's solve on an oversampled internal grid (the paper
solves on grids whose pixel is the detector pixel divided by o; reading R11:
model on the fine grid, residual against the detector image as the mean of
each o x o block, replicated back to the fine pixels).  CPU only."""
import numpy as np
import pytest


def _bumps(n, centres):
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    out = np.zeros((n, n))
    for cx, cy, R, A in centres:
        r2 = ((xx - cx) ** 2 + (yy - cy) ** 2) / R ** 2
        out += A * np.where(r2 < 1, (1 - r2) ** 2, 0.0)
    return out


def test_block_mean(oracle):
    g = np.random.default_rng(0)
    det = g.normal(size=(6, 5))
    for os_ in (1, 2, 3, 4):
        fine = np.kron(det, np.ones((os_, os_)))          # replication
        assert np.allclose(oracle.bin_mean(fine, os_), det, rtol=0, atol=1e-15)
        f = g.normal(size=(6 * os_, 5 * os_))
        assert np.isclose(oracle.bin_mean(f, os_).sum() * os_ * os_, f.sum(), rtol=1e-13)
        assert np.allclose(oracle.bin_mean(np.full_like(f, 2.5), os_), 2.5, rtol=0, atol=0)


def test_factor_one_is_the_plain_solve(oracle):
    g = np.random.default_rng(1)
    ln = oracle.Lines([60.0, 90.0], [1.4e-7, 7e-8], [9e-11, 3e-11], [0.6, 0.4], L=0.05,
                      pixel=6.5e-6)
    tau = _bumps(24, [(11.0, 12.5, 7.0, 2e-3)])
    D = oracle.forward(ln, tau) * (1 + 1e-3 * g.normal(size=tau.shape))
    for model in (oracle.MODEL_NONLOCAL, oracle.MODEL_LOCAL2):
        Ta, ia = oracle.solve(ln, D, n_iter=7, omega=0.7, model=model)
        Tb, ib = oracle.solve_os(ln, D, 1, n_iter=7, omega=0.7, model=model)
        assert np.array_equal(Ta, Tb) and np.array_equal(ia["rho"], ib["rho"])


def test_flat_field_stays_flat(oracle):
    ln = oracle.Lines([60.0], [1.4e-7], [9e-11], [1.0], L=0.05, pixel=13e-6)
    T, info = oracle.solve_os(ln, np.ones((12, 10)), 2, n_iter=5)
    assert T.shape == (24, 20) and np.all(T == 0.0) and np.all(info["rho"] == 0.0)


@pytest.mark.parametrize("os_,model,lines", [(2, 0, 1), (2, 1, 1), (2, 2, 1), (4, 0, 2)])
def test_solve_reproduces_the_detector_data(oracle, os_, model, lines):
    """Noise-free data made on the fine grid and averaged to the detector: the
    solve reaches a fine thickness whose averaged model equals the data to
    round-off (the fine thickness itself is not unique)."""
    p_det, nd = 13e-6, 16
    n = nd * os_
    s = n / 32.0
    tau = _bumps(n, [(14.6 * s, 16.4 * s, 10.0 * s, 2e-3), (19.2 * s, 12.2 * s, 7.0 * s, 1.32e-3)])
    E, d, b, w = ([60.0], [1.4e-7], [9e-11], [1.0]) if lines == 1 else \
        ([60.0, 90.0], [1.4e-7, 7e-8], [9e-11, 3e-11], [0.6, 0.4])
    fine = oracle.Lines(E, d, b, w, L=0.05, pixel=p_det / os_)
    D = oracle.bin_mean(oracle.forward(fine, tau, model=model), os_)
    ln = oracle.Lines(E, d, b, w, L=0.05, pixel=p_det)
    T, info = oracle.solve_os(ln, D, os_, n_iter=200, omega=1.0, model=model)
    assert info["rho"][-1] < 1e-13
    assert np.abs(oracle.bin_mean(oracle.forward(fine, T, model=model), os_) - D).max() < 1e-13
    # and it is not the trivial answer: the thickness moved from the flat field
    assert np.linalg.norm(oracle.bin_mean(T, os_) - oracle.bin_mean(tau, os_)) < \
        0.05 * np.linalg.norm(oracle.bin_mean(tau, os_))


def test_first_iteration_is_paganin_of_the_replicated_data(oracle):
    """From tau = 0 (flat model, mean 1 on every block) with omega = 1 the
    first update is the Paganin retrieval of the detector image replicated
    to the fine grid, with the fine pixel p / o in the filter (numpy.fft)."""
    nyd, nxd, os_, p, L = 20, 24, 2, 13e-6, 2.0
    ln = oracle.Lines([60.0], [1.4e-7], [9e-11], [1.0], L=L, pixel=p)
    f, mu, *_ = ln.params()
    g = np.random.default_rng(12)
    D = 1.0 + 0.05 * g.normal(size=(nyd, nxd))
    T, _ = oracle.solve_os(ln, D, os_, n_iter=1, omega=1.0)
    up = np.kron(D, np.ones((os_, os_)))
    ny, nx, pf = nyd * os_, nxd * os_, p / os_
    fy = np.fft.fftfreq(ny, pf)[:, None]
    fx = np.fft.fftfreq(nx, pf)[None, :]
    H = mu[0] / (mu[0] + L * 1.4e-7 * 4 * np.pi ** 2 * (fx ** 2 + fy ** 2))
    pag = -np.log(np.real(np.fft.ifft2(H * np.fft.fft2(up)))) / mu[0]
    assert np.abs(T - pag).max() < 1e-12 * np.abs(pag).max()
