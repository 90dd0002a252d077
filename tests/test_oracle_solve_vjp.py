"""Pins of the oracle's vector-Jacobian product through the unrolled
non-local solve (calibration gradients: not in the paper).

The derivative it returns is checked against central finite differences of
the oracle solve itself, on a two-line phantom whose shifts stay away from
integer pixel crossings at every iterate (the bilinear transport is not
differentiable there), with no pixel at the update's floor."""
import numpy as np
import pytest

from oracle import oracle as O

NY, NX = 20, 24
E = np.array([60.0, 90.0])
DELTA = 2e-7 * (E[0] / E) ** 2
BETA = 1e-10 * (E[0] / E) ** 4
W = np.array([0.6, 0.4])
L0, PIX = 2.0, 6.5e-6
N_ITER, OMEGA = 4, 0.7


def lines(L=L0, delta=DELTA, beta=BETA):
    return O.Lines(E, delta, beta, W, L=L, pixel=PIX)


def plane():
    y, x = np.mgrid[0:NY, 0:NX].astype(np.float64)
    return 4.75e-5 * x + 3.2e-5 * y


def data():
    y, x = np.mgrid[0:NY, 0:NX].astype(np.float64)
    bump = 8e-5 * np.exp(-((x - 11.0) ** 2 + (y - 9.0) ** 2) / (2 * 5.0 ** 2))
    return O.forward(lines(), plane() + bump)


def tau_n(ln, D, T0, n_iter=N_ITER):
    T, _ = O.solve(ln, D, T0=T0, n_iter=n_iter, omega=OMEGA, tol=0.0)
    return T


def test_shifts_stay_off_integer_crossings_and_above_the_floor():
    """Precondition of the finite-difference pins below: at every iterate the
    shifts keep 0.02 px from an integer, and each line's update
    I_s + omega h_s (split residual, adjoint, preconditioner) stays far above
    the floor eps_I f_s."""
    ln, D, T = lines(), data(), plane()
    f, mu, k, c, eps = ln.params()
    for it in range(N_ITER + 1):
        gy, gx = O.gradient(T)
        for s in range(2):
            for u in (c[s] * gx, c[s] * gy):
                frac = u - np.floor(u)
                assert frac.min() > 0.02 and frac.max() < 0.98, (it, s)
        if it == N_ITER:
            break
        P, Ps, _ = O.forward(ln, T, per_line=True)
        r = D - P
        for s in range(2):
            h = O.precondition(ln, O.adjoint(ln, T, r * Ps[s] / P, line=s), line=s)
            assert (f[s] * np.exp(-mu[s] * T) + OMEGA * h).min() > 0.5 * f[s], (it, s)
        T = tau_n(ln, D, T, 1)


@pytest.fixture(scope="module")
def grads():
    rng = np.random.default_rng(11)
    wts = rng.standard_normal((NY, NX))
    D, T0 = data(), plane()
    g = O.solve_vjp(lines(), D, wts, N_ITER, omega=OMEGA, T0=T0)
    return wts, D, T0, g


def fd(F, x, h):
    return (F(x + h) - F(x - h)) / (2 * h)


def test_gradient_in_L(grads):
    wts, D, T0, (_, _, _, _, Lb) = grads
    d = fd(lambda L: np.sum(wts * tau_n(lines(L=L), D, T0)), L0, 1e-6 * L0)
    assert abs(Lb - d) <= 1e-5 * abs(d)


@pytest.mark.parametrize("s", [0, 1])
def test_gradient_in_delta(grads, s):
    wts, D, T0, (_, _, db, _, _) = grads

    def F(v):
        dl = DELTA.copy()
        dl[s] = v
        return np.sum(wts * tau_n(lines(delta=dl), D, T0))

    d = fd(F, DELTA[s], 1e-6 * DELTA[s])
    assert abs(db[s] - d) <= 1e-5 * abs(d)


@pytest.mark.parametrize("s", [0, 1])
def test_gradient_in_beta(grads, s):
    wts, D, T0, (_, _, _, bb, _) = grads

    def F(v):
        bt = BETA.copy()
        bt[s] = v
        return np.sum(wts * tau_n(lines(beta=bt), D, T0))

    d = fd(F, BETA[s], 1e-6 * BETA[s])
    assert abs(bb[s] - d) <= 1e-5 * abs(d)


def test_gradient_in_the_initial_thickness_and_the_data(grads):
    wts, D, T0, (t0b, Db, _, _, _) = grads
    rng = np.random.default_rng(12)
    y, x = np.mgrid[0:NY, 0:NX].astype(np.float64)
    vT = np.sin(0.3 * x + 0.2 * y) + 0.3 * rng.standard_normal((NY, NX))
    vD = np.cos(0.25 * x - 0.4 * y) + 0.3 * rng.standard_normal((NY, NX))
    ln = lines()
    dT = fd(lambda e: np.sum(wts * tau_n(ln, D, T0 + e * vT)), 0.0, 1e-10)
    dD = fd(lambda e: np.sum(wts * tau_n(ln, D + e * vD, T0)), 0.0, 1e-6)
    assert abs(np.sum(t0b * vT) - dT) <= 1e-5 * abs(dT)
    assert abs(np.sum(Db * vD) - dD) <= 1e-5 * abs(dD)


def test_zero_iterations_is_the_identity_in_the_initial_thickness():
    rng = np.random.default_rng(13)
    wts = rng.standard_normal((NY, NX))
    t0b, Db, db, bb, Lb = O.solve_vjp(lines(), data(), wts, 0, omega=OMEGA, T0=plane())
    assert np.array_equal(t0b, wts)
    assert not Db.any() and not db.any() and not bb.any() and Lb == 0.0
