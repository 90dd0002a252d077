"""GPU parity on branches of the update that the workloads do not reach,
against the FP64 oracle through the C ABI.

* The positivity floor of the update, I'_s = max(I_s + omega h_s, eps_I f_s)
  ("Iterative inversion", Eq. 7): data with a dark block drive the first
  update of every line below the floor inside the block.  eps_I = 1e-3 keeps
  the floor far above the float32 rounding of the filtered data, so both
  sides take the same branch except where the value is within rounding of
  the floor, where max() is continuous.
* A solve that starts from the caller's thickness (init = 1).
* The residual split without transport (L = 0): with omega = 1 every line is
  scaled by D / P (the positivity-preserving split), on data far from the
  model.
* An overflow list too small for the long-shift sources: the condition is
  reported (and cleared by the check), and a list with room for every pixel
  gives the oracle's forward.

Tolerance: relative L2 <= 1e-4 on the thickness."""
import numpy as np
import pytest

from paper_2601_22793_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_22793_gb300 import build
    build.build()
    from paper_2601_22793_gb300 import epr
    epr.load()
    return torch


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gpu_solve(torch, E, nx, ny, p, L, Es, d, b, w, D, n_iter, omega, eps_I=1e-8, T0=None,
               **kw):
    with E.Plan(nx, ny, p, L, Es, d, b, w, **kw) as plan:
        Dd = torch.from_numpy(np.ascontiguousarray(D, np.float32)).cuda()
        T = torch.zeros_like(Dd) if T0 is None else torch.from_numpy(
            np.ascontiguousarray(T0, np.float32)).cuda()
        info = E.epr_solve_nonlocal(plan.handle, Dd, T, n_iter=n_iter, omega=omega,
                                    eps_I=eps_I, init=0 if T0 is None else 1)
        return T.cpu().numpy().astype(np.float64), info


def _dark_block(ny, nx, seed=21):
    g = np.random.default_rng(seed)
    D = 1.0 + 0.02 * g.normal(size=(ny, nx))
    D[ny // 5:ny - ny // 5, nx // 5:nx - nx // 5] = 0.0
    return D.astype(np.float32)


@pytest.mark.parametrize("n_lines", [1, 2])
@pytest.mark.parametrize("ny,nx", [(64, 72), (256, 256)])
def test_update_floor_branch(torch, oracle, n_lines, ny, nx):
    from paper_2601_22793_gb300 import epr as E
    p, L, eps_I = 1.0e-6, 5e-4, 1e-3
    Es, d, b, w = [55.0, 95.0], [2.4e-7, 8.0e-8], [2.0e-10, 2.6e-11], [0.35, 0.65]
    Es, d, b, w = Es[:n_lines], d[:n_lines], b[:n_lines], w[:n_lines]
    D = _dark_block(ny, nx)
    ln = oracle.Lines(Es, d, b, w, L=L, pixel=p)
    Tr, _ = oracle.solve(ln, D.astype(np.float64), n_iter=1, omega=1.0, eps_I=eps_I)
    Tg, info = _gpu_solve(torch, E, nx, ny, p, L, Es, d, b, w, D, 1, 1.0, eps_I=eps_I)
    assert rel(Tg, Tr) < 1e-4
    # the floor is active on a good share of the block
    _, mu, *_ = ln.params()
    if n_lines == 1:
        floored = np.isclose(Tr, -np.log(eps_I) / mu[0], rtol=1e-12, atol=0)
        assert floored.sum() > 0.1 * (0.6 * ny) * (0.6 * nx)
        assert np.allclose(Tg[floored], Tr[floored], rtol=1e-6)


def test_solve_from_the_callers_thickness(torch, oracle):
    """init = 1: the solve starts from the caller's T (here half the true
    thickness), 8 iterations, mono and two lines."""
    from paper_2601_22793_gb300 import epr as E
    wl, tau = ph.spheres_mono_256()
    ln = oracle.Lines(wl.energy_keV, wl.delta, wl.beta, wl.weights, wl.L, wl.pixel)
    D = ph.poisson(oracle.forward(ln, tau), wl.photons, 3).astype(np.float32)
    T0 = (0.5 * tau).astype(np.float32)
    Tr, ir = oracle.solve(ln, D.astype(np.float64), T0=T0.astype(np.float64), n_iter=8,
                          omega=wl.omega)
    Tg, ig = _gpu_solve(torch, E, wl.nx, wl.ny, wl.pixel, wl.L, wl.energy_keV, wl.delta,
                        wl.beta, wl.weights, D, 8, wl.omega, T0=T0)
    assert rel(Tg, Tr) < 1e-4
    assert np.allclose(ig["rho_hist"][0], ir["rho"], rtol=1e-3)
    # two lines, fixed-point splat
    Es, d, b, w = ph.spectrum(2, 60.0, 100.0, 80.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, 4)
    l2 = oracle.Lines(Es, d, b, w, L=wl.L, pixel=wl.pixel)
    D2 = ph.poisson(oracle.forward(l2, tau), wl.photons, 4).astype(np.float32)
    Tr2, _ = oracle.solve(l2, D2.astype(np.float64), T0=T0.astype(np.float64), n_iter=8,
                          omega=wl.omega)
    Tg2, _ = _gpu_solve(torch, E, wl.nx, wl.ny, wl.pixel, wl.L, Es, d, b, w, D2, 8, wl.omega,
                        T0=T0, deterministic=True)
    assert rel(Tg2, Tr2) < 1e-4


def test_split_without_transport_scales_every_line(torch, oracle):
    from paper_2601_22793_gb300 import epr as E
    p = 1.0e-6
    Es, d, b, w = [50.0, 80.0, 140.0], [3e-7, 1.2e-7, 4e-8], [4e-10, 1e-10, 1.5e-11], [0.2, 0.5, 0.3]
    ln = oracle.Lines(Es, d, b, w, L=0.0, pixel=p)
    f, mu, *_ = ln.params()
    g = np.random.default_rng(31)
    ny, nx = 48, 64
    tau = (1e-3 * (1.0 + g.random((ny, nx)))).astype(np.float32)
    I = f[:, None, None] * np.exp(-mu[:, None, None] * tau.astype(np.float64)[None])
    D = (I.sum(0) * np.exp(g.normal(scale=1.5, size=(ny, nx)))).astype(np.float32)
    Tr, _ = oracle.solve(ln, D.astype(np.float64), T0=tau.astype(np.float64), n_iter=1,
                         omega=1.0)
    Tg, _ = _gpu_solve(torch, E, nx, ny, p, 0.0, Es, d, b, w, D, 1, 1.0, T0=tau)
    assert rel(Tg, Tr) < 1e-5


def test_full_overflow_list_is_reported(torch, oracle):
    """Long-shift sources beyond the overflow list's capacity are reported:
    EPR_ERR_SHIFT_OVERFLOW from a solve with info, and from
    epr_check_device_status after a forward, which is then cleared; with room
    in the list the same forward matches the oracle."""
    from paper_2601_22793_gb300 import epr as E
    wl, tau = ph.ellipsoids_mono(n=256, n_ell=20, seed=41, semi=(6.0, 40.0))
    tau = (4.0 * tau).astype(np.float32)          # shifts of many pixels at the edges
    ln = oracle.Lines(wl.energy_keV, wl.delta, wl.beta, wl.weights, wl.L, wl.pixel)
    gy, gx = oracle.gradient(tau.astype(np.float64))
    c = ln.params()[3][0]
    n_far = int(np.sum((np.abs(c * gx) > 2) | (np.abs(c * gy) > 2)))
    assert n_far > 64
    args = (wl.nx, wl.ny, wl.pixel, wl.L, wl.energy_keV, wl.delta, wl.beta, wl.weights)
    Tt = torch.from_numpy(tau).cuda()
    P = torch.empty_like(Tt)
    with E.Plan(*args, max_shift_px=2, overflow_capacity=16) as p:
        E.epr_forward(p.handle, Tt, P)
        with pytest.raises(E.EprError) as e:
            E.epr_check_device_status(p.handle)
        assert e.value.status == E.EPR_ERR_SHIFT_OVERFLOW
        E.epr_check_device_status(p.handle)          # cleared
        D = torch.ones_like(Tt)
        T = tau.copy()
        Td = torch.from_numpy(T).cuda()
        with pytest.raises(E.EprError) as e:
            E.epr_solve_nonlocal(p.handle, D, Td, n_iter=1, omega=0.4, init=1)
        assert e.value.status == E.EPR_ERR_SHIFT_OVERFLOW
    with E.Plan(*args, max_shift_px=2, overflow_capacity=wl.nx * wl.ny) as p:
        E.epr_forward(p.handle, Tt, P)
        E.epr_check_device_status(p.handle)
        assert rel(P.cpu().numpy(), oracle.forward(ln, tau.astype(np.float64))) < 1e-5


@pytest.mark.parametrize("deterministic", [False, True])
def test_split_where_the_model_vanishes(torch, oracle, deterministic):
    """The residual split where P <= 1e-30 takes r f_s (the second branch of
    the split): a block of the starting thickness is so thick (mu T = 75 for
    the less absorbed of two lines at 80 and 82 keV, 81 for the other, so
    exp(mu T) stays finite in float32) that no line reaches the detector
    there; one iteration from that thickness, float and fixed-point splat.
    Tolerance 1e-4: the update cancels T = 0.9 against ln(1 + q) / mu."""
    from paper_2601_22793_gb300 import epr as E
    p, L = 20e-6, 30.0
    Es = [80.0, 82.0]
    d = [ph.BONE[0] * (80.0 / e) ** 2 for e in Es]
    b = [ph.BONE[1] * (80.0 / e) ** 4 for e in Es]
    w = [0.45, 0.55]
    ln = oracle.Lines(Es, d, b, w, L=L, pixel=p)
    _, mu, *_ = ln.params()
    ny, nx = 128, 192
    ells = ph.random_ellipsoids(ny, nx, 12, 4.0, 20.0, seed=61)
    T0 = ph.project_ellipsoids(ells, ny, nx, p)
    T0[40:80, 50:110] = 75.0 / float(np.min(mu))
    Pr = oracle.forward(ln, T0)
    assert np.all(Pr[45:75, 55:105] <= 1e-30)
    D = (1.0 + 0.02 * np.random.default_rng(62).normal(size=(ny, nx))).astype(np.float32)
    Tr, _ = oracle.solve(ln, D.astype(np.float64), T0=T0, n_iter=1, omega=0.4)
    Tg, _ = _gpu_solve(torch, E, nx, ny, p, L, Es, d, b, w, D, 1, 0.4,
                       T0=T0.astype(np.float32), deterministic=deterministic)
    assert np.all(np.isfinite(Tg))
    assert rel(Tg, Tr) < 1e-4
    blk = (slice(40, 80), slice(50, 110))
    assert rel(Tg[blk], Tr[blk]) < 1e-4
