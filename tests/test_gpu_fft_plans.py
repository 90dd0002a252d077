"""The radix-16 plan of the 2048-row column transforms (stages 16, 16, 8
instead of 8, 8, 8, 4) and the autotuner's column-pass choice, against the
FP64 oracle through the C ABI: the preconditioner at <= 1e-5 relative L2 and
solves at <= 1e-4, like the default plan."""
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


@pytest.mark.parametrize("n_lines", [1, 3])
def test_radix16_preconditioner_vs_oracle(torch, oracle, n_lines):
    from paper_2601_22793_gb300 import epr as E
    ny, nx, p, L = 2048, 256, 20e-6, 30.0
    Es, d, b, w = ph.spectrum(n_lines, 60.0, 140.0, 90.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, 3)
    ln = oracle.Lines(Es, d, b, w, L=L, pixel=p)
    g0 = np.random.default_rng(8).normal(size=(2, ny, nx)).astype(np.float32)
    with E.Plan(nx, ny, p, L, Es, d, b, w, fft_radix=16) as plan:
        for s in range(n_lines):
            g = torch.from_numpy(g0).cuda()
            E.epr_precondition(plan.handle, g, line=s, batch=2)
            torch.cuda.synchronize()
            out = g.cpu().numpy()
            for bb in range(2):
                assert rel(out[bb], oracle.precondition(ln, g0[bb].astype(np.float64), line=s)) < 1e-5


@pytest.mark.parametrize("n_lines,radix,col_blocks", [(1, 16, 4), (2, 16, 4), (1, 8, 4),
                                                     (1, 16, 5), (2, 16, 5)])
def test_solve_with_radix_plan_vs_oracle(torch, oracle, n_lines, radix, col_blocks):
    """col_blocks = 5: the radix-16 column pass bounded to five blocks per SM
    (set through epr_plan_set_tuning)."""
    from paper_2601_22793_gb300 import epr as E
    ny, nx = 2048, 512
    Es, d, b, w = ph.spectrum(n_lines, 60.0, 140.0, 90.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, 5)
    wl = ph.Workload("crop", ny, nx, 20e-6, 30.0, Es, d, b, w, 5, 0.4, 1e4)
    ells = ph.random_ellipsoids(ny, nx, 30, 6.0, 60.0, seed=21)
    tau = ph.project_ellipsoids(ells, ny, nx, wl.pixel)
    ln = oracle.Lines(Es, d, b, w, L=wl.L, pixel=wl.pixel)
    D = ph.poisson(oracle.forward(ln, tau), 1e4, 22).astype(np.float32)
    Tr, ir = oracle.solve(ln, D.astype(np.float64), n_iter=5, omega=0.4)
    with E.Plan(nx, ny, wl.pixel, wl.L, Es, d, b, w, fft_radix=radix) as plan:
        assert E.epr_plan_get_tuning(plan.handle)["col_radix"] == radix
        if col_blocks != 4:
            tun = dict(E.epr_plan_get_tuning(plan.handle), col_radix=radix,
                       col_blocks_per_sm=col_blocks)
            E.epr_plan_set_tuning(plan.handle, tun)
            assert E.epr_plan_get_tuning(plan.handle)["col_blocks_per_sm"] == col_blocks
        Dd = torch.from_numpy(D).cuda()
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(plan.handle, Dd, T, n_iter=5, omega=0.4)
        Tg = T.cpu().numpy()
    assert rel(Tg, Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], ir["rho"], rtol=1e-3)


@pytest.mark.parametrize("tile,reach", [((32, 64), 3), ((64, 32), 4), ((32, 32), 3)])
def test_occupancy_variants_vs_oracle(torch, oracle, tile, reach):
    """The six-blocks-per-SM residual splat, the five-blocks-per-SM radix-16
    column pass and the six-blocks-per-SM row passes, set through
    epr_plan_set_tuning, on a one-line 512 x 2048 solve (5 iterations)."""
    from paper_2601_22793_gb300 import epr as E
    ny, nx = 2048, 512
    wl = ph.Workload("crop", ny, nx, 20e-6, 30.0, [80.0], [ph.BONE[0]], [ph.BONE[1]], [1.0], 5,
                     0.4, 1e4)
    ells = ph.random_ellipsoids(ny, nx, 30, 6.0, 60.0, seed=23)
    tau = ph.project_ellipsoids(ells, ny, nx, wl.pixel)
    ln = oracle.Lines(wl.energy_keV, wl.delta, wl.beta, wl.weights, L=wl.L, pixel=wl.pixel)
    D = ph.poisson(oracle.forward(ln, tau), 1e4, 24).astype(np.float32)
    Tr, ir = oracle.solve(ln, D.astype(np.float64), n_iter=5, omega=0.4)
    with E.Plan(nx, ny, wl.pixel, wl.L, wl.energy_keV, wl.delta, wl.beta, wl.weights) as plan:
        tun = dict(E.epr_plan_get_tuning(plan.handle), splat_tile=list(tile), splat_reach=reach,
                   splat_blocks_per_sm=6, col_tile_width=0, col_radix=16, col_blocks_per_sm=5,
                   row_blocks_per_sm=6)
        E.epr_plan_set_tuning(plan.handle, tun)
        got = E.epr_plan_get_tuning(plan.handle)
        assert got == dict(tun, tuned=True)
        Dd = torch.from_numpy(D).cuda()
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(plan.handle, Dd, T, n_iter=5, omega=0.4)
        Tg = T.cpu().numpy()
        with pytest.raises(E.EprError):   # no six-block variant of the 64 x 64 tile
            E.epr_plan_set_tuning(plan.handle, dict(tun, splat_tile=[64, 64]))
    assert rel(Tg, Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], ir["rho"], rtol=1e-3)


def test_autotuned_plan_solves_like_the_default(torch, oracle):
    """The tuner times splat tiles, reach, the column pass's radix plan and
    tile width on the first solve; later solves use its choice and agree with
    the untuned plan and the oracle."""
    from paper_2601_22793_gb300 import epr as E
    wl, tau = ph.ellipsoids_mono(n=1024, n_ell=60, seed=31, n_iter=6)
    ln = oracle.Lines(wl.energy_keV, wl.delta, wl.beta, wl.weights, wl.L, wl.pixel)
    D = ph.poisson(oracle.forward(ln, tau), 1e4, 32).astype(np.float32)
    Tr, _ = oracle.solve(ln, D.astype(np.float64), n_iter=6, omega=0.4)
    outs = {}
    for tune in (False, True):
        with E.Plan(wl.nx, wl.ny, wl.pixel, wl.L, wl.energy_keV, wl.delta, wl.beta, wl.weights,
                    autotune=tune) as plan:
            Dd = torch.from_numpy(D).cuda()
            for _ in range(2):   # the first solve of the tuned plan runs the tuner
                T = torch.empty_like(Dd)
                E.epr_solve_nonlocal(plan.handle, Dd, T, n_iter=6, omega=0.4)
            outs[tune] = T.cpu().numpy()
    assert rel(outs[True], outs[False]) < 1e-5
    assert rel(outs[True], Tr) < 1e-4


def test_autotuned_polychromatic_plan_vs_oracle(torch, oracle):
    """A three-line plan with the tuner on (splat tiles, reach and the column
    plans, timed on the split residuals of its first solve): its later solves
    match the oracle."""
    from paper_2601_22793_gb300 import epr as E
    ny, nx = 2048, 512
    Es, d, b, w = ph.spectrum(3, 60.0, 140.0, 90.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, 7)
    ells = ph.random_ellipsoids(ny, nx, 30, 6.0, 60.0, seed=25)
    tau = ph.project_ellipsoids(ells, ny, nx, 20e-6)
    ln = oracle.Lines(Es, d, b, w, L=30.0, pixel=20e-6)
    D = ph.poisson(oracle.forward(ln, tau), 1e4, 26).astype(np.float32)
    Tr, ir = oracle.solve(ln, D.astype(np.float64), n_iter=5, omega=0.4)
    with E.Plan(nx, ny, 20e-6, 30.0, Es, d, b, w, autotune=True) as plan:
        Dd = torch.from_numpy(D).cuda()
        for _ in range(2):   # the first solve runs the tuner
            T = torch.empty_like(Dd)
            info = E.epr_solve_nonlocal(plan.handle, Dd, T, n_iter=5, omega=0.4)
        assert E.epr_plan_get_tuning(plan.handle)["tuned"]
        Tg = T.cpu().numpy()
    assert rel(Tg, Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], ir["rho"], rtol=1e-3)


def test_tuning_carries_over_between_plans(torch, oracle):
    """epr_plan_get_tuning / epr_plan_set_tuning: a second plan given the
    first plan's tuned choices solves as the tuned plan does; invalid choices
    are refused."""
    from paper_2601_22793_gb300 import epr as E
    wl, tau = ph.ellipsoids_mono(n=1024, n_ell=60, seed=33, n_iter=4)
    ln = oracle.Lines(wl.energy_keV, wl.delta, wl.beta, wl.weights, wl.L, wl.pixel)
    D = ph.poisson(oracle.forward(ln, tau), 1e4, 34).astype(np.float32)
    args = (wl.nx, wl.ny, wl.pixel, wl.L, wl.energy_keV, wl.delta, wl.beta, wl.weights)
    Dd = torch.from_numpy(D).cuda()
    with E.Plan(*args, autotune=True) as a, E.Plan(*args) as b:
        T = torch.empty_like(Dd)
        E.epr_solve_nonlocal(a.handle, Dd, T, n_iter=4, omega=0.4)   # tunes
        tun = E.epr_plan_get_tuning(a.handle)
        assert tun["tuned"]
        E.epr_solve_nonlocal(a.handle, Dd, T, n_iter=4, omega=0.4)
        Ta = T.cpu().numpy()
        assert not E.epr_plan_get_tuning(b.handle)["tuned"]
        E.epr_plan_set_tuning(b.handle, tun)
        assert E.epr_plan_get_tuning(b.handle) == tun
        T2 = torch.empty_like(Dd)
        E.epr_solve_nonlocal(b.handle, Dd, T2, n_iter=4, omega=0.4)
        assert rel(T2.cpu().numpy(), Ta) < 1e-6
        for bad in (dict(tun, col_radix=12), dict(tun, col_radix=8, col_blocks_per_sm=5),
                    dict(tun, col_blocks_per_sm=6)):
            with pytest.raises(E.EprError):
                E.epr_plan_set_tuning(b.handle, bad)
