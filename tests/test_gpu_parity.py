"""GPU parity: the CUDA path, called through the C ABI (libepr.so), against
the FP64 oracle on the same seeded float32 inputs.

Tolerances (relative L2): 1e-5 per forward / adjoint / preconditioner
application, 1e-4 on the solved thickness; bit-exact across runs in the
fixed-point splat mode.  Sizes span several tiles and ragged tails; the
full-size 2048 x 2048 case runs in the launch configuration of bench.py."""
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


@pytest.fixture(scope="module")
def E():
    from paper_2601_22793_gb300 import epr
    return epr


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def lines_of(oracle, wl):
    return oracle.Lines(wl.energy_keV, wl.delta, wl.beta, wl.weights, wl.L, wl.pixel)


def plan_of(E, wl, **kw):
    return E.Plan(wl.nx, wl.ny, wl.pixel, wl.L, wl.energy_keV, wl.delta, wl.beta, wl.weights, **kw)


def small_poly(ny=144, nx=96, n_lines=4, seed=5):
    """Polychromatic ellipsoid phantom on a ragged grid (nx not a multiple of
    the 64-pixel splat tile)."""
    Es, d, b, w = ph.spectrum(n_lines, 60.0, 160.0, 95.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, seed)
    wl = ph.Workload("poly_small", ny, nx, 20e-6, 30.0, Es, d, b, w, 10, 0.4, 1e4)
    ells = ph.random_ellipsoids(ny, nx, 10, 4.0, 20.0, margin=8.0, seed=seed)
    tau = ph.project_ellipsoids(ells, ny, nx, wl.pixel)
    return wl, tau.astype(np.float32)


# --------------------------------------------------------------------------
# forward transport
# --------------------------------------------------------------------------

def test_forward_spheres_mono(torch, E, oracle):
    wl, tau = ph.spheres_mono_256()
    T32 = tau.astype(np.float32)
    with plan_of(E, wl) as p:
        T = cuda(torch, T32)
        P = torch.empty_like(T)
        E.epr_forward(p.handle, T, P)
        torch.cuda.synchronize()
    ref = oracle.forward(lines_of(oracle, wl), T32.astype(np.float64))
    assert rel(host(P), ref) < 1e-5


def test_forward_poly_per_line_ragged(torch, E, oracle):
    wl, T32 = small_poly()
    with plan_of(E, wl) as p:
        T = cuda(torch, T32)
        P = torch.empty_like(T)
        Ps = torch.empty((wl.energy_keV.size, wl.ny, wl.nx), device="cuda")
        E.epr_forward(p.handle, T, P, Ps)
        torch.cuda.synchronize()
    Pr, Psr, dropped = oracle.forward(lines_of(oracle, wl), T32.astype(np.float64), per_line=True)
    assert rel(host(P), Pr) < 1e-5
    for s in range(wl.energy_keV.size):
        assert rel(host(Ps[s]), Psr[s]) < 1e-5


def test_forward_overflow_path_keeps_all_mass(torch, E, oracle):
    """With a 1-pixel fast-path reach most large shifts take the overflow
    list; the prediction must still equal the oracle's."""
    wl, T32 = small_poly(n_lines=2, seed=6)
    gy, gx = np.gradient(T32.astype(np.float64))
    umax = (np.abs(wl.L * wl.delta.max() / wl.pixel ** 2) * np.hypot(gy, gx)).max()
    assert umax > 2.0
    with plan_of(E, wl, max_shift_px=1) as p:
        T = cuda(torch, T32)
        P = torch.empty_like(T)
        E.epr_forward(p.handle, T, P)
        E.epr_check_device_status(p.handle)
    ref = oracle.forward(lines_of(oracle, wl), T32.astype(np.float64))
    assert rel(host(P), ref) < 1e-5


def test_forward_negative_thickness_keeps_the_accumulators_in_range(torch, E, oracle):
    """Where f_s exp(-mu_s T) exceeds 2 f_s (T < -ln 2 / mu_s) a source would
    not fit the float mode's 32-bit tile accumulators; such sources take the
    overflow path, so the prediction still equals the oracle's."""
    wl, tau = ph.spheres_mono_256()
    ln = lines_of(oracle, wl)
    f, mu, *_ = ln.params()
    yy, xx = np.mgrid[0:wl.ny, 0:wl.nx].astype(np.float64)
    bump = 1.5 * np.log(2.0) / mu[0] * np.exp(-((yy - 90.0) ** 2 + (xx - 170.0) ** 2) / 20.0 ** 2)
    T32 = (tau - bump).astype(np.float32)
    assert (T32 < -np.log(2.0) / mu[0]).sum() > 300   # ~500 heavy sources
    with plan_of(E, wl) as p:
        T = cuda(torch, T32)
        P = torch.empty_like(T)
        E.epr_forward(p.handle, T, P)
        E.epr_check_device_status(p.handle)
    ref = oracle.forward(ln, T32.astype(np.float64))
    assert rel(host(P), ref) < 1e-5


def test_forward_fixed_point_is_bit_exact(torch, E, oracle):
    wl, T32 = small_poly(seed=7)
    outs = []
    with plan_of(E, wl, deterministic=True) as p:
        T = cuda(torch, T32)
        for _ in range(3):
            P = torch.empty_like(T)
            E.epr_forward(p.handle, T, P)
            torch.cuda.synchronize()
            outs.append(P.cpu().numpy().copy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    ref = oracle.forward(lines_of(oracle, wl), T32.astype(np.float64))
    assert rel(outs[0], ref) < 1e-5


def test_forward_zero_thickness_is_flat_field(torch, E):
    wl, _ = ph.spheres_mono_256()
    with plan_of(E, wl) as p:
        T = torch.zeros((wl.ny, wl.nx), device="cuda")
        P = torch.empty_like(T)
        E.epr_forward(p.handle, T, P)
        torch.cuda.synchronize()
    assert torch.equal(P, torch.ones_like(P))


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

def test_adjoint_vs_oracle_and_dot_product(torch, E, oracle):
    wl, T32 = small_poly(seed=8)
    ln = lines_of(oracle, wl)
    f, mu, *_ = ln.params()
    g = np.random.default_rng(3)
    r = g.normal(size=T32.shape).astype(np.float32)
    with plan_of(E, wl) as p:
        T = cuda(torch, T32)
        P = torch.empty_like(T)
        Ps = torch.empty((wl.energy_keV.size, wl.ny, wl.nx), device="cuda")
        E.epr_forward(p.handle, T, P, Ps)
        for s in range(wl.energy_keV.size):
            out = torch.empty_like(T)
            E.epr_adjoint(p.handle, T, cuda(torch, r), out, line=s)
            torch.cuda.synchronize()
            ref = oracle.adjoint(ln, T32.astype(np.float64), r.astype(np.float64), line=s)
            assert rel(host(out), ref) < 1e-5
            # <M_s I_s, r> = <I_s, M_s^T r> with the GPU pair
            Is = f[s] * np.exp(-mu[s] * T32.astype(np.float64))
            lhs = np.sum(host(Ps[s]) * r)
            rhs = np.sum(Is * host(out))
            assert abs(lhs - rhs) < 2e-6 * np.sum(np.abs(Is * host(out)))


# --------------------------------------------------------------------------
# preconditioner
# --------------------------------------------------------------------------

@pytest.mark.parametrize("ny,nx", [(16, 16), (48, 96), (256, 256), (384, 96), (96, 1536)])
def test_precondition_vs_oracle(torch, E, oracle, ny, nx):
    Es, d, b, w = ph.spectrum(3, 60.0, 160.0, 95.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, 1)
    wl = ph.Workload("pc", ny, nx, 20e-6, 30.0, Es, d, b, w, 1, 1.0, 1e4)
    g0 = np.random.default_rng(ny * nx).normal(size=(2, ny, nx)).astype(np.float32)
    ln = lines_of(oracle, wl)
    with plan_of(E, wl) as p:
        for s in range(3):
            gt = cuda(torch, g0)
            E.epr_precondition(p.handle, gt, line=s, batch=2)
            torch.cuda.synchronize()
            for bb in range(2):
                ref = oracle.precondition(ln, g0[bb].astype(np.float64), line=s)
                assert rel(host(gt[bb]), ref) < 1e-5


# --------------------------------------------------------------------------
# solvers
# --------------------------------------------------------------------------

def _spheres_data(oracle):
    wl, tau = ph.spheres_mono_256()
    ln = lines_of(oracle, wl)
    D = ph.poisson(oracle.forward(ln, tau), wl.photons, 1).astype(np.float32)
    return wl, ln, D


@pytest.mark.parametrize("det", [False, True])
def test_solve_nonlocal_spheres_mono(torch, E, oracle, det):
    wl, ln, D = _spheres_data(oracle)
    Tr, info_r = oracle.solve(ln, D.astype(np.float64), n_iter=wl.n_iter, omega=wl.omega)
    with plan_of(E, wl, deterministic=det) as p:
        Dd = cuda(torch, D)
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=wl.n_iter, omega=wl.omega)
    assert rel(host(T), Tr) < 1e-4
    assert info["iters"][0] == wl.n_iter
    assert np.allclose(info["rho_hist"][0], info_r["rho"], rtol=1e-3)
    assert np.allclose(info["kappa_hist"][0][1:], info_r["kappa"][1:], rtol=1e-2)


def test_solve_nonlocal_poly(torch, E, oracle):
    wl, T32 = small_poly(seed=9)
    ln = lines_of(oracle, wl)
    D = ph.poisson(oracle.forward(ln, T32.astype(np.float64)), wl.photons, 2).astype(np.float32)
    Tr, info_r = oracle.solve(ln, D.astype(np.float64), n_iter=wl.n_iter, omega=wl.omega)
    with plan_of(E, wl) as p:
        Dd = cuda(torch, D)
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=wl.n_iter, omega=wl.omega)
    assert rel(host(T), Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], info_r["rho"], rtol=1e-3)


@pytest.mark.parametrize("ny,nx", [(256, 256), (256, 512)])
@pytest.mark.parametrize("det", [False, True])
def test_solve_poly_compile_time_row_kernels(torch, E, oracle, ny, nx, det):
    """Row lengths with compile-time row kernels (the line-per-block gather and
    the line-looping inverse) against the oracle, float and fixed point."""
    wl, T32 = small_poly(ny=ny, nx=nx, n_lines=4, seed=12)
    ln = lines_of(oracle, wl)
    D = ph.poisson(oracle.forward(ln, T32.astype(np.float64)), wl.photons, 6).astype(np.float32)
    Tr, info_r = oracle.solve(ln, D.astype(np.float64), n_iter=6, omega=0.4)
    with plan_of(E, wl, deterministic=det) as p:
        Dd = cuda(torch, D)
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=6, omega=0.4)
    assert rel(host(T), Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], info_r["rho"], rtol=1e-3)
    assert np.allclose(info["kappa_hist"][0][1:], info_r["kappa"][1:], rtol=1e-2)


@pytest.mark.parametrize("ny,nx,n_lines", [(96, 1536, 1), (1536, 96, 1), (64, 3072, 2),
                                           (3072, 64, 2), (32, 4096, 1), (32, 4096, 2),
                                           (4096, 32, 1), (4096, 48, 2)])
def test_solve_three_smooth_sizes(torch, E, oracle, ny, nx, n_lines):
    """Row and column lengths 3 * 2^k on the compile-time kernels (radix-3
    stages; the 1536-row column pass moves its tile by TMA), and the largest
    detector side, 4096: the compile-time 4096-point row kernels and the
    bulk-copy column pass of two 4096-point columns."""
    wl, T32 = small_poly(ny=ny, nx=nx, n_lines=n_lines, seed=13)
    ln = lines_of(oracle, wl)
    D = ph.poisson(oracle.forward(ln, T32.astype(np.float64)), wl.photons, 7).astype(np.float32)
    Tr, info_r = oracle.solve(ln, D.astype(np.float64), n_iter=4, omega=0.4)
    with plan_of(E, wl) as p:
        Dd = cuda(torch, D)
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=4, omega=0.4)
    assert rel(host(T), Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], info_r["rho"], rtol=1e-3)


def test_solve_fixed_point_bit_exact_and_graph_replay(torch, E, oracle):
    wl, T32 = small_poly(seed=10)
    ln = lines_of(oracle, wl)
    D = ph.poisson(oracle.forward(ln, T32.astype(np.float64)), wl.photons, 3).astype(np.float32)
    res = []
    with plan_of(E, wl, deterministic=True) as p:
        Dd = cuda(torch, D)
        T = torch.empty_like(Dd)
        for _ in range(3):   # the 2nd and 3rd calls replay the cached graph
            E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=6, omega=0.4)
            res.append(T.cpu().numpy().copy())
    assert all(np.array_equal(res[0], r) for r in res[1:])
    Tr, _ = oracle.solve(ln, D.astype(np.float64), n_iter=6, omega=0.4)
    assert rel(res[0], Tr) < 1e-4


def test_programmatic_launch_matches_serial_launches(torch, E, oracle):
    """Programmatic dependent launch changes only when kernels start.  In the
    fixed-point mode every solve (graph replay or stream launches, with one
    projection retiring after its first iteration) is bit-identical to the
    serial launches; the monochromatic float solve agrees to float atomics
    ordering."""
    wl, T32 = small_poly(seed=11)
    ln = lines_of(oracle, wl)
    D = np.stack([
        ph.poisson(oracle.forward(ln, T32.astype(np.float64)), wl.photons, 4),
        ph.poisson(oracle.forward(ln, 0.3 * T32.astype(np.float64)), wl.photons, 5),
        oracle.forward(ln, np.zeros_like(T32, dtype=np.float64)),   # retires at once
    ]).astype(np.float32)
    out = {}
    for serial in (False, True):
        for graphs in (False, True):
            with plan_of(E, wl, deterministic=True, serial_launches=serial, use_graphs=graphs) as p:
                Dd = cuda(torch, D)
                T = torch.empty_like(Dd)
                info = E.epr_solve_nonlocal(p.handle, Dd, T, batch=3, n_iter=8, omega=0.4,
                                            tol=1e-3)
                out[(serial, graphs)] = (T.cpu().numpy().copy(), tuple(info["iters"]))
    ref = out[(True, False)]
    assert ref[1][2] == 1 and ref[1][0] > 1
    for key, (T_k, it_k) in out.items():
        assert it_k == ref[1], key
        assert np.array_equal(T_k, ref[0]), key

    wl, ln, Dm = _spheres_data(oracle)
    res = []
    for serial in (False, True):
        with plan_of(E, wl, serial_launches=serial) as p:
            Dd = cuda(torch, Dm)
            T = torch.empty_like(Dd)
            E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=wl.n_iter, omega=wl.omega)
            res.append(host(T))
    assert rel(res[0], res[1]) < 1e-5


def test_solve_tolerance_stops_like_the_oracle(torch, E, oracle):
    wl, ln, D = _spheres_data(oracle)
    tol = 0.01
    Tr, info_r = oracle.solve(ln, D.astype(np.float64), n_iter=20, omega=1.0, tol=tol)
    with plan_of(E, wl) as p:
        Dd = cuda(torch, D)
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=20, omega=1.0, tol=tol)
    assert info["iters"][0] == info_r["iters"] < 20
    assert rel(host(T), Tr) < 1e-4


def test_single_iteration_reports_rho_and_kappa(torch, E, oracle):
    """One iteration: rho comes from the column pass and kappa from the kernel
    after the loop (no later forward pass forms it); from T = 0, kappa = 1."""
    wl, ln, D = _spheres_data(oracle)
    Tr, info_r = oracle.solve(ln, D.astype(np.float64), n_iter=1, omega=wl.omega)
    with plan_of(E, wl) as p:
        T = torch.empty(D.shape, device="cuda")
        info = E.epr_solve_nonlocal(p.handle, cuda(torch, D), T, n_iter=1, omega=wl.omega)
    assert info["iters"][0] == 1
    assert rel(host(T), Tr) < 1e-4
    assert np.isclose(info["rho"][0], info_r["rho"][0], rtol=1e-4)
    assert np.isclose(info["kappa"][0], 1.0, rtol=1e-6) and np.isclose(info_r["kappa"][0], 1.0)


def test_convergence_on_the_last_iteration(torch, E, oracle):
    """A solve whose tolerance is met exactly at its last allowed iteration: the
    kernel after the loop forms that kappa and the iteration count."""
    wl, ln, D = _spheres_data(oracle)
    tol = 0.01
    _, info_r = oracle.solve(ln, D.astype(np.float64), n_iter=20, omega=1.0, tol=tol)
    k = info_r["iters"]
    assert 2 <= k < 20
    Tr, _ = oracle.solve(ln, D.astype(np.float64), n_iter=k, omega=1.0, tol=tol)
    with plan_of(E, wl) as p:
        T = torch.empty(D.shape, device="cuda")
        info = E.epr_solve_nonlocal(p.handle, cuda(torch, D), T, n_iter=k, omega=1.0, tol=tol)
    assert info["iters"][0] == k
    assert info["kappa"][0] <= tol
    assert np.isclose(info["kappa"][0], info_r["kappa"][k - 1], rtol=1e-2)
    assert rel(host(T), Tr) < 1e-4


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_data_is_reported(torch, E, oracle, bad):
    """A NaN or an infinity in D is reported as EPR_ERR_NONFINITE: by the solve
    when it fills info, else by the device status check, which then clears."""
    wl, ln, D = _spheres_data(oracle)
    Dbad = D.copy()
    Dbad[100, 37] = bad
    with plan_of(E, wl) as p:
        T = torch.empty(D.shape, device="cuda")
        with pytest.raises(E.EprError) as ex:
            E.epr_solve_nonlocal(p.handle, cuda(torch, Dbad), T, n_iter=3, omega=wl.omega)
        assert ex.value.status == 5
        with pytest.raises(E.EprError) as ex:        # the word still holds it: read and clear
            E.epr_check_device_status(p.handle)
        assert ex.value.status == 5
        E.epr_check_device_status(p.handle)          # cleared
        E.epr_solve_nonlocal(p.handle, cuda(torch, Dbad), T, n_iter=3, omega=wl.omega,
                             want_info=False)
        with pytest.raises(E.EprError) as ex:
            E.epr_check_device_status(p.handle)
        assert ex.value.status == 5
        info = E.epr_solve_nonlocal(p.handle, cuda(torch, D), T, n_iter=3, omega=wl.omega)
        assert info["iters"][0] == 3 and np.isfinite(host(T)).all()


def test_batch_equals_single_projections(torch, E, oracle):
    wl, T32 = small_poly(seed=11)
    ln = lines_of(oracle, wl)
    Ds = []
    for k in range(3):
        _, tk = small_poly(seed=20 + k)
        Ds.append(ph.poisson(oracle.forward(ln, tk.astype(np.float64)), 1e4, k).astype(np.float32))
    Db = np.stack(Ds)
    with plan_of(E, wl, deterministic=True) as p:
        Tb = torch.empty((3, wl.ny, wl.nx), device="cuda")
        info = E.epr_solve_nonlocal(p.handle, cuda(torch, Db), Tb, batch=3, n_iter=5, omega=0.4)
        outs = []
        for k in range(3):
            T1 = torch.empty((wl.ny, wl.nx), device="cuda")
            E.epr_solve_nonlocal(p.handle, cuda(torch, Ds[k]), T1, n_iter=5, omega=0.4)
            outs.append(T1.cpu().numpy())
    for k in range(3):
        assert np.array_equal(Tb[k].cpu().numpy(), outs[k])
    assert list(info["iters"]) == [5, 5, 5]


def test_host_buffers_match_device_buffers(torch, E, oracle):
    wl, ln, D = _spheres_data(oracle)
    with plan_of(E, wl, deterministic=True) as p:
        Td = torch.empty((wl.ny, wl.nx), device="cuda")
        E.epr_solve_nonlocal(p.handle, cuda(torch, D), Td, n_iter=4)
        Th = np.zeros((wl.ny, wl.nx), np.float32)
        Dh = torch.from_numpy(D).pin_memory()
        Thp = torch.zeros((wl.ny, wl.nx)).pin_memory()
        E.epr_solve_nonlocal(p.handle, D.copy(), Th, n_iter=4)
        E.epr_solve_nonlocal(p.handle, Dh, Thp, n_iter=4)
    assert np.array_equal(Td.cpu().numpy(), Th)
    assert np.array_equal(Th, Thp.numpy())


# --------------------------------------------------------------------------
# local closure
# --------------------------------------------------------------------------

@pytest.mark.parametrize("model", [1, 2])
def test_local_forward_vs_oracle(torch, E, oracle, model):
    wl, T32 = small_poly(seed=12)
    with plan_of(E, wl) as p:
        T = cuda(torch, T32)
        P = torch.empty_like(T)
        Ps = torch.empty((wl.energy_keV.size, wl.ny, wl.nx), device="cuda")
        E.epr_forward(p.handle, T, P, Ps, model=model)
        torch.cuda.synchronize()
    Pr, Psr, _ = oracle.forward(lines_of(oracle, wl), T32.astype(np.float64), model=model,
                                per_line=True)
    assert rel(host(P), Pr) < 1e-5
    assert rel(host(Ps), Psr) < 1e-5


@pytest.mark.parametrize("order", [1, 2])
def test_local_solve_vs_oracle(torch, E, oracle, order):
    wl, ln, D = _spheres_data(oracle)
    Tr, _ = oracle.solve(ln, D.astype(np.float64), n_iter=8, omega=1.0, model=order)
    with plan_of(E, wl) as p:
        Dd = cuda(torch, D)
        T = torch.empty_like(Dd)
        E.epr_solve_local(p.handle, Dd, T, order=order, n_iter=8, omega=1.0)
    assert rel(host(T), Tr) < 1e-4


# --------------------------------------------------------------------------
# full size, as timed by bench.py
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def full(oracle):
    wl, tau = ph.ellipsoids_mono()
    ln = lines_of(oracle, wl)
    P = oracle.forward(ln, tau)
    D = ph.poisson(P, wl.photons, 7).astype(np.float32)
    return wl, ln, tau.astype(np.float32), D


def test_full_size_forward_and_mass(torch, E, oracle, full):
    wl, ln, T32, D = full
    with plan_of(E, wl) as p:
        T = cuda(torch, T32)
        P = torch.empty_like(T)
        E.epr_forward(p.handle, T, P)
        torch.cuda.synchronize()
    Pg = host(P)
    Pr, _, dropped = oracle.forward(ln, T32.astype(np.float64), per_line=True)
    assert rel(Pg, Pr) < 1e-5
    I = np.exp(-ln.params()[1][0] * T32.astype(np.float64))
    assert abs(Pg.sum() + dropped[0] - I.sum()) < 1e-6 * I.sum()


def test_full_size_solve_iterations(torch, E, oracle, full):
    wl, ln, T32, D = full
    n_it = 3
    Tr, info_r = oracle.solve(ln, D.astype(np.float64), n_iter=n_it, omega=wl.omega)
    with plan_of(E, wl) as p:
        Dd = cuda(torch, D)
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=n_it, omega=wl.omega)
    assert rel(host(T), Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], info_r["rho"], rtol=1e-4)
