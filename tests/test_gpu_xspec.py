"""GPU parity of the x-dependent effective spectrum (the paper's "Remark on
spatially varying spectra"; a knot table of per-line weights, delta and beta
across the detector columns) against the FP64 oracle, through the C ABI:
forward, adjoint and preconditioner at <= 1e-5 relative L2, the solve at
<= 1e-4, float and fixed-point splat, ragged sizes, and the row lengths with
compile-time row kernels that read the per-column constants (1024, 2048,
4096)."""
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


def _case(n_lines, ny, nx, seed):
    """Bone-like lines 60-160 keV, L = 30 m, p = 20 um; across the columns the
    weights vary by +-30 % and delta, beta by +-20 % (a filtered, tilted
    beam), five knots."""
    Es, d, b, w = ph.spectrum(n_lines, 60.0, 160.0, 95.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, seed)
    g = np.random.default_rng(seed)
    X = np.linspace(-3.0, nx + 2.0, 5)
    W = w[:, None] * g.uniform(0.7, 1.3, size=(n_lines, 5))
    Dl = d[:, None] * g.uniform(0.8, 1.2, size=(n_lines, 5))
    Bt = b[:, None] * g.uniform(0.8, 1.2, size=(n_lines, 5))
    ells = ph.random_ellipsoids(ny, nx, 12, 4.0, 24.0, margin=8.0, seed=seed)
    tau = ph.project_ellipsoids(ells, ny, nx, 20e-6).astype(np.float32)
    return (Es, d, b, w), (X, W, Dl, Bt), tau


def _plan(E, phys, tab, ny, nx, **kw):
    Es, d, b, w = phys
    plan = E.Plan(nx, ny, 20e-6, 30.0, Es, d, b, w, **kw)
    E.epr_plan_set_xspec(plan.handle, *tab)
    return plan


@pytest.mark.parametrize("n_lines,ny,nx,det", [(1, 96, 192, False), (3, 144, 96, False),
                                               (3, 144, 96, True)])
def test_xspec_forward_adjoint_precondition(torch, oracle, n_lines, ny, nx, det):
    from paper_2601_22793_gb300 import epr as E
    phys, tab, tau = _case(n_lines, ny, nx, 11 + n_lines)
    xs = oracle.XSpec(phys[0], *tab, 30.0, 20e-6, nx)
    Pr, Psr, _ = oracle.forward_x(xs, tau.astype(np.float64), per_line=True)
    g = np.random.default_rng(3)
    r = g.normal(size=(ny, nx))
    gy, gx = oracle.gradient(tau.astype(np.float64))
    with _plan(E, phys, tab, ny, nx, deterministic=det) as p:
        T = torch.from_numpy(tau).cuda()
        P = torch.empty_like(T)
        Ps = torch.empty((n_lines, ny, nx), device="cuda")
        E.epr_forward(p.handle, T, P, Ps)
        assert rel(P.cpu().numpy(), Pr) < 1e-5
        assert rel(Ps.cpu().numpy(), Psr) < 1e-5
        for s in range(n_lines):
            rg = torch.from_numpy(r.astype(np.float32)).cuda()
            out = torch.empty_like(rg)
            E.epr_adjoint(p.handle, T, rg, out, line=s)
            ref = oracle.gather(r.astype(np.float32).astype(np.float64), xs.c[s][None, :] * gy,
                                xs.c[s][None, :] * gx)
            assert rel(out.cpu().numpy(), ref) < 1e-5, s
            h = rg.clone()
            E.epr_precondition(p.handle, h, line=s)
            ref = oracle.paganin(r.astype(np.float32).astype(np.float64), 20e-6, xs.mu_h[s],
                                 xs.Ld_h[s])
            torch.cuda.synchronize()
            assert rel(h.cpu().numpy(), ref) < 1e-5, s


@pytest.mark.parametrize("n_lines,ny,nx,det", [(2, 128, 192, False), (4, 256, 512, True),
                                               (1, 256, 256, False), (3, 64, 1024, False),
                                               (1, 48, 2048, False), (2, 32, 2048, True),
                                               (2, 32, 4096, False)])
def test_xspec_solve_vs_oracle(torch, oracle, n_lines, ny, nx, det):
    from paper_2601_22793_gb300 import epr as E
    phys, tab, tau = _case(n_lines, ny, nx, 21 + n_lines)
    xs = oracle.XSpec(phys[0], *tab, 30.0, 20e-6, nx)
    D = ph.poisson(oracle.forward_x(xs, tau.astype(np.float64)), 1e4, 4).astype(np.float32)
    Tr, ir = oracle.solve_x(xs, D.astype(np.float64), n_iter=10, omega=0.4)
    with _plan(E, phys, tab, ny, nx, deterministic=det) as p:
        Dd = torch.from_numpy(D).cuda()
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=10, omega=0.4)
        Tg = T.cpu().numpy()
        # back to the uniform spectrum: the plan solves like a fresh one
        E.epr_plan_set_xspec(p.handle)
        T2 = torch.empty_like(Dd)
        E.epr_solve_nonlocal(p.handle, Dd, T2, n_iter=3, omega=0.4)
        Tu = T2.cpu().numpy()
    assert rel(Tg, Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], ir["rho"], rtol=1e-3)
    Es, d, b, w = phys
    with E.Plan(nx, ny, 20e-6, 30.0, Es, d, b, w, deterministic=det) as q:
        T3 = torch.empty_like(Dd)
        E.epr_solve_nonlocal(q.handle, Dd, T3, n_iter=3, omega=0.4)
        assert rel(Tu, T3.cpu().numpy()) < (1e-12 if det else 1e-5)


def test_xspec_refuses_the_other_models(torch):
    from paper_2601_22793_gb300 import epr as E
    phys, tab, tau = _case(2, 64, 64, 5)
    with _plan(E, phys, tab, 64, 64) as p:
        D = torch.ones((64, 64), device="cuda")
        T = torch.empty_like(D)
        for call in (lambda: E.epr_solve_local(p.handle, D, T, order=2, n_iter=2),
                     lambda: E.epr_solve_nonlocal_wkb1(p.handle, D, T, n_iter=2),
                     lambda: E.epr_vjp(p.handle, D, D, T, 2)):
            with pytest.raises(E.EprError) as e:
                call()
            assert e.value.status == E.EPR_ERR_INVALID_ARG
        # a table with a non-positive weight is refused
        X, W, Dl, Bt = tab
        W = W.copy()
        W[0, 2] = 0.0
        with pytest.raises(E.EprError) as e:
            E.epr_plan_set_xspec(p.handle, X, W, Dl, Bt)
        assert e.value.status == E.EPR_ERR_INVALID_ARG
