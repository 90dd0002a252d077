"""GPU reverse mode through the unrolled non-local solve (epr_solve_vjp),
through the C ABI:

* against the FP64 oracle's reverse pass (orc_solve_vjp) element by element
  on a two-line 24 x 32 phantom whose shifts keep 0.03 px from integer pixel
  crossings at every iterate and whose updates stay far above the floor (the
  preconditions of the oracle's finite-difference pins, checked here too):
  dF/dT0 and dF/dD within 1e-4 relative L2, dF/dL, dF/ddelta_s, dF/dbeta_s
  within 1e-4 relative;
* against central finite differences of the GPU solve itself (relative step
  1e-3) within 1e-3, as calibration by gradient descent would use it;
* checkpointing every m iterations gives the gradients of keeping every
  iterate."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NY, NX = 24, 32
E = np.array([60.0, 90.0])
DELTA = 2e-7 * (E[0] / E) ** 2
BETA = 1e-10 * (E[0] / E) ** 4
W = np.array([0.6, 0.4])
L0, PIX = 2.0, 6.5e-6
N_ITER, OMEGA = 4, 0.7


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


def _phantom():
    y, x = np.mgrid[0:NY, 0:NX].astype(np.float64)
    plane = 4.75e-5 * x + 3.2e-5 * y
    bump = 8e-5 * np.exp(-((x - 15.0) ** 2 + (y - 11.0) ** 2) / (2 * 6.0 ** 2))
    return plane.astype(np.float32), (plane + bump)


@pytest.fixture(scope="module")
def case(oracle):
    T0, tau = _phantom()
    ln = oracle.Lines(E, DELTA, BETA, W, L=L0, pixel=PIX)
    D = oracle.forward(ln, tau).astype(np.float32)
    wts = np.random.default_rng(11).standard_normal((NY, NX)).astype(np.float32)
    # preconditions: shifts off integer crossings, updates above the floor
    f, mu, k, c, eps = ln.params()
    T = T0.astype(np.float64)
    for it in range(N_ITER + 1):
        gy, gx = oracle.gradient(T)
        for s in range(2):
            for u in (c[s] * gx, c[s] * gy):
                frac = u - np.floor(u)
                assert frac.min() > 0.03 and frac.max() < 0.97
        T, _ = oracle.solve(ln, D.astype(np.float64), T0=T, n_iter=1, omega=OMEGA)
    ref = oracle.solve_vjp(ln, D.astype(np.float64), wts.astype(np.float64), N_ITER, omega=OMEGA,
                           T0=T0.astype(np.float64))
    return T0, D, wts, ref


def _plan(E_, L=L0, delta=DELTA, beta=BETA):
    return E_.Plan(NX, NY, PIX, L, E, delta, beta, W)


def _gpu_vjp(torch, E_, T0, D, wts, checkpoint_every=0, batch=1):
    with _plan(E_) as p:
        Dd = torch.from_numpy(np.ascontiguousarray(D)).cuda()
        T0d = torch.from_numpy(np.ascontiguousarray(T0)).cuda()
        Wd = torch.from_numpy(np.ascontiguousarray(wts)).cuda()
        t0b = torch.empty_like(Dd)
        Db = torch.empty_like(Dd)
        Tn = torch.empty_like(Dd)
        db, bb, lb = E_.epr_solve_vjp(p.handle, Dd, Wd, 2, N_ITER, omega=OMEGA, T0=T0d,
                                      checkpoint_every=checkpoint_every, batch=batch, T_out=Tn,
                                      T0_bar=t0b, D_bar=Db)
        return t0b.cpu().numpy(), Db.cpu().numpy(), db, bb, lb, Tn.cpu().numpy()


def test_solve_vjp_matches_the_oracle(torch, case):
    from paper_2601_22793_gb300 import epr as E_
    T0, D, wts, (t0r, Dr, dr, br, Lr) = case
    t0b, Db, db, bb, lb, _ = _gpu_vjp(torch, E_, T0, D, wts)
    assert rel(t0b, t0r) < 1e-4
    assert rel(Db, Dr) < 1e-4
    assert np.allclose(db[0], dr, rtol=1e-4, atol=0)
    assert np.allclose(bb[0], br, rtol=1e-4, atol=0)
    assert abs(lb[0] - Lr) <= 1e-4 * abs(Lr)


def test_checkpointing_gives_the_same_gradients(torch, case):
    from paper_2601_22793_gb300 import epr as E_
    T0, D, wts, _ = case
    full = _gpu_vjp(torch, E_, T0, D, wts, checkpoint_every=0)
    for m in (2, 3):
        seg = _gpu_vjp(torch, E_, T0, D, wts, checkpoint_every=m)
        # maps to 1e-6; the scalars to the ordering of the reverse splat's
        # float atomics (1e-5)
        for k, (a, b) in enumerate(zip(full, seg)):
            tol = 1e-5 if k in (2, 3, 4) else 1e-6
            assert np.allclose(a, b, rtol=tol, atol=tol * np.abs(b).max()), (m, k)


def test_batch_of_projections_is_per_projection(torch, case):
    from paper_2601_22793_gb300 import epr as E_
    T0, D, wts, _ = case
    one = _gpu_vjp(torch, E_, T0, D, wts)
    D2 = np.stack([D, D * np.float32(1.01)])
    T2 = np.stack([T0, T0])
    W2 = np.stack([wts, -wts])
    two = _gpu_vjp(torch, E_, T2, D2, W2, batch=2)
    assert rel(two[0][0], one[0]) < 1e-6 and rel(two[1][0], one[1]) < 1e-6
    assert np.allclose(two[2][0], one[2][0], rtol=1e-5) and abs(two[4][0] / one[4][0] - 1) < 1e-5
    # the second projection is another problem: its gradient differs
    assert rel(two[0][1], -one[0]) > 1e-4


def _gpu_F(torch, E_, wts, D, T0, L=L0, delta=DELTA, beta=BETA):
    with _plan(E_, L=L, delta=delta, beta=beta) as p:
        Dd = torch.from_numpy(np.ascontiguousarray(D, np.float32)).cuda()
        T = torch.from_numpy(np.ascontiguousarray(T0, np.float32)).cuda()
        E_.epr_solve_nonlocal(p.handle, Dd, T, n_iter=N_ITER, omega=OMEGA, init=1, want_info=False)
        return float(np.sum(wts.astype(np.float64) * T.cpu().numpy().astype(np.float64)))


def test_solve_vjp_matches_finite_differences_of_the_gpu_solve(torch, case):
    from paper_2601_22793_gb300 import epr as E_
    T0, D, wts, _ = case
    t0b, Db, db, bb, lb, _ = _gpu_vjp(torch, E_, T0, D, wts)
    h = 1e-3

    def cd(fn, x):
        return (fn(x * (1 + h)) - fn(x * (1 - h))) / (2 * h * x)

    dL = cd(lambda L: _gpu_F(torch, E_, wts, D, T0, L=L), L0)
    assert abs(lb[0] - dL) <= 1e-3 * abs(dL)
    for s in range(2):
        def Fd(v, s=s):
            d = DELTA.copy()
            d[s] = v
            return _gpu_F(torch, E_, wts, D, T0, delta=d)

        def Fb(v, s=s):
            b = BETA.copy()
            b[s] = v
            return _gpu_F(torch, E_, wts, D, T0, beta=b)

        dd = cd(Fd, DELTA[s])
        assert abs(db[0][s] - dd) <= 1e-3 * abs(dd), s
        dbt = cd(Fb, BETA[s])
        assert abs(bb[0][s] - dbt) <= 1e-3 * abs(dbt), s
    # directional derivatives in T0 and D, step 1e-3 of the field's scale
    g = np.random.default_rng(12)
    y, x = np.mgrid[0:NY, 0:NX].astype(np.float64)
    vT = (np.sin(0.3 * x + 0.2 * y) + 0.3 * g.standard_normal((NY, NX))) * np.abs(T0).max()
    vD = (np.cos(0.25 * x - 0.4 * y) + 0.3 * g.standard_normal((NY, NX)))
    eT = h
    dT = (_gpu_F(torch, E_, wts, D, T0 + eT * vT) - _gpu_F(torch, E_, wts, D, T0 - eT * vT)) / (2 * eT)
    dD = (_gpu_F(torch, E_, wts, D + h * vD, T0) - _gpu_F(torch, E_, wts, D - h * vD, T0)) / (2 * h)
    assert abs(np.sum(t0b * vT) - dT) <= 1e-3 * abs(dT)
    assert abs(np.sum(Db * vD) - dD) <= 1e-3 * abs(dD)


def test_set_params_solves_like_a_fresh_plan(torch, case):
    """epr_plan_set_params on an existing plan gives the plan of the new
    values (fixed-point splat: bit for bit), without a new plan."""
    from paper_2601_22793_gb300 import epr as E_
    T0, D, _, _ = case
    d2, b2, L2 = DELTA * 1.1, BETA * 0.9, L0 * 1.2
    Dd = torch.from_numpy(D).cuda()
    with E_.Plan(NX, NY, PIX, L0, E, DELTA, BETA, W, deterministic=True) as p:
        T = torch.empty_like(Dd)
        E_.epr_solve_nonlocal(p.handle, Dd, T, n_iter=3, omega=OMEGA)   # caches a graph
        E_.epr_plan_set_params(p.handle, L2, d2, b2)
        E_.epr_solve_nonlocal(p.handle, Dd, T, n_iter=3, omega=OMEGA)
        a = T.cpu().numpy()
    with E_.Plan(NX, NY, PIX, L2, E, d2, b2, W, deterministic=True) as q:
        T = torch.empty_like(Dd)
        E_.epr_solve_nonlocal(q.handle, Dd, T, n_iter=3, omega=OMEGA)
        assert np.array_equal(a, T.cpu().numpy())


def test_unrolled_solve_autograd(torch, case):
    """torch.autograd through UnrolledSolve gives epr_solve_vjp's gradients
    (to the ordering of the float atomics of the reverse splat: 1e-5 on the
    scalars), and a step of L changes F as the gradient predicts."""
    from paper_2601_22793_gb300 import epr as E_
    from paper_2601_22793_gb300.autograd import unrolled_solve
    T0, D, wts, _ = case
    direct = _gpu_vjp(torch, E_, T0, D, wts)
    Dd = torch.from_numpy(D).cuda().requires_grad_(True)
    T0d = torch.from_numpy(T0).cuda().requires_grad_(True)
    L = torch.tensor(L0, dtype=torch.float64, requires_grad=True)
    dl = torch.tensor(DELTA, requires_grad=True)
    bt = torch.tensor(BETA, requires_grad=True)
    Wd = torch.from_numpy(wts).cuda()
    for ck in (0, 2):
        T = unrolled_solve(Dd, L, dl, bt, energy_keV=E, pixel=PIX, weights=W, n_iter=N_ITER,
                           omega=OMEGA, T0=T0d, checkpoint_every=ck)
        F = (T.double() * Wd.double()).sum()
        gD, gT0, gL, gd, gb = torch.autograd.grad(F, (Dd, T0d, L, dl, bt))
        assert rel(gT0.cpu().numpy(), direct[0]) < 1e-6
        assert rel(gD.cpu().numpy(), direct[1]) < 1e-6
        assert np.allclose(gd.numpy(), direct[2][0], rtol=1e-5)
        assert np.allclose(gb.numpy(), direct[3][0], rtol=1e-5)
        assert abs(gL.item() / direct[4][0] - 1.0) < 1e-5
    h = 1e-3 * L0
    with torch.no_grad():
        Fp = (unrolled_solve(Dd, L0 + h, dl, bt, energy_keV=E, pixel=PIX, weights=W,
                             n_iter=N_ITER, omega=OMEGA, T0=T0d).double() * Wd.double()).sum()
        Fm = (unrolled_solve(Dd, L0 - h, dl, bt, energy_keV=E, pixel=PIX, weights=W,
                             n_iter=N_ITER, omega=OMEGA, T0=T0d).double() * Wd.double()).sum()
    fd = (Fp - Fm).item() / (2 * h)
    assert abs(gL.item() - fd) <= 1e-3 * abs(fd)
