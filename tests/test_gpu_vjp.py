"""GPU vector-Jacobian product of the non-local forward (epr_vjp) and the
torch.autograd binding, against the FP64 oracle's VJP and against central
finite differences of the oracle forward.  The phantom keeps every mapped
point at least 1e-2 px from a pixel boundary, where the transport is not
differentiable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_22793_gb300 import build
    build.build()
    return torch


def _case(oracle, ny=96, nx=128):
    E, delta, beta, w = [60.0, 90.0], [1.4e-7, 7e-8], [9e-11, 3e-11], [0.6, 0.4]
    p, L = 6.5e-6, 2.0
    ln = oracle.Lines(E, delta, beta, w, L=L, pixel=p)
    f, mu, k, c, eps = ln.params()
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    ax, ay = 0.45 / c[0], 0.35 / c[0]
    A = 0.08 * 40 / (2 * np.pi * abs(c[0]))
    tau = 3e-3 + ax * (xx - nx / 2) + ay * (yy - ny / 2) \
        + A * np.sin(2 * np.pi * xx / 40) * np.sin(2 * np.pi * yy / 50)
    tau = tau.astype(np.float32)
    gy, gx = oracle.gradient(tau.astype(np.float64))
    for s in range(2):
        for u in (c[s] * gx, c[s] * gy):
            assert np.abs(u - np.round(u)).min() > 1e-2
    gbar = np.random.default_rng(4).normal(size=(ny, nx)).astype(np.float32)
    return ln, tau, gbar, (E, delta, beta, w, p, L)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


def test_vjp_matches_oracle(torch, oracle):
    from paper_2601_22793_gb300 import epr
    ln, tau, gbar, (E, delta, beta, w, p, L) = _case(oracle)
    Tb_o, db_o, bb_o, lb_o = oracle.vjp(ln, tau.astype(np.float64), gbar.astype(np.float64))
    with epr.Plan(tau.shape[1], tau.shape[0], p, L, E, delta, beta, w) as plan:
        T = torch.from_numpy(tau).cuda()
        G = torch.from_numpy(gbar).cuda()
        Tb = torch.empty_like(T)
        db, bb, lb = epr.epr_vjp(plan.handle, T, G, Tb, 2)
    assert rel(Tb.cpu().numpy(), Tb_o) < 1e-4
    assert np.allclose(db[0], db_o, rtol=1e-4)
    assert np.allclose(bb[0], bb_o, rtol=1e-4)
    assert abs(lb[0] - lb_o) <= 1e-4 * abs(lb_o)


def test_autograd_matches_finite_differences(torch, oracle):
    """Gradients of F = <W, P> through the autograd function against central
    finite differences (relative step 1e-3) of the FP64 oracle forward."""
    from paper_2601_22793_gb300.autograd import eikonal_forward
    ln, tau, W, (E, delta, beta, w, p, L) = _case(oracle)
    T = torch.from_numpy(tau).cuda().requires_grad_(True)
    Lt = torch.tensor(L, dtype=torch.float64, requires_grad=True)
    dt = torch.tensor(delta, dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    P = eikonal_forward(T, Lt, dt, bt, energy_keV=E, pixel=p, weights=w)
    F = (P * torch.from_numpy(W).cuda()).sum()
    F.backward()

    W64, T64 = W.astype(np.float64), tau.astype(np.float64)

    def Fo(T_=T64, L_=L, d=delta, b=beta):
        return float(np.sum(W64 * oracle.forward(oracle.Lines(E, d, b, w, L=L_, pixel=p), T_)))

    v = np.cos(np.arange(tau.size).reshape(tau.shape) * 0.013)
    h = 1e-3 * 1e-3    # 1e-3 of the thickness scale (~1e-3 m)
    fd = (Fo(T_=T64 + h * v) - Fo(T_=T64 - h * v)) / (2 * h)
    an = float((T.grad.double().cpu().numpy() * v).sum())
    assert abs(an - fd) <= 1e-3 * abs(fd)
    hL = 1e-3 * L
    fd = (Fo(L_=L + hL) - Fo(L_=L - hL)) / (2 * hL)
    assert abs(Lt.grad.item() - fd) <= 1e-3 * abs(fd)
    for s in range(2):
        dp, dm = list(delta), list(delta)
        dp[s] *= 1 + 1e-3
        dm[s] *= 1 - 1e-3
        fd = (Fo(d=dp) - Fo(d=dm)) / (2e-3 * delta[s])
        assert abs(dt.grad[s].item() - fd) <= 1e-3 * abs(fd)
        bp, bm = list(beta), list(beta)
        bp[s] *= 1 + 1e-3
        bm[s] *= 1 - 1e-3
        fd = (Fo(b=bp) - Fo(b=bm)) / (2e-3 * beta[s])
        assert abs(bt.grad[s].item() - fd) <= 1e-3 * abs(fd)
