"""GPU parity of the oversampled internal grid (reading R11) through the C
ABI: solves against the oracle's oversampled solve, the forward's detector
image against the block mean of the oracle's fine forward, and the calls
that refuse an oversampled plan."""
import numpy as np
import pytest

from paper_2601_22793_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu

P_DET = 20e-6


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_22793_gb300 import build
    build.build()
    return torch


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _phys(n_lines):
    if n_lines == 1:
        return [80.0], [2e-7], [1e-10], [1.0]
    return [60.0, 90.0], [3.6e-7, 1.6e-7], [3.2e-10, 4e-11], [0.6, 0.4]


def _data(oracle, nyd, nxd, os_, n_lines, model, seed, L=10.0):
    E, d, b, w = _phys(n_lines)
    ny, nx = nyd * os_, nxd * os_
    ells = ph.random_ellipsoids(ny, nx, 8, 3.0 * os_, 12.0 * os_, margin=6.0 * os_, seed=seed)
    tau = ph.project_ellipsoids(ells, ny, nx, P_DET / os_)
    fine = oracle.Lines(E, d, b, w, L=L, pixel=P_DET / os_)
    Dd = oracle.bin_mean(oracle.forward(fine, tau, model=model), os_)
    return ph.poisson(Dd, 1e4, seed).astype(np.float32), tau.astype(np.float32)


# The order-2 local closure at L = 10 m on the 10 um fine pixel diverges in
# the oracle as well (its diffraction-pressure term grows as 1/p^4), so that
# case runs at L = 4 m, where the iteration contracts.
@pytest.mark.parametrize("nyd,nxd,os_,n_lines,model,det,L", [
    (48, 64, 2, 1, 0, False, 10.0), (48, 64, 2, 1, 0, True, 10.0), (32, 32, 4, 2, 0, False, 10.0),
    (64, 48, 2, 2, 2, False, 4.0), (32, 48, 2, 1, 1, False, 10.0),
    (16, 2048, 4, 1, 0, False, 10.0), (2048, 16, 4, 2, 0, False, 10.0),
    # 4096 internal rows: the bulk-copy column pass of two 4096-point columns
    (1024, 16, 4, 1, 0, False, 10.0), (2048, 24, 2, 2, 0, False, 10.0),
    (2048, 16, 2, 1, 2, False, 4.0)])
def test_oversampled_solve_vs_oracle(torch, oracle, nyd, nxd, os_, n_lines, model, det, L):
    from paper_2601_22793_gb300 import epr as E
    D, _ = _data(oracle, nyd, nxd, os_, n_lines, model, 80 + nyd + os_, L)
    Ee, d, b, w = _phys(n_lines)
    ln = oracle.Lines(Ee, d, b, w, L=L, pixel=P_DET)
    Tr, ir = oracle.solve_os(ln, D.astype(np.float64), os_, n_iter=6, omega=0.5, model=model)
    with E.Plan(nxd, nyd, P_DET, L, Ee, d, b, w, oversample=os_, deterministic=det) as p:
        Dd = torch.from_numpy(D).cuda()
        T = torch.empty((nyd * os_, nxd * os_), device="cuda")
        if model == 0:
            info = E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=6, omega=0.5)
        else:
            info = E.epr_solve_local(p.handle, Dd, T, order=model, n_iter=6, omega=0.5)
        Tg = T.cpu().numpy()
    assert rel(Tg, Tr) < 1e-4
    assert np.allclose(info["rho_hist"][0], ir["rho"], rtol=1e-3)


@pytest.mark.parametrize("os_,n_lines,det", [(2, 1, False), (4, 2, False), (2, 2, True)])
def test_oversampled_forward_is_the_block_mean(torch, oracle, os_, n_lines, det):
    from paper_2601_22793_gb300 import epr as E
    nyd, nxd = 32, 48
    _, tau = _data(oracle, nyd, nxd, os_, n_lines, 0, 90 + os_)
    Ee, d, b, w = _phys(n_lines)
    fine = oracle.Lines(Ee, d, b, w, L=10.0, pixel=P_DET / os_)
    Pf, Psf, _ = oracle.forward(fine, tau.astype(np.float64), per_line=True)
    with E.Plan(nxd, nyd, P_DET, 10.0, Ee, d, b, w, oversample=os_, deterministic=det) as p:
        T = torch.from_numpy(tau).cuda()
        P = torch.empty((nyd, nxd), device="cuda")
        Ps = torch.empty((n_lines, nyd, nxd), device="cuda")
        E.epr_forward(p.handle, T, P, Ps)
        torch.cuda.synchronize()
        Pg, Psg = P.cpu().numpy(), Ps.cpu().numpy()
    assert rel(Pg, oracle.bin_mean(Pf, os_)) < 1e-5
    for s in range(n_lines):
        assert rel(Psg[s], oracle.bin_mean(Psf[s], os_)) < 1e-5


def test_oversampled_plan_refuses_vjp_and_batches(torch):
    from paper_2601_22793_gb300 import epr as E
    with E.Plan(32, 32, P_DET, 10.0, [80.0], [2e-7], [1e-10], [1.0], oversample=2) as p:
        T = torch.zeros((64, 64), device="cuda")
        with pytest.raises(E.EprError):
            E.epr_vjp(p.handle, T, T, torch.empty_like(T), 1)
    with pytest.raises(E.EprError):
        E.epr_batch_create(P_DET, 10.0, [80.0], [2e-7], [1e-10], [1.0], oversample=2)


def test_internal_grid_limits(torch):
    """Detector sides up to 4096 and internal sides up to 8192; the plain
    preconditioner entry point, on the runtime-sized engine, refuses 8192."""
    from paper_2601_22793_gb300 import epr as E
    phys = (P_DET, 10.0, [80.0], [2e-7], [1e-10], [1.0])
    with pytest.raises(E.EprError):
        E.Plan(4096, 16, *phys, oversample=4)          # 16384 internal
    with E.Plan(2048, 16, *phys, oversample=4) as p:    # 8192 x 64 internal
        g = torch.zeros((64, 8192), device="cuda")
        with pytest.raises(E.EprError):
            E.epr_precondition(p.handle, g, 0)
