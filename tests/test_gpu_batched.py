"""Batched solve of projections of uneven sizes and the splat autotuner,
through the C ABI.  In fixed-point mode the splat sums are exact, so a
batched solve must reproduce the single-size solves bit for bit, whatever
grouping, stream or tile shape it uses."""
import numpy as np
import pytest

from paper_2601_22793_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu

PHYS = dict(pixel=20e-6, L=30.0, E=[70.0, 110.0], delta=[2.6e-7, 1.06e-7], beta=[1.7e-10, 2.8e-11],
            w=[0.6, 0.4])


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_22793_gb300 import build
    build.build()
    return torch


def _data(oracle, ny, nx, seed):
    ells = ph.random_ellipsoids(ny, nx, 8, 4.0, min(ny, nx) / 8, margin=8.0, seed=seed)
    tau = ph.project_ellipsoids(ells, ny, nx, PHYS["pixel"])
    ln = oracle.Lines(PHYS["E"], PHYS["delta"], PHYS["beta"], PHYS["w"], L=PHYS["L"], pixel=PHYS["pixel"])
    return ph.poisson(oracle.forward(ln, tau), 1e4, seed).astype(np.float32)


def _single(E, torch, D, n_iter, tol, **kw):
    ny, nx = D.shape
    with E.Plan(nx, ny, PHYS["pixel"], PHYS["L"], PHYS["E"], PHYS["delta"], PHYS["beta"], PHYS["w"],
                **kw) as p:
        T = torch.empty((ny, nx), device="cuda")
        info = E.epr_solve_nonlocal(p.handle, torch.from_numpy(D).cuda(), T, n_iter=n_iter,
                                    omega=0.4, tol=tol)
        return T.cpu().numpy(), info


def test_batched_uneven_sizes_match_single_solves(torch, oracle):
    from paper_2601_22793_gb300 import epr as E
    shapes = [(128, 128), (96, 192), (128, 256), (128, 128), (48, 96)]
    Ds = [_data(oracle, ny, nx, 40 + i) for i, (ny, nx) in enumerate(shapes)]
    bh = E.epr_batch_create(PHYS["pixel"], PHYS["L"], PHYS["E"], PHYS["delta"], PHYS["beta"],
                            PHYS["w"], deterministic=True)
    try:
        Ts = [torch.empty(D.shape, device="cuda") for D in Ds]
        info = E.epr_solve_nonlocal_batched(bh, [torch.from_numpy(D).cuda() for D in Ds], Ts,
                                            n_iter=6, omega=0.4)
        for i, D in enumerate(Ds):
            Tref, iref = _single(E, torch, D, 6, 0.0, deterministic=True)
            assert np.array_equal(Ts[i].cpu().numpy(), Tref), i
            assert info["iters"][i] == 6
            assert np.array_equal(info["rho_hist"][i], iref["rho_hist"][0])
        # host buffers, second call on the same batch object (cached plans)
        Th = [np.zeros(D.shape, np.float32) for D in Ds]
        E.epr_solve_nonlocal_batched(bh, Ds, Th, n_iter=6, omega=0.4)
        for i in range(len(Ds)):
            assert np.array_equal(Th[i], Ts[i].cpu().numpy())
    finally:
        E.epr_batch_destroy(bh)


def test_batched_projections_stop_on_their_own(torch, oracle):
    from paper_2601_22793_gb300 import epr as E
    shapes = [(96, 96), (96, 96), (64, 128)]
    Ds = [_data(oracle, ny, nx, 60 + i) for i, (ny, nx) in enumerate(shapes)]
    Ds[1] = np.ones_like(Ds[1])      # flat field: converges at once
    bh = E.epr_batch_create(PHYS["pixel"], PHYS["L"], PHYS["E"], PHYS["delta"], PHYS["beta"],
                            PHYS["w"], deterministic=True)
    try:
        Ts = [torch.empty(D.shape, device="cuda") for D in Ds]
        info = E.epr_solve_nonlocal_batched(bh, [torch.from_numpy(D).cuda() for D in Ds], Ts,
                                            n_iter=30, omega=0.4, tol=2e-3)
        for i, D in enumerate(Ds):
            Tref, iref = _single(E, torch, D, 30, 2e-3, deterministic=True)
            assert info["iters"][i] == iref["iters"][0], i
            assert np.array_equal(Ts[i].cpu().numpy(), Tref), i
        assert info["iters"][1] <= 2 < info["iters"][0]   # each projection stops on its own
    finally:
        E.epr_batch_destroy(bh)


def test_autotune_changes_speed_not_results(torch, oracle):
    from paper_2601_22793_gb300 import epr as E
    D = _data(oracle, 192, 256, 77)
    Tref, _ = _single(E, torch, D, 8, 0.0, deterministic=True)
    with E.Plan(256, 192, PHYS["pixel"], PHYS["L"], PHYS["E"], PHYS["delta"], PHYS["beta"], PHYS["w"],
                deterministic=True, autotune=True) as p:
        Dd = torch.from_numpy(D).cuda()
        outs = []
        for _ in range(3):     # the first solve triggers the tuning
            T = torch.empty_like(Dd)
            E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=8, omega=0.4)
            outs.append(T.cpu().numpy())
    for o in outs:
        assert np.array_equal(o, Tref)
    # float mode: tuned and untuned agree to float rounding
    Tf, _ = _single(E, torch, D, 8, 0.0)
    with E.Plan(256, 192, PHYS["pixel"], PHYS["L"], PHYS["E"], PHYS["delta"], PHYS["beta"], PHYS["w"],
                autotune=True) as p:
        Dd = torch.from_numpy(D).cuda()
        for _ in range(2):
            T = torch.empty_like(Dd)
            E.epr_solve_nonlocal(p.handle, Dd, T, n_iter=8, omega=0.4)
    Tt = T.cpu().numpy()
    assert np.linalg.norm(Tt - Tf) / np.linalg.norm(Tf) < 1e-5
