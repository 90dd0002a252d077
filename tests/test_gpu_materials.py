"""GPU parity on data that violate the single-material hypothesis: a
tissue / bone / void phantom whose tissue absorbs a third of what its phase
implies for bone (delta / beta 6000 against 2000), forward-modelled by the
oracle from the per-material phase and attenuation line integrals
(orc_forward_fields), Poisson(1e4) noise, 4 lines 60-160 keV, retrieved with
the single-material model (bone as reference, "Unknowns and single-thickness
constraint").  The solver is unchanged; the data are not a fixed point of its
model.  Tolerance: relative L2 <= 1e-4 on the thickness against the oracle's
retrieval of the same data, 1e-3 on the residual history.  The retrieval
error against the phase-equivalent thickness is larger than on matched data
of the same object."""
import numpy as np
import pytest

from paper_2601_22793_gb300 import phantoms as ph

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def case(oracle):
    """Data and oracle references, before any CUDA call of this module."""
    ny, nx, p, L = 256, 384, 20e-6, 30.0
    Es, d, b, w = ph.spectrum(4, 60.0, 160.0, 95.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, 91)
    ln = oracle.Lines(Es, d, b, w, L=L, pixel=p)
    ells = ph.random_ellipsoids(ny, nx, 24, 4.0, 40.0, seed=92)
    chords = ph.project_materials(ells, ny, nx, p)
    tau_pe = (ph.TISSUE[0] / ph.BONE[0]) * chords[0] + chords[1]
    Phi, A = oracle.material_fields(ln, chords, [ph.TISSUE[0], ph.BONE[0]],
                                    [ph.TISSUE[1], ph.BONE[1]], 80.0)
    D = ph.poisson(oracle.forward_fields(ln, Phi, A), 1e4, 93).astype(np.float32)
    Dm = ph.poisson(oracle.forward(ln, tau_pe), 1e4, 93).astype(np.float32)
    n_iter = 20
    Tr, ir = oracle.solve(ln, D.astype(np.float64), n_iter=n_iter, omega=0.4)
    Trm, _ = oracle.solve(ln, Dm.astype(np.float64), n_iter=n_iter, omega=0.4)
    return dict(ny=ny, nx=nx, p=p, L=L, spec=(Es, d, b, w), D=D, Tr=Tr, rho=ir["rho"],
                Trm=Trm, tau_pe=tau_pe, n_iter=n_iter)


@pytest.fixture(scope="module")
def torch(case):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_22793_gb300 import build
    build.build()
    from paper_2601_22793_gb300 import epr
    epr.load()
    return torch


@pytest.mark.parametrize("deterministic", [False, True])
def test_single_material_retrieval_of_two_material_data(torch, case, deterministic):
    from paper_2601_22793_gb300 import epr as E
    c = case
    Es, d, b, w = c["spec"]
    with E.Plan(c["nx"], c["ny"], c["p"], c["L"], Es, d, b, w, deterministic=deterministic) as plan:
        Dd = torch.from_numpy(c["D"]).cuda()
        T = torch.empty_like(Dd)
        info = E.epr_solve_nonlocal(plan.handle, Dd, T, n_iter=c["n_iter"], omega=0.4)
        Tg = T.cpu().numpy()
    assert rel(Tg, c["Tr"]) < 1e-4
    assert np.allclose(info["rho_hist"][0], c["rho"], rtol=1e-3)
    # the model mismatch shows in the retrieval error, not in the parity
    assert rel(c["Tr"], c["tau_pe"]) > rel(c["Trm"], c["tau_pe"])
