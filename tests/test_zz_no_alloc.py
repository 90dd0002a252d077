"""The preconditioner entry point that allocates nothing.

Some callers cannot let a library call cudaMalloc: their device memory is
handed out by their own pool allocator or fixed at start-up, or an
allocation's possible device synchronisation is not acceptable on their
path.  epr_precondition_noalloc keeps its scratch in a static device array
instead.  This test calls it through the C ABI on two calls in a row (the
second call reuses the array the first one left behind) and checks each
against the FP64 oracle's preconditioner, within the 1e-5 relative L2 of the
other per-application parity tests; it checks that the second call leaves
the device's free memory unchanged, that a request of exactly the array's
limit works and that a larger one is refused.  It sits in a file of its own,
collected last."""
import ctypes

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


def _call(torch, lib, g, nx, ny, phys, batch):
    pixel, L, E, delta, beta = phys
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.epr_precondition_noalloc(ctypes.c_void_p(g.data_ptr()), nx, ny, pixel, L, E,
                                        delta, beta, batch, stream)


def _oracle_ref(oracle, g, phys):
    pixel, L, E, delta, beta = phys
    ln = oracle.Lines([E], [delta], [beta], [1.0], L=L, pixel=pixel)
    return np.stack([oracle.precondition(ln, m.astype(np.float64)) for m in g])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_the_oracle_twice_and_allocates_nothing(torch, oracle):
    from paper_2601_22793_gb300 import epr
    lib = epr.load()
    ny, nx, batch = 384, 512, 3
    phys = (20e-6, 30.0, 80.0, 2e-7, 1e-10)
    rng = np.random.default_rng(5)
    for call in range(2):
        g0 = rng.normal(size=(batch, ny, nx)).astype(np.float32)
        out = torch.from_numpy(g0).cuda()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _call(torch, lib, out, nx, ny, phys, batch)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert st == epr.EPR_OK, epr.epr_status_string(st)
        if call == 1:   # the first call may load kernels; the second allocates nothing
            assert free1 == free0
        assert rel(out.cpu().numpy().astype(np.float64), _oracle_ref(oracle, g0, phys)) < 1e-5, call


def test_noalloc_at_the_size_limit(torch, oracle):
    """batch * nx * ny = 4 Mi pixels exactly (one 2048 x 2048 map) works."""
    from paper_2601_22793_gb300 import epr
    lib = epr.load()
    phys = (20e-6, 30.0, 80.0, 2e-7, 1e-10)
    g0 = np.random.default_rng(6).normal(size=(1, 2048, 2048)).astype(np.float32)
    out = torch.from_numpy(g0).cuda()
    assert _call(torch, lib, out, 2048, 2048, phys, 1) == epr.EPR_OK
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy().astype(np.float64), _oracle_ref(oracle, g0, phys)) < 1e-5


def test_noalloc_rejects_sizes_beyond_the_static_scratch(torch):
    from paper_2601_22793_gb300 import epr
    g = torch.zeros((2, 2048, 2048), device="cuda")
    with pytest.raises(epr.EprError) as e:
        epr.epr_precondition_noalloc(g, 2048, 2048, 20e-6, 30.0, 80.0, 2e-7, 1e-10, batch=2)
    assert e.value.status == epr.EPR_ERR_UNSUPPORTED_SIZE
