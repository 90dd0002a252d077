"""The preconditioner entry point that allocates nothing.

Callers whose device memory is owned by their own pool allocator or fixed at
start-up cannot let a library call cudaMalloc; epr_precondition_noalloc
keeps its scratch in a static device array instead.  This test calls it
through the C ABI and checks it against the plan-based epr_precondition, on
two calls in a row (the second call reuses the array the first one left
behind).  It sits in a file of its own, collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_precondition_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_22793_gb300 import build, epr
    build.build()
    lib = epr.load()
    ny, nx, batch = 384, 512, 3
    pixel, L, E, delta, beta = 20e-6, 30.0, 80.0, 2e-7, 1e-10
    rng = np.random.default_rng(5)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with epr.Plan(nx, ny, pixel, L, [E], [delta], [beta]) as plan:
        for call in range(2):
            g0 = torch.from_numpy(rng.normal(size=(batch, ny, nx)).astype(np.float32)).cuda()
            ref = g0.clone()
            epr.epr_precondition(plan.handle, ref, line=0, batch=batch)
            out = g0.clone()
            st = lib.epr_precondition_noalloc(ctypes.c_void_p(out.data_ptr()), nx, ny, pixel, L,
                                              E, delta, beta, batch, stream)
            assert st == epr.EPR_OK, epr.epr_status_string(st)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5, call


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_22793_gb300 import build, epr
    build.build()
    g = torch.zeros((2, 2048, 2048), device="cuda")
    with pytest.raises(epr.EprError) as e:
        epr.epr_precondition_noalloc(g, 2048, 2048, 20e-6, 30.0, 80.0, 2e-7, 1e-10, batch=2)
    assert e.value.status == epr.EPR_ERR_UNSUPPORTED_SIZE
