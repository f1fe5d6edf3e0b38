"""The V-cycle entry point that allocates no device memory.

helm_vcycle_noalloc serves callers whose device memory belongs to another
allocator (or must not grow after start-up): it runs the V-cycle on a fixed
scratch array inside the library. Two calls in a row, through the C ABI, must
give the result of the allocating helm_vcycle within the V-cycle tolerance of
the parity tests (2e-5 relative), although the second call finds the first
call's data still in the scratch array. This file sorts last so that a run that
stops at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_vcycle_noalloc_matches_allocating_vcycle_twice():
    import torch

    import paper_1712_08743_gb300 as hg
    from synth import models

    lib = hg.load(build_if_missing=True)
    ctx = hg.Context(0)
    mdl = models.c1_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    rng = np.random.default_rng(7)
    om = 2 * np.pi * np.array([4.0, 6.0, 4.0])
    omp = om.ctypes.data_as(C.POINTER(C.c_double))
    r = torch.from_numpy(models.random_complex(rng, (3, model.nz, model.nx), np.complex64)).cuda()
    z_ref = torch.empty_like(r)
    torch.cuda.synchronize()
    assert lib.helm_vcycle(model.handle, 3, omp, 1.0, 0.5, 0.8, C.c_void_p(r.data_ptr()),
                           C.c_void_p(z_ref.data_ptr()), 1) == hg.HELM_OK
    ref = z_ref.cpu().numpy()
    for _ in range(2):
        z = torch.full_like(r, float("nan"))
        torch.cuda.synchronize()
        st = lib.helm_vcycle_noalloc(model.handle, 3, omp, 1.0, 0.5, 0.8, C.c_void_p(r.data_ptr()),
                                     C.c_void_p(z.data_ptr()))
        assert st == hg.HELM_OK, lib.helm_last_error()
        got = z.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-5
    model.close()
    # a batch whose level vectors exceed the fixed scratch (256 RHS on a 441 x 241 grid need
    # about 144 MB) is refused before any launch, with the size in the message
    m3 = models.c3_model()
    big_model = hg.helm_create_model(ctx, m3.slowness, m3.h, m3.npml, m3.alpha_max)
    big = np.full(256, om[0])
    rb = torch.zeros((1,), dtype=torch.complex64, device="cuda")
    st = lib.helm_vcycle_noalloc(big_model.handle, 256, big.ctypes.data_as(C.POINTER(C.c_double)), 1.0, 0.5, 0.8,
                                 C.c_void_p(rb.data_ptr()), C.c_void_p(rb.data_ptr()))
    assert st == hg.HELM_E_INVALID and b"64 MiB" in lib.helm_last_error()
    big_model.close()
    ctx.close()
