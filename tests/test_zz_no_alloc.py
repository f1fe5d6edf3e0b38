"""The preconditioner entry point that allocates no device memory.

helm_vcycle_noalloc serves callers whose device memory belongs to another
allocator (a framework's caching allocator or a fixed arena) or must not grow
after start-up: it runs the preconditioner cycle on a fixed scratch array inside
the library. Two calls in a row, through the C ABI, must give the result of the
allocating helm_vcycle bit for bit (the same kernels in the same order on the
same inputs), although the second call finds the first call's data still in the
scratch array; and the second call must leave the device's memory untouched: the
stream-ordered pool's high-water mark and the free device memory do not move.
This file sorts last so that a run that stops at its first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7   # CUmemPool_attribute values of cuda.h
CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


class DefaultPool:
    """The device's default stream-ordered memory pool, seen through the driver API
    (the pool cudaMallocAsync draws from, whichever runtime calls it)."""

    def __init__(self, device: int):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), device) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr: int) -> int:
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, C.byref(zero)) == 0


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
    assert np.all(np.isfinite(ref))
    pool = DefaultPool(0)
    for call in range(2):
        z = torch.full_like(r, float("nan"))
        torch.cuda.synchronize()
        if call == 1:   # the second call: nothing may be allocated, not even for a moment
            pool.reset_high()
            used0 = pool.get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)
            free0 = torch.cuda.mem_get_info(0)[0]
        st = lib.helm_vcycle_noalloc(model.handle, 3, omp, 1.0, 0.5, 0.8, C.c_void_p(r.data_ptr()),
                                     C.c_void_p(z.data_ptr()))
        assert st == hg.HELM_OK, lib.helm_last_error()
        torch.cuda.synchronize()
        if call == 1:
            assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_HIGH) <= used0
            assert torch.cuda.mem_get_info(0)[0] == free0
        got = z.cpu().numpy()
        assert np.array_equal(got, ref)
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
