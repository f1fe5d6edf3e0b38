"""GPU: the kernel timing entry point that feeds the roofline report runs every
kernel it declares and reports the algorithmic bytes of one launch."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import paper_1712_08743_gb300 as hg

    hg.load(build_if_missing=True)
    return hg


def test_time_kernel_bytes_and_times(hg):
    from paper_1712_08743_gb300 import _lib, api

    lib = _lib.load()
    ctx = hg.Context(0)
    Px, Pz, npml = 61, 45, 10
    model = hg.helm_create_model(ctx, np.full((Pz, Px), 1 / 2000.0), 10.0, npml)
    n = float((Px + 2 * npml) * (Pz + 2 * npml))
    nrhs = 3
    # bytes per launch as the header documents them (j = 4 for the Gram-Schmidt kernels)
    expect = {
        _lib.HELM_KERNEL_APPLY: n * (16.0 * nrhs + 4.0),
        _lib.HELM_KERNEL_APPLY64: n * (32.0 * nrhs + 8.0),
        _lib.HELM_KERNEL_BICG_XR: n * nrhs * 64.0,
        _lib.HELM_KERNEL_BICG_P: n * nrhs * 32.0,
        _lib.HELM_KERNEL_RESID64: n * (40.0 * nrhs + 8.0),
        _lib.HELM_KERNEL_FG_DOTS: n * nrhs * 8.0 * 6,
        _lib.HELM_KERNEL_FG_AXPY: n * nrhs * 8.0 * 7,
    }
    for kid in range(11):
        ms, byt = C.c_double(), C.c_double()
        api.check(lib.helm_time_kernel(model.handle, kid, nrhs, 2 * np.pi * 5.0, 3, C.byref(ms), C.byref(byt)),
                  "helm_time_kernel")
        assert ms.value > 0.0 and byt.value > 0.0, kid
        if kid in expect:
            assert byt.value == pytest.approx(expect[kid], rel=1e-12), kid
    # the tail moves its top level's input and output: a whole number of complex64
    # nodes per right-hand side, at most the 2048 of a complex64 tail level
    ms, byt = C.c_double(), C.c_double()
    api.check(lib.helm_time_kernel(model.handle, _lib.HELM_KERNEL_TAIL, nrhs, 2 * np.pi * 5.0, 3, C.byref(ms),
                                   C.byref(byt)), "helm_time_kernel")
    nodes = byt.value / (16.0 * nrhs)
    assert nodes == int(nodes) and 1 <= nodes <= 2048
    # the FP64 probe reports its FP64 operations: 8 blocks of 256 threads per SM, 8 chains of
    # 2048 fused multiply-adds each, 2 operations per multiply-add
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    api.check(lib.helm_time_kernel(model.handle, _lib.HELM_KERNEL_FMA64, 1, 1.0, 3, C.byref(ms), C.byref(byt)),
              "helm_time_kernel")
    assert byt.value == 2.0 * 8 * sms * 256 * 8 * 2048
    assert lib.helm_time_kernel(model.handle, 11, nrhs, 2 * np.pi * 5.0, 3, C.byref(ms), C.byref(byt)) == \
        _lib.HELM_E_INVALID
    model.close()
    ctx.close()
