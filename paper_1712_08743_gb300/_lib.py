"""ctypes view of the C ABI in ``include/helm.h`` (argument marshalling only).

``load()`` opens the in-tree ``_build/libhelm.so`` and raises if it is missing:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

HELM_OK = 0
HELM_PENDING = 1
HELM_E_INVALID = -1
HELM_E_NOMEM = -2
HELM_E_NOT_CONVERGED = -3
HELM_E_CUDA = -4
HELM_E_TIMEOUT = -5
HELM_E_BUSY = -6

HELM_PREC_MIXED = 0
HELM_PREC_FP64 = 1
HELM_PREC_FP32 = 2
HELM_PRECOND_MG = 0
HELM_PRECOND_NONE = 1
HELM_REORTH_ALWAYS = 0
HELM_REORTH_NEVER = 1
HELM_REORTH_IFNEEDED = 2
HELM_COARSE_AUTO = 0
HELM_COARSE_TAIL = 1
HELM_COARSE_DENSE = 2
HELM_COARSE_FUSED = 3
HELM_KERNEL_APPLY = 0
HELM_KERNEL_RESTRICT = 1
HELM_KERNEL_PROLONG = 2
HELM_KERNEL_BICG_XR = 3
HELM_KERNEL_RESID64 = 4
HELM_KERNEL_BICG_P = 5
HELM_KERNEL_APPLY64 = 6
HELM_KERNEL_FG_DOTS = 7
HELM_KERNEL_FG_AXPY = 8
HELM_KERNEL_TAIL = 9
HELM_KERNEL_FMA64 = 10
HELM_KRYLOV_BICGSTAB = 0
HELM_KRYLOV_FGMRES = 1
HELM_FWI_SIMULTANEOUS = 0
HELM_FWI_SEQUENTIAL = 1


class helm_solve_opts(C.Structure):
    _fields_ = [
        ("tol", C.c_double),
        ("max_it", C.c_int),
        ("krylov", C.c_int),
        ("restart", C.c_int),
        ("precision", C.c_int),
        ("beta1", C.c_double),
        ("beta2", C.c_double),
        ("omega_jacobi", C.c_double),
        ("inner_tol", C.c_double),
        ("max_outer", C.c_int),
        ("check_every", C.c_int),
        ("device_ptrs", C.c_int),
        ("use_graphs", C.c_int),
        ("precond", C.c_int),
        ("reorth", C.c_int),
        ("coarse", C.c_int),
    ]


class helm_fwi_opts(C.Structure):
    _fields_ = [
        ("strategy", C.c_int),
        ("gn_iters", C.c_int),
        ("cg_iters", C.c_int),
        ("max_halvings", C.c_int),
        ("m_lo", C.c_double),
        ("m_hi", C.c_double),
    ]


# void (*)(int group, int iter, const double* m, double J, void* user)
helm_fwi_checkpoint = C.CFUNCTYPE(None, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_double, C.c_void_p)


class helm_solve_stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("outer_its", C.c_int),
        ("converged", C.c_int),
        ("relres", C.c_double),
        ("dense_level", C.c_int),
        ("shift_switched", C.c_int),
    ]


class helm_request(C.Structure):
    _fields_ = [
        ("Px", C.c_int),
        ("Pz", C.c_int),
        ("h", C.c_double),
        ("slowness", C.POINTER(C.c_double)),
        ("npml", C.c_int),
        ("alpha_max", C.c_double),
        ("omega", C.c_double),
        ("src_ix", C.c_int),
        ("src_iz", C.c_int),
        ("opts", helm_solve_opts),
    ]


class helm_result(C.Structure):
    _fields_ = [
        ("u", C.c_void_p),
        ("nx", C.c_int),
        ("nz", C.c_int),
        ("status", C.c_int),
        ("stats", helm_solve_stats),
        ("latency_ms", C.c_double),
        ("queue_ms", C.c_double),
        ("batch_size", C.c_int),
    ]


class helm_profile_entry(C.Structure):
    _fields_ = [
        ("name", C.c_char * 32),
        ("nx", C.c_int),
        ("nz", C.c_int),
        ("launches", C.c_uint64),
        ("ms", C.c_double),
        ("bytes", C.c_double),
    ]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_pI = C.POINTER(C.c_int)
_pD = C.POINTER(C.c_double)
_pOpts = C.POINTER(helm_solve_opts)
_pStats = C.POINTER(helm_solve_stats)

# name -> (restype, argtypes); every function declared in include/helm.h
SIGNATURES = {
    "helm_default_opts": (None, [_pOpts]),
    "helm_strerror": (C.c_char_p, [_I]),
    "helm_last_error": (C.c_char_p, []),
    "helm_launch_count": (C.c_uint64, []),
    "helm_ctx_create": (_I, [_I, _P, C.POINTER(_P)]),
    "helm_ctx_destroy": (None, [_P]),
    "helm_create_model": (_I, [_P, _I, _I, _D, _pD, _I, _D, C.POINTER(_P)]),
    "helm_create_model_rho": (_I, [_P, _I, _I, _D, _pD, _pD, _I, _D, C.POINTER(_P)]),
    "helm_destroy_model": (None, [_P]),
    "helm_model_info": (_I, [_P, _pI, _pI, _pI]),
    "helm_solve": (_I, [_P, _I, _pD, _pI, _pI, _P, _P, _pOpts, _pStats]),
    "helm_adjoint_gradient": (_I, [_P, _I, _pD, _I, _pI, _pI, _I, _pI, _pI, _P, _D, _pD, _P, _P, _pOpts, _pStats]),
    "helm_fwi_forward": (_I, [_P, _I, _pD, _I, _pI, _pI, _I, _pI, _pI, _P, _D, _pD, _P, _pOpts, _pStats, C.POINTER(_P)]),
    "helm_fwi_backward": (_I, [_P, _P, _pOpts, _pStats]),
    "helm_fwi_state_destroy": (None, [_P]),
    "helm_gn_hvp": (_I, [_P, _P, _P, _pOpts, _pStats]),
    "helm_gn_step": (_I, [_P, _P, _I, _P, _pD, _pOpts]),
    "helm_fwi_run": (_I, [_P, _I, _I, _D, _I, _D, _pD, _I, _pD, _I, _pI, _pI, _I, _pI, _pI, _P, _D,
                          C.POINTER(helm_fwi_opts), _pOpts, _pD, _pD, _pI, helm_fwi_checkpoint, _P]),
    "helm_apply": (_I, [_P, _I, _pD, _I, _P, _P, _I]),
    "helm_vcycle": (_I, [_P, _I, _pD, _D, _D, _D, _P, _P, _I]),
    "helm_vcycle_noalloc": (_I, [_P, _I, _pD, _D, _D, _D, _P, _P]),
    "helm_vcycle_ex": (_I, [_P, _I, _pD, _pOpts, _P, _P]),
    "helm_profile_begin": (_I, []),
    "helm_profile_end": (_I, [C.POINTER(helm_profile_entry), _I, _pI]),
    "helm_autotune": (_I, [_P, _I, _D, _pI]),
    "helm_set_tiles": (_I, [_P, _pI]),
    "helm_time_kernel": (_I, [_P, _I, _I, _D, _I, _pD, _pD]),
    "helm_submit": (_I, [_P, C.POINTER(helm_request), C.POINTER(C.c_uint64)]),
    "helm_poll": (_I, [_P, C.c_uint64, _I, C.POINTER(helm_result)]),
    "helm_release": (_I, [_P, C.c_uint64]),
    "helm_serve_config": (_I, [_P, _I, _I, C.c_uint64, C.c_uint64]),
}

_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Open libhelm.so (optionally building it first). Raises if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path) and build_if_missing:
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libhelm.so is not built ({path}); run paper_1712_08743_gb300.build.build() "
                           "or __graft_entry__.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class HelmError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.helm_strerror(status).decode()
        detail = lib.helm_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


def check(status: int, where: str, allow=(HELM_OK,)) -> int:
    if status not in allow:
        raise HelmError(status, where)
    return status
