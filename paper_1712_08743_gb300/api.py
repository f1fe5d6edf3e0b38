"""Thin Python binding of the C ABI, with the same names as ``include/helm.h``.

Arguments are marshalled to the library and nothing else: every step of the
solve, the V-cycle and the gradient runs in the CUDA kernels of libhelm.so.
Host arrays are NumPy arrays; device arrays are contiguous CUDA torch tensors
(then ``opts.device_ptrs`` is set and the library reads/writes them in place).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import check, load

try:  # torch is plumbing only (device memory, streams)
    import torch
except Exception:  # pragma: no cover
    torch = None


def _is_cuda_tensor(x) -> bool:
    return torch is not None and isinstance(x, torch.Tensor) and x.is_cuda


def _np(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _ptr_d(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptr_i(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


# ------------------------------------------------------------------ options
def helm_default_opts(**overrides) -> _lib.helm_solve_opts:
    o = _lib.helm_solve_opts()
    load().helm_default_opts(C.byref(o))
    for k, v in overrides.items():
        if k == "beta":
            o.beta1, o.beta2 = float(v[0]), float(v[1])
        elif k == "precision" and isinstance(v, str):
            o.precision = {"mixed": _lib.HELM_PREC_MIXED, "fp64": _lib.HELM_PREC_FP64,
                           "fp32": _lib.HELM_PREC_FP32}[v]
        else:
            if not hasattr(o, k):
                raise KeyError(f"unknown option {k}")
            setattr(o, k, v)
    return o


def _opts(opts, **extra) -> _lib.helm_solve_opts:
    if opts is None:
        o = helm_default_opts()
    elif isinstance(opts, dict):
        o = helm_default_opts(**opts)
    else:
        o = _lib.helm_solve_opts()
        C.pointer(o)[0] = opts
    for k, v in extra.items():
        setattr(o, k, v)
    return o


def stats_list(arr, n):
    return [dict(iters=arr[i].iters, outer_its=arr[i].outer_its, converged=bool(arr[i].converged),
                 relres=arr[i].relres, dense_level=arr[i].dense_level, shift_switched=bool(arr[i].shift_switched))
            for i in range(n)]


# ------------------------------------------------------------------ context
class Context:
    """A helm_ctx on one device; all calls of its models run on its stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        self.handle = C.c_void_p()
        s = None
        if stream is not None:
            s = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        check(self.lib.helm_ctx_create(int(device), s, C.byref(self.handle)), "helm_ctx_create")
        self.device = int(device)

    def close(self):
        if self.handle:
            self.lib.helm_ctx_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def helm_ctx_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def helm_ctx_destroy(ctx: Context) -> None:
    ctx.close()


class Model:
    """A helm_model: padded slowness and its multigrid hierarchy on the device."""

    def __init__(self, ctx: Context, slowness, h: float, npml: int = 20, alpha_max: float = 0.5, density=None):
        m = _np(slowness, np.float64)
        if m.ndim != 2:
            raise ValueError("slowness must be [Pz][Px]")
        self.ctx = ctx
        self.lib = ctx.lib
        self.Pz, self.Px = m.shape
        self.h, self.npml, self.alpha_max = float(h), int(npml), float(alpha_max)
        self.handle = C.c_void_p()
        if density is None:
            check(self.lib.helm_create_model(ctx.handle, self.Px, self.Pz, self.h, _ptr_d(m), self.npml,
                                             self.alpha_max, C.byref(self.handle)), "helm_create_model")
        else:
            rho = _np(density, np.float64)
            if rho.shape != m.shape:
                raise ValueError("density must have the slowness's shape")
            check(self.lib.helm_create_model_rho(ctx.handle, self.Px, self.Pz, self.h, _ptr_d(m), _ptr_d(rho),
                                                 self.npml, self.alpha_max, C.byref(self.handle)),
                  "helm_create_model_rho")
        nx, nz, nl = C.c_int(), C.c_int(), C.c_int()
        check(self.lib.helm_model_info(self.handle, C.byref(nx), C.byref(nz), C.byref(nl)), "helm_model_info")
        self.nx, self.nz, self.nlevels = nx.value, nz.value, nl.value

    @property
    def n(self) -> int:
        return self.nx * self.nz

    def close(self):
        if self.handle:
            self.lib.helm_destroy_model(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def helm_create_model(ctx: Context, slowness, h: float, npml: int = 20, alpha_max: float = 0.5,
                      density=None) -> Model:
    """A model of Eq. 2, or with `density` ([Pz][Px], > 0) of Eq. 1 (helm_create_model_rho)."""
    return Model(ctx, slowness, h, npml, alpha_max, density)


def helm_destroy_model(model: Model) -> None:
    model.close()


# -------------------------------------------------------------------- solve
def helm_solve(model: Model, omega, src=None, f=None, opts=None, out=None):
    """u = B^{-1} f for every right-hand side (Eq. 3).

    omega: [nrhs] angular frequencies. src: [nrhs, 2] physical (ix, iz) of unit point
    sources (used when f is None). f: complex128 [nrhs][nz][nx] (NumPy, or CUDA
    tensor). Returns (u [nrhs][nz][nx] complex128, stats list, status).
    """
    lib = model.lib
    om = _np(omega, np.float64).reshape(-1)
    nrhs = om.size
    dev = _is_cuda_tensor(f) or _is_cuda_tensor(out)
    o = _opts(opts, device_ptrs=1 if dev else 0)
    sx = sz = None
    if f is None:
        s = _np(src, np.int32).reshape(nrhs, 2)
        sx, sz = _np(s[:, 0], np.int32), _np(s[:, 1], np.int32)
    stats = (_lib.helm_solve_stats * nrhs)()
    if dev:
        if out is None:
            out = torch.empty((nrhs, model.nz, model.nx), dtype=torch.complex128, device=f.device if f is not None else "cuda")
        assert out.is_contiguous() and out.dtype == torch.complex128
        fp = None
        if f is not None:
            assert f.is_contiguous() and f.dtype == torch.complex128
            fp = C.c_void_p(f.data_ptr())
        torch.cuda.synchronize()
        st = lib.helm_solve(model.handle, nrhs, _ptr_d(om), _ptr_i(sx) if sx is not None else None,
                            _ptr_i(sz) if sz is not None else None, fp, C.c_void_p(out.data_ptr()),
                            C.byref(o), stats)
        u = out
    else:
        u = np.empty((nrhs, model.nz, model.nx), np.complex128) if out is None else out
        fp = None
        if f is not None:
            fa = _np(f, np.complex128)
            fp = C.c_void_p(fa.ctypes.data)
        st = lib.helm_solve(model.handle, nrhs, _ptr_d(om), _ptr_i(sx) if sx is not None else None,
                            _ptr_i(sz) if sz is not None else None, fp, C.c_void_p(u.ctypes.data),
                            C.byref(o), stats)
    check(st, "helm_solve", allow=(_lib.HELM_OK, _lib.HELM_E_NOT_CONVERGED))
    return u, stats_list(stats, nrhs), st


def helm_apply(model: Model, omega, u, precision: int = _lib.HELM_PREC_FP64, y=None):
    """y = B u (Eq. 3) per right-hand side; complex128 for FP64 else complex64."""
    lib = model.lib
    om = _np(omega, np.float64).reshape(-1)
    nrhs = om.size
    if _is_cuda_tensor(u):
        if y is None:
            y = torch.empty_like(u)
        torch.cuda.synchronize()
        st = lib.helm_apply(model.handle, nrhs, _ptr_d(om), int(precision), C.c_void_p(u.data_ptr()),
                            C.c_void_p(y.data_ptr()), 1)
    else:
        dt = np.complex128 if precision == _lib.HELM_PREC_FP64 else np.complex64
        ua = _np(u, dt)
        y = np.empty_like(ua)
        st = lib.helm_apply(model.handle, nrhs, _ptr_d(om), int(precision), C.c_void_p(ua.ctypes.data),
                            C.c_void_p(y.ctypes.data), 0)
    check(st, "helm_apply")
    return y


def helm_vcycle(model: Model, omega, r, beta=(1.0, 0.5), omega_jacobi: float = 0.8, coarse=None):
    """One cycle z ~ M^{-1} r of the shifted-Laplace preconditioner, complex64.

    coarse=None calls helm_vcycle (the default coarse end); otherwise helm_vcycle_ex
    with opts.coarse = coarse (HELM_COARSE_AUTO or HELM_COARSE_TAIL)."""
    lib = model.lib
    om = _np(omega, np.float64).reshape(-1)
    nrhs = om.size
    dev = _is_cuda_tensor(r)
    if dev:
        z = torch.empty_like(r)
        torch.cuda.synchronize()
        rp, zp = C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr())
    else:
        ra = _np(r, np.complex64)
        z = np.empty_like(ra)
        rp, zp = C.c_void_p(ra.ctypes.data), C.c_void_p(z.ctypes.data)
    if coarse is None:
        st = lib.helm_vcycle(model.handle, nrhs, _ptr_d(om), float(beta[0]), float(beta[1]), float(omega_jacobi),
                             rp, zp, 1 if dev else 0)
    else:
        o = helm_default_opts(beta=beta, omega_jacobi=float(omega_jacobi), coarse=int(coarse),
                              device_ptrs=1 if dev else 0)
        st = lib.helm_vcycle_ex(model.handle, nrhs, _ptr_d(om), C.byref(o), rp, zp)
    check(st, "helm_vcycle")
    return z


def helm_vcycle_noalloc(model: Model, omega, r, z, beta=(1.0, 0.5), omega_jacobi: float = 0.8):
    """helm_vcycle on the library's fixed scratch array (no device allocation).

    r, z: contiguous complex64 CUDA tensors [nrhs][nz][nx]; z is written in place.
    For callers that must not allocate device memory; see include/helm.h.
    """
    om = _np(omega, np.float64).reshape(-1)
    torch.cuda.synchronize()
    st = model.lib.helm_vcycle_noalloc(model.handle, om.size, _ptr_d(om), float(beta[0]), float(beta[1]),
                                       float(omega_jacobi), C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()))
    check(st, "helm_vcycle_noalloc")
    return z


# ----------------------------------------------------------------- gradient
def _geometry(omegas, src, rec):
    om = _np(omegas, np.float64).reshape(-1)
    s = _np(src, np.int32).reshape(-1, 2)
    r = _np(rec, np.int32).reshape(-1, 2)
    return om, _np(s[:, 0], np.int32), _np(s[:, 1], np.int32), _np(r[:, 0], np.int32), _np(r[:, 1], np.int32)


def helm_adjoint_gradient(model: Model, omegas, src, rec, d_obs, lam: float, opts=None):
    """(J, grad [Pz][Px], d_cal [nf][ns][nrec], stats, status) for Eq. 4 / Eq. 7 (host arrays)."""
    lib = model.lib
    om, sx, sz, rx, rz = _geometry(omegas, src, rec)
    nf, ns, nr = om.size, sx.size, rx.size
    d = _np(d_obs, np.complex128).reshape(nf, ns, nr)
    o = _opts(opts, device_ptrs=0)
    J = C.c_double()
    g = np.empty((model.Pz, model.Px), np.float64)
    dcal = np.empty_like(d)
    stats = (_lib.helm_solve_stats * (2 * nf * ns))()
    st = lib.helm_adjoint_gradient(model.handle, nf, _ptr_d(om), ns, _ptr_i(sx), _ptr_i(sz), nr, _ptr_i(rx),
                                   _ptr_i(rz), C.c_void_p(d.ctypes.data), float(lam), C.byref(J), _ptr_d(g),
                                   C.c_void_p(dcal.ctypes.data), C.byref(o), stats)
    check(st, "helm_adjoint_gradient", allow=(_lib.HELM_OK, _lib.HELM_E_NOT_CONVERGED))
    return J.value, g, dcal, stats_list(stats, 2 * nf * ns), st


class FwiState:
    def __init__(self, lib, handle):
        self.lib, self.handle = lib, handle

    def close(self):
        if self.handle:
            self.lib.helm_fwi_state_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def helm_fwi_forward(model: Model, omegas, src, rec, d_obs, lam: float, opts=None):
    """Forward half: (J, d_cal, state, stats, status); the state keeps u on the device."""
    lib = model.lib
    om, sx, sz, rx, rz = _geometry(omegas, src, rec)
    nf, ns, nr = om.size, sx.size, rx.size
    d = _np(d_obs, np.complex128).reshape(nf, ns, nr)
    o = _opts(opts, device_ptrs=0)
    J = C.c_double()
    dcal = np.empty_like(d)
    stats = (_lib.helm_solve_stats * (nf * ns))()
    h = C.c_void_p()
    st = lib.helm_fwi_forward(model.handle, nf, _ptr_d(om), ns, _ptr_i(sx), _ptr_i(sz), nr, _ptr_i(rx), _ptr_i(rz),
                              C.c_void_p(d.ctypes.data), float(lam), C.byref(J), C.c_void_p(dcal.ctypes.data),
                              C.byref(o), stats, C.byref(h))
    check(st, "helm_fwi_forward", allow=(_lib.HELM_OK, _lib.HELM_E_NOT_CONVERGED))
    return J.value, dcal, FwiState(lib, h), stats_list(stats, nf * ns), st


def helm_fwi_backward(model: Model, state: FwiState, opts=None, grad_out=None):
    """Adjoint half: the gradient [Pz][Px] float64 (NumPy, or into a CUDA tensor)."""
    lib = model.lib
    dev = _is_cuda_tensor(grad_out)
    o = _opts(opts, device_ptrs=1 if dev else 0)
    if dev:
        torch.cuda.synchronize()
        gp = C.cast(C.c_void_p(grad_out.data_ptr()), C.POINTER(C.c_double))
        g = grad_out
    else:
        g = np.empty((model.Pz, model.Px), np.float64)
        gp = _ptr_d(g)
    st = lib.helm_fwi_backward(state.handle, gp, C.byref(o), None)
    check(st, "helm_fwi_backward", allow=(_lib.HELM_OK, _lib.HELM_E_NOT_CONVERGED))
    return g, st


def helm_gn_hvp(model: Model, state: FwiState, dm, opts=None):
    """Gauss-Newton Hessian-vector product (Eq. 8 without its second term):
    (H dm [Pz][Px] float64, status)."""
    lib = model.lib
    x = _np(dm, np.float64).reshape(model.Pz, model.Px)
    out = np.empty_like(x)
    o = _opts(opts, device_ptrs=0)
    st = lib.helm_gn_hvp(state.handle, C.c_void_p(x.ctypes.data), C.c_void_p(out.ctypes.data), C.byref(o), None)
    check(st, "helm_gn_hvp", allow=(_lib.HELM_OK, _lib.HELM_E_NOT_CONVERGED))
    return out, st


def helm_gn_step(model: Model, state: FwiState, grad, cg_iters: int, opts=None):
    """One Gauss-Newton step (Eq. 9) by cg_iters CG iterations from zero:
    (dm [Pz][Px] float64, relative CG residuals [cg_iters + 1], status)."""
    lib = model.lib
    g = _np(grad, np.float64).reshape(model.Pz, model.Px)
    dm = np.empty_like(g)
    rel = np.empty(int(cg_iters) + 1, np.float64)
    o = _opts(opts, device_ptrs=0)
    st = lib.helm_gn_step(state.handle, C.c_void_p(g.ctypes.data), int(cg_iters), C.c_void_p(dm.ctypes.data),
                          _ptr_d(rel), C.byref(o))
    check(st, "helm_gn_step", allow=(_lib.HELM_OK, _lib.HELM_E_NOT_CONVERGED))
    return dm, rel, st


def helm_fwi_run(ctx: Context, m0, h: float, omegas, src, rec, d_obs, lam: float, strategy="sequential",
                 gn_iters=2, cg_iters=5, max_halvings=4, m_bounds=(1 / 6000.0, 1 / 1000.0), npml=20,
                 alpha_max=0.5, opts=None, checkpoint=None):
    """Gauss-Newton FWI loop over frequency groups ("simultaneous": all at once;
    "sequential": one at a time from the lowest). Returns (m [Pz][Px], J history,
    status); `checkpoint(group, iter, m, J)` is called with a copy of every
    accepted model."""
    lib = ctx.lib
    m = _np(m0, np.float64)
    Pz, Px = m.shape
    om, sx, sz, rx, rz = _geometry(omegas, src, rec)
    nf, ns, nr = om.size, sx.size, rx.size
    d = _np(d_obs, np.complex128).reshape(nf, ns, nr)
    fo = _lib.helm_fwi_opts(_lib.HELM_FWI_SEQUENTIAL if strategy == "sequential" else _lib.HELM_FWI_SIMULTANEOUS,
                            int(gn_iters), int(cg_iters), int(max_halvings), float(m_bounds[0]), float(m_bounds[1]))
    o = _opts(opts, device_ptrs=0)
    ngroups = nf if strategy == "sequential" else 1
    hist = np.zeros(ngroups * (int(gn_iters) + 1), np.float64)
    nh = C.c_int()
    out = np.empty_like(m)

    def _cb(group, it, mp, J, _user):
        checkpoint(group, it, np.ctypeslib.as_array(mp, shape=(Pz, Px)).copy(), J)

    cb = _lib.helm_fwi_checkpoint(_cb) if checkpoint else _lib.helm_fwi_checkpoint()
    st = lib.helm_fwi_run(ctx.handle, Px, Pz, float(h), int(npml), float(alpha_max), _ptr_d(m), nf, _ptr_d(om), ns,
                          _ptr_i(sx), _ptr_i(sz), nr, _ptr_i(rx), _ptr_i(rz), C.c_void_p(d.ctypes.data), float(lam),
                          C.byref(fo), C.byref(o), _ptr_d(out), _ptr_d(hist), C.byref(nh), cb, None)
    check(st, "helm_fwi_run", allow=(_lib.HELM_OK, _lib.HELM_E_NOT_CONVERGED))
    return out, hist[: nh.value].copy(), st


# ------------------------------------------------------------------ serving
@dataclass
class ServedResult:
    u: np.ndarray
    status: int
    stats: dict
    latency_ms: float
    queue_ms: float
    batch_size: int


def helm_serve_config(ctx: Context, max_batch=32, max_slots=4, reserve_bytes=512 << 20, budget_bytes=0):
    check(ctx.lib.helm_serve_config(ctx.handle, int(max_batch), int(max_slots), int(reserve_bytes),
                                    int(budget_bytes)), "helm_serve_config")


def helm_submit(ctx: Context, slowness, h, omega, src, npml=20, alpha_max=0.5, opts=None) -> int:
    m = _np(slowness, np.float64)
    req = _lib.helm_request()
    req.Pz, req.Px = m.shape
    req.h = float(h)
    req.slowness = _ptr_d(m)
    req.npml = int(npml)
    req.alpha_max = float(alpha_max)
    req.omega = float(omega)
    req.src_ix, req.src_iz = int(src[0]), int(src[1])
    req.opts = _opts(opts, device_ptrs=0)
    t = C.c_uint64()
    check(ctx.lib.helm_submit(ctx.handle, C.byref(req), C.byref(t)), "helm_submit")
    return t.value


def helm_poll(ctx: Context, ticket: int, timeout_ms: int = -1, copy_u: bool = True):
    """ServedResult when done (the field array is copied out unless copy_u is False), None if
    still pending."""
    res = _lib.helm_result()
    st = ctx.lib.helm_poll(ctx.handle, C.c_uint64(ticket), int(timeout_ms), C.byref(res))
    if st in (_lib.HELM_PENDING, _lib.HELM_E_TIMEOUT):
        return None
    check(st, "helm_poll")
    u = None
    if res.u and copy_u:
        n = res.nx * res.nz
        buf = (C.c_double * (2 * n)).from_address(res.u)
        u = np.frombuffer(buf, dtype=np.complex128, count=n).reshape(res.nz, res.nx).copy()
    s = res.stats
    return ServedResult(u, res.status, dict(iters=s.iters, outer_its=s.outer_its, converged=bool(s.converged),
                                            relres=s.relres, dense_level=s.dense_level,
                                            shift_switched=bool(s.shift_switched)), res.latency_ms, res.queue_ms, res.batch_size)


def helm_release(ctx: Context, ticket: int) -> int:
    return check(ctx.lib.helm_release(ctx.handle, C.c_uint64(ticket)), "helm_release",
                 allow=(_lib.HELM_OK, _lib.HELM_PENDING))
