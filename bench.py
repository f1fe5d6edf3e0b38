#!/usr/bin/env python
"""Benchmark: shifted-Laplace-preconditioned Helmholtz solves on one GB300.

Workload (one step): one forward solve of the single large case - 1001 x 1001
physical nodes (1041 x 1041 with the 20-node damping layer, 1.08M unknowns),
h = 5 m, 15 Hz, 12 random layers + 3 Gaussian anomalies (seed 2), surface point
source - by flexible GMRES(10) right-preconditioned with one shifted-Laplace
multigrid cycle in complex64 and FP64 true-residual refinement to relative
residual 1e-6 (BiCGSTAB is timed beside it).

Prints one JSON line: solves/s (device-resident inputs), the same through host
buffers (e2e), p50/p99 step latency, the plain FP64 GPU solve of the same
problem, the roofline of the dominant kernel, clocks, and the CPU oracle as
`cpu_baseline`. ``--impl reference`` times the CPU oracle alone.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one independent solve per rank per step (weak scaling,
no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "single_large_1001x1001_h5m_15Hz_layered12_anom3_seed2_mixed_tol1e-6"
L2_BYTES = 129 * 2 ** 20
REORTH = {"always": 0, "never": 1, "ifneeded": 2}        # helm_reorth
GS_NAME = {"always": "CGS2", "never": "CGS", "ifneeded": "CGS + DGKS second pass"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-alt", action="store_true", help="skip the other Krylov method's leg of the single-case line")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the batched and Gauss-Newton legs of the single-case line")
    ap.add_argument("--krylov", default=None, choices=["bicgstab", "fgmres"],
                    help="Krylov method (default: FGMRES(10) for the single case, the paper's engine, with "
                         "BiCGSTAB timed beside it; BiCGSTAB for the batched and ablation workloads)")
    ap.add_argument("--restart", type=int, default=10, help="FGMRES restart length")
    ap.add_argument("--reorth", default="never", choices=["always", "never", "ifneeded"],
                    help="FGMRES Gram-Schmidt: second pass always (CGS2), never, or by the DGKS test")
    ap.add_argument("--inner-tol", type=float, default=5e-2, help="mixed precision: reduction per inner solve")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the autotuner (default: the multigrid tile shapes are chosen by helm_autotune for "
                         "the workload's grid and batch size before timing; the choice is cached per shape)")
    ap.add_argument("--coarse", default="auto", choices=["auto", "dense", "fused", "tail"],
                    help="coarse end of the multigrid cycle (helm_coarse) of the single-case solves")
    ap.add_argument("--density", action="store_true",
                    help="single: the variable-density operator (Eq. 1) with a Gardner density on the same model")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "serving", "gn", "ablation", "fwi"],
                    help="single: the single large case (the default line); batched: 64 shots x 5 "
                         "frequencies in one call; serving: a Poisson stream of requests; gn: one "
                         "Gauss-Newton iteration of the gradient case; ablation: preconditioner on/off")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time only the hot kernels alone (the roofline legs), print one line per kernel")
    ap.add_argument("--requests", type=int, default=48, help="serving: number of requests per stream")
    ap.add_argument("--rates", default="0.8", help="serving: arrival rates as fractions of the saturated throughput")
    ap.add_argument("--sat-requests", type=int, default=200,
                    help="serving: requests of the saturated-throughput run (all queued at once)")
    ap.add_argument("--seq-requests", type=int, default=16,
                    help="serving: requests solved one after another in plain FP64 for the baseline")
    ap.add_argument("--serve-beta2", type=float, default=None,
                    help="serving: imaginary shift beta2 of the preconditioner (default: the library's (1, 0.5), "
                         "whose stall guard switches a stalled solve to the paper's (1, 1))")
    ap.add_argument("--serve-sizes", default="128,256,512,1024",
                    help="serving: physical grid sizes N (N x N) the requests draw from")
    ap.add_argument("--cg", type=int, default=5, help="gn, fwi: conjugate-gradient iterations per Gauss-Newton step")
    ap.add_argument("--gn", type=int, default=2, help="fwi: Gauss-Newton iterations per frequency group")
    ap.add_argument("--fwi-strategy", default="sequential", choices=["sequential", "simultaneous"])
    ap.add_argument("--rate", type=float, default=0.0, help="serving: arrivals per second (0: 0.8 x measured)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# ------------------------------------------------------------ CPU oracle arm
def oracle_c2_timing(nsolves: int, want_field: bool = False):
    """Sparse-LU oracle on the same problem: assembly and factorisation once
    (timed together from the padded model), then nsolves triangular solves of
    the point-source right-hand side. Returns (setup seconds, [solve seconds]),
    and the oracle wavefield [1][nz][nx] as a third item when want_field."""
    import oracle
    from synth import models

    mdl = models.c2_model()
    t0 = time.perf_counter()
    m_pad = oracle.pad_slowness(mdl.slowness, mdl.npml)
    alpha = oracle.damping_profile(mdl.Px, mdl.Pz, mdl.npml, mdl.alpha_max)
    fac = oracle.Factorised(m_pad, mdl.h, mdl.omegas[0], alpha)
    t_fac = time.perf_counter() - t0
    F = oracle.point_sources(m_pad.shape[1], m_pad.shape[0], mdl.h, mdl.sources + mdl.npml)
    ts = []
    U = None
    for _ in range(nsolves):
        t0 = time.perf_counter()
        U = fac.solve(F)
        ts.append(time.perf_counter() - t0)
    return (t_fac, ts, U) if want_field else (t_fac, ts)


def oracle_c2_full_solve() -> tuple[float, float]:
    """One complete oracle solve of the single large case, as one step of our
    arm is one complete solve: assemble and factorise B(omega), then solve.
    Returns (seconds, of which factorisation)."""
    t_fac, ts = oracle_c2_timing(1)
    return t_fac + ts[0], t_fac


def run_reference(args):
    """The CPU oracle on the bench workload. Each timed step is one complete
    solve (operator assembly, SuperLU factorisation, triangular solve): our arm
    solves a new right-hand side of a new operator from scratch each step, and
    a direct solver pays its factorisation per (model, frequency). Warm-up steps
    run the same code on the small 101 x 101 case (the oracle has no state that
    a warm-up of the large case would prepare), which keeps the run within a
    few minutes: each timed step takes about 22 s on one Grace core."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from synth import models

    small = models.c1_model()
    for _ in range(max(args.warmup, 0)):
        oracle.solve_fields(small.slowness, small.h, small.omegas[0], small.sources, small.npml, small.alpha_max)
    steps = max(args.steps, 1)
    full, fac = [], []
    for _ in range(steps):
        t, tf = oracle_c2_full_solve()
        full.append(t)
        fac.append(tf)
    t_step = float(np.mean(full))
    value = 1.0 / t_step
    line = {
        "impl": "reference", "metric": "helmholtz_solves_per_s", "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solver": "CPU oracle: SuperLU sparse LU (complex128)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "per step one complete solve of the same problem (operator assembly, SuperLU "
                                   "factorisation, triangular solve of the point source); SuperLU runs "
                                   "single-threaded; warm-up steps solve the 101 x 101 case",
                         "factor_s": float(np.mean(fac)), "solve_only_s": t_step - float(np.mean(fac))},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
KERNELS = (("fg_axpy", "HELM_KERNEL_FG_AXPY"), ("fg_dots", "HELM_KERNEL_FG_DOTS"),
           ("bicg_xr", "HELM_KERNEL_BICG_XR"), ("prolong_fine", "HELM_KERNEL_PROLONG"),
           ("restrict_fine", "HELM_KERNEL_RESTRICT"), ("stencil_apply", "HELM_KERNEL_APPLY"),
           ("bicg_p", "HELM_KERNEL_BICG_P"), ("resid64", "HELM_KERNEL_RESID64"), ("tail", "HELM_KERNEL_TAIL"))


def time_kernels(lib, api, _lib, model, omega, reps=20):
    """Each hot kernel timed alone (CUDA events on the library's stream, inside
    helm_time_kernel) on a batch large enough that one launch moves more than
    three times the L2 size, so consecutive launches cannot run from L2."""
    out = {}
    for name, kid_name in KERNELS:
        kid = getattr(_lib, kid_name)
        tms, byt = api.C.c_double(), api.C.c_double()
        # bytes of one right-hand side first (one launch of a single-RHS batch)
        api.check(lib.helm_time_kernel(model.handle, kid, 1, omega, 1, api.C.byref(tms), api.C.byref(byt)),
                  "helm_time_kernel")
        nb = int(min(64, max(8, -(-3 * L2_BYTES // int(byt.value)))))
        if name == "tail":
            nb = 1   # one block on one SM, bound by its chain of dependent steps: the solve's case
        api.check(lib.helm_time_kernel(model.handle, kid, nb, omega, reps, api.C.byref(tms), api.C.byref(byt)),
                  "helm_time_kernel")
        if name == "tail":   # one block per right-hand side: a latency, not a bandwidth
            out[name] = {"ms": tms.value, "nrhs": nb, "bound": "latency (one block on one SM)"}
            continue
        out[name] = {"ms": tms.value, "bytes": byt.value, "gbs": byt.value / tms.value / 1e6, "nrhs": nb}
    # FP64 peak measured here (independent fused multiply-add chains) and the FP64 residual's rate
    # against it. Algorithmic FP64 operations per node and right-hand side of r = f - A u and
    # ||r||^2: scale s = (h w)^2 m^2 1, real diagonal 4 - s 1, diagonal times u 2, the four
    # neighbours 6, residual 4, ||r||^2 3 = 17; nodes in the absorbing layer add the damping
    # term i s alpha u (alpha 1, s alpha 1, two products 2, two additions 2 = 6). ||f||^2 is formed
    # only on a solve's first call, not in this timed one.
    api.check(lib.helm_time_kernel(model.handle, _lib.HELM_KERNEL_FMA64, 1, omega, reps, api.C.byref(tms),
                                   api.C.byref(byt)), "helm_time_kernel")
    peak64 = byt.value / tms.value / 1e9
    out["fma64"] = {"ms": tms.value, "flops": byt.value, "tflops": peak64, "bound": "fp64 alu"}
    r = out["resid64"]
    p = model.npml
    n_layer = model.nx * model.nz - max(model.nx - 2 * p, 0) * max(model.nz - 2 * p, 0)
    flops = (17.0 * model.nx * model.nz + 6.0 * n_layer) * r["nrhs"]
    r["fp64_flops_per_launch"] = flops
    r["fp64_tflops"] = flops / r["ms"] / 1e9
    r["fp64_frac"] = r["fp64_tflops"] / peak64
    return out


def profile_solve(lib, _lib, step_fn):
    """One solve of the bench workload with every launch of the library timed by
    CUDA events on its stream (helm_profile_begin/end, no graphs, launches
    serialised); returns per-kernel totals summed over the grids each ran on."""
    import ctypes as C

    lib.helm_profile_begin()
    step_fn()
    cap = 512
    buf = (_lib.helm_profile_entry * cap)()
    n = C.c_int()
    lib.helm_profile_end(buf, cap, C.byref(n))
    per = {}
    grids = []
    for e in buf[: min(n.value, cap)]:
        name = e.name.decode()
        d = per.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0})
        d["launches"] += int(e.launches)
        d["ms"] += e.ms
        d["bytes"] += e.bytes
        grids.append({"kernel": name, "grid": f"{e.nx}x{e.nz}", "launches": int(e.launches), "ms": e.ms,
                      "bytes": e.bytes})
    return per, grids


def traffic_for(kernel: str, grids):
    """DRAM bytes per launch of `kernel` in the profiled solve: the committed ncu summary
    of its launches, per level grid, weighted by the solve's own launches on each grid,
    when the summary was taken of the kernel's current sources (else None)."""
    import hashlib

    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        tr = json.load(f)
    e = tr.get(kernel)
    if not isinstance(e, dict) or "by_grid" not in e:
        return None
    for fn, sha in e.get("src_sha1", {}).items():
        src = os.path.join(ROOT, "paper_1712_08743_gb300", "csrc", fn)
        if not os.path.exists(src):
            return None
        with open(src, "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != sha:
                return None
    mine = [g for g in grids if g["kernel"] == kernel]
    if not mine or any(g["grid"] not in e["by_grid"] for g in mine):
        return None
    n = sum(g["launches"] for g in mine)
    return sum(g["launches"] * e["by_grid"][g["grid"]] for g in mine) / n


def run_kernels_only(args):
    import torch

    from paper_1712_08743_gb300 import _lib, api, build
    from synth import models

    build.build()
    lib = _lib.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = api.Context(0, stream)
    mdl = models.c2_model()
    model = api.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    peak, kind = measured_peaks()
    for name, k in time_kernels(lib, api, _lib, model, float(mdl.omegas[0]), reps=max(args.steps, 1)).items():
        print(json.dumps({"kernel": name, "workload": WORKLOAD, **k, "frac": k["gbs"] / peak if "gbs" in k else None,
                          "peak": peak, "peak_kind": kind}), flush=True)
    model.close()
    ctx.close()


def batched_leg(api, _lib, ctx, stream, steps: int, tune: bool = True, inner_tol: float = 1e-2,
                krylov: str = "bicgstab"):
    """64 surface shots x 5 frequencies (3..7 Hz) on the 401 x 201 layered model with a dipping
    interface, 320 right-hand sides in one helm_solve, mixed precision to relres 1e-6, the tiles
    of the multigrid kernels chosen by the autotuner first. Timed with CUDA events on the
    library's stream, one warm-up batch."""
    import torch

    from synth import models

    mdl = models.c3_model()
    model = api.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    om = np.repeat(mdl.omegas, len(mdl.sources))
    src = np.tile(mdl.sources, (len(mdl.omegas), 1))
    kry = {"bicgstab": _lib.HELM_KRYLOV_BICGSTAB, "fgmres": _lib.HELM_KRYLOV_FGMRES}[krylov]
    opts = api.helm_default_opts(tol=1e-6, precision="mixed", krylov=kry, inner_tol=inner_tol)
    tiles = None
    if tune:
        from paper_1712_08743_gb300 import autotune
        tiles = autotune.autotune(model, len(om), float(om[0]))
    F = np.zeros((len(om), model.nz, model.nx), np.complex128)
    for k, (sx, sz) in enumerate(src):
        F[k, sz + mdl.npml, sx + mdl.npml] = 1.0 / mdl.h ** 2
    f_dev = torch.from_numpy(F).cuda()
    u_dev = torch.empty_like(f_dev)
    api.helm_solve(model, om, f=f_dev, opts=opts, out=u_dev)
    ms = []
    st = None
    for _ in range(max(steps, 1)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, st, _ = api.helm_solve(model, om, f=f_dev, opts=opts, out=u_dev)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    model.close()
    its = [x["iters"] for x in st]
    return {"workload": "batched_401x201_64src_5f_tol1e-6", "solves_per_s": len(om) * 1e3 / float(np.mean(ms)),
            "ms_per_batch": float(np.mean(ms)), "nrhs": len(om), "krylov": krylov, "inner_tol": inner_tol,
            "iters_min": min(its), "iters_max": max(its), "converged": all(x["converged"] for x in st),
            "autotuned_tiles": tiles, "steps": len(ms)}


def observed_data(api, ctx, true):
    """Observed data of the gradient case: the library's modelled data P u of the true model at
    every frequency and shot (the paper likewise makes its data with the same discretisation)."""
    om = true.omegas
    mt = api.helm_create_model(ctx, true.slowness, true.h, true.npml, true.alpha_max)
    zero = np.zeros((len(om), len(true.sources), len(true.receivers)), np.complex128)
    _, d_obs, st0, _, _ = api.helm_fwi_forward(mt, om, true.sources, true.receivers, zero, 0.0,
                                               dict(tol=1e-10, precision="mixed"))
    st0.close()
    mt.close()
    return d_obs


def gn_leg(api, ctx, steps: int, cg: int = 5):
    """One Gauss-Newton iteration (Eq. 9) of the gradient case: 401 x 201 smoothed start model,
    32 shots x 4 frequencies (3..6 Hz), 201 receivers, lambda = 1e-3: forward solves and misfit,
    adjoint solves and gradient, then `cg` CG iterations (a Born and an adjoint solve per shot
    and frequency each). The observed data are the library's own modelled data of the true
    model. Wall time per iteration (each call synchronises), one warm-up iteration."""
    from synth import models

    true, start = models.c4_models()
    om = true.omegas
    opts = dict(tol=1e-6, precision="mixed")
    lam = 1e-3
    d_obs = observed_data(api, ctx, true)
    model = api.helm_create_model(ctx, start.slowness, start.h, start.npml, start.alpha_max)

    def iteration():
        t0 = time.perf_counter()
        J, _, state, _, _ = api.helm_fwi_forward(model, om, start.sources, start.receivers, d_obs, lam, opts)
        t1 = time.perf_counter()
        g, _ = api.helm_fwi_backward(model, state, opts)
        t2 = time.perf_counter()
        dm, rel, _ = api.helm_gn_step(model, state, g, cg, opts)
        t3 = time.perf_counter()
        state.close()
        return J, rel, (t1 - t0, t2 - t1, t3 - t2)

    iteration()
    times = []
    J = rel = None
    for _ in range(max(steps, 1)):
        J, rel, t = iteration()
        times.append(t)
    model.close()
    tf, tb, tg = (float(np.mean([t[k] for t in times])) for k in range(3))
    nrhs = len(om) * len(start.sources)
    solves = nrhs * (2 + 2 * cg)
    return {"workload": "gradient_401x201_32shots_4f_gn", "iters_per_s": 1.0 / (tf + tb + tg), "cg_iters": cg,
            "solves_per_iteration": solves, "solves_per_s": solves / (tf + tb + tg), "forward_s": tf,
            "gradient_s": tb, "cg_s": tg, "misfit": J, "cg_relres": [float(x) for x in rel], "steps": len(times)}


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1712_08743_gb300 import _lib, api, build, shard
    from synth import models

    build.build()
    lib = _lib.load()
    stream = torch.cuda.Stream()             # the library launches on this stream; events are recorded on it
    torch.cuda.set_stream(stream)
    ctx = api.Context(local, stream)
    mdl = models.c2_model()
    # --density: the variable-density operator of Eq. 1 on the same model, density by Gardner's relation
    rho = models.gardner_density(mdl.velocity) if args.density else None
    model = api.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max, density=rho)
    n = model.n
    om = mdl.omegas
    kry = {"bicgstab": _lib.HELM_KRYLOV_BICGSTAB, "fgmres": _lib.HELM_KRYLOV_FGMRES}[args.krylov]
    ro = REORTH[args.reorth]
    coarse = {"auto": _lib.HELM_COARSE_AUTO, "dense": _lib.HELM_COARSE_DENSE, "fused": _lib.HELM_COARSE_FUSED,
              "tail": _lib.HELM_COARSE_TAIL}[args.coarse]
    opts = api.helm_default_opts(tol=1e-6, precision="mixed", krylov=kry, restart=args.restart,
                                 inner_tol=args.inner_tol, max_it=20000, reorth=ro, coarse=coarse)
    tiles = None
    if args.tune:
        from paper_1712_08743_gb300 import autotune
        tiles = autotune.autotune(model, 1, float(om[0]))
    # device-resident input (point source, grid-scaled form is built by the library from f)
    f_host = np.zeros((1, model.nz, model.nx), np.complex128)
    sx, sz = mdl.sources[0]
    f_host[0, sz + mdl.npml, sx + mdl.npml] = 1.0 / mdl.h ** 2
    f_dev = torch.from_numpy(f_host).cuda()
    u_dev = torch.empty_like(f_dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    def step(o):
        return api.helm_solve(model, om, f=f_dev, opts=o, out=u_dev)

    for _ in range(max(args.warmup, 0)):
        step(opts)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats_all = []
    l0 = lib.helm_launch_count()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))            # L2 flush between timed steps, outside the events
            ev[k][0].record(stream)
            _, st, status = step(opts)
            ev[k][1].record(stream)
            stats_all.append(st[0])
        barrier()
    launches = lib.helm_launch_count() - l0
    clocks = clk.summary()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(ms) / 1e3
    t_total = shard.allreduce_max(t_total)     # max over ranks (no-op at N = 1)
    value = world * args.steps / t_total
    conv = all(s["converged"] for s in stats_all)

    # end to end through the public API with host buffers (pinned input, result read back)
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_host = np.empty_like(f_host)
    e2e_ms = []
    for k in range(max(1, min(args.steps, 3))):
        flush.fill_(0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.helm_solve(model, om, f=f_pin.numpy(), opts=opts, out=u_host)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = world * 1e3 / float(np.mean(e2e_ms))

    # plain FP64 GPU solve of the same problem (the baseline the precision split must beat)
    fp64 = None
    if not args.no_fp64:
        o64 = api.helm_default_opts(tol=1e-6, precision="fp64", krylov=kry, restart=args.restart, max_it=20000,
                                    reorth=ro, coarse=coarse)
        step(o64)
        t64 = []
        its64 = None
        for k in range(max(1, min(args.steps, 2))):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, st64, _ = step(o64)
            b.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(b))
            its64 = st64[0]["iters"]
        fp64 = {"solves_per_s": 1e3 / float(np.mean(t64)), "ms": float(np.mean(t64)), "iters": its64}

    # the other Krylov method on the same problem and timing rules: BiCGSTAB beside
    # the FGMRES headline (the paper's engine), or FGMRES(10) beside BiCGSTAB
    alt = None
    if not args.no_alt:
        if args.krylov == "fgmres":
            oalt = api.helm_default_opts(tol=1e-6, precision="mixed", krylov=_lib.HELM_KRYLOV_BICGSTAB,
                                         inner_tol=args.inner_tol, coarse=coarse)
            alt_name = f"BiCGSTAB (inner reduction {args.inner_tol:g})"
        else:
            oalt = api.helm_default_opts(tol=1e-6, precision="mixed", krylov=_lib.HELM_KRYLOV_FGMRES, restart=10,
                                         max_it=20000, reorth=ro)
            alt_name = f"FGMRES(10, {GS_NAME[args.reorth]})"
        step(oalt)
        talt = []
        stalt = None
        for k in range(max(1, min(args.steps, 3))):
            flush.fill_(2.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, stalt, _ = step(oalt)
            b.record(stream)
            torch.cuda.synchronize()
            talt.append(a.elapsed_time(b))
        alt = {"krylov": alt_name, "solves_per_s": 1e3 / float(np.mean(talt)), "ms": float(np.mean(talt)),
               "iters": stalt[0]["iters"], "relres": stalt[0]["relres"], "converged": bool(stalt[0]["converged"])}

    # roofline: per-kernel times of one solve of this workload, measured here with CUDA events
    # around every launch (helm_profile_*: serialised launches, so shares are the figure), the
    # dominant kernel by its share of the solve, and each hot kernel timed alone on inputs > L2
    peak, peak_kind = measured_peaks()
    per, grids = profile_solve(lib, _lib, lambda: step(opts))
    total_ms = sum(d["ms"] for d in per.values())
    total_bytes = sum(d["bytes"] for d in per.values())
    dom = max(per, key=lambda k: per[k]["ms"])
    achieved = per[dom]["bytes"] / (per[dom]["ms"] * 1e-3) / 1e9
    kern = time_kernels(lib, api, _lib, model, float(om[0]))
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic_for(dom, grids),
            "peak_kind": f"{peak_kind} burst copy",
            "bytes_per_launch": per[dom]["bytes"] / per[dom]["launches"],
            "ms_per_launch": per[dom]["ms"] / per[dom]["launches"], "launches": per[dom]["launches"],
            "share": per[dom]["ms"] / total_ms,
            "how": "one solve of this workload with a CUDA event pair around every launch (helm_profile_*; "
                   "no graphs, launches serialised); achieved = the kernel's summed algorithmic bytes / summed "
                   "event time",
            # the whole solve: algorithmic bytes of every launch over the timed step time
            "solve_frac": total_bytes / (t_total / args.steps) / 1e9 / peak,
            "solve_bytes": total_bytes,
            "shares": {k: {"share": d["ms"] / total_ms, "launches": d["launches"],
                           "gbs": d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else None}
                       for k, d in sorted(per.items(), key=lambda kv: -kv[1]["ms"])},
            "profiled_ms": total_ms, "kernels_alone": kern}

    # the batched and Gauss-Newton configurations, each timed on its own (not part of `value`)
    legs = {}
    if not args.no_legs and not args.density:
        legs["batched"] = batched_leg(api, _lib, ctx, stream, steps=3)
        legs["gauss_newton"] = gn_leg(api, ctx, steps=2)

    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.density:
        t_fac, ts, U = oracle_c2_timing(1, want_field=True)
        U = np.asarray(U).reshape(u_host.shape)
        cpu = {"value": 1.0 / (t_fac + ts[0]), "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": "one full solve of the same problem: SuperLU factorisation + triangular solve "
                         "(single-threaded)", "factor_s": t_fac, "solve_s": ts[0]}
        # each result's error against the FP64 oracle: the timed configuration's wavefield (the e2e
        # leg's output, the same solve) and a complex64-only solve of the same problem
        p = slice(mdl.npml, -mdl.npml)

        def rel(a, b):
            return float(np.linalg.norm(a - b) / np.linalg.norm(b))

        # complex64 only: one BiCGSTAB solve with no FP64 refinement (FGMRES restarts through the
        # FP64 residual, so it has no complex64-only mode)
        o32 = api.helm_default_opts(tol=1e-6, precision="fp32", krylov=_lib.HELM_KRYLOV_BICGSTAB, max_it=20000)
        u32, st32, status32 = api.helm_solve(model, om, f=f_host, opts=o32)
        err = {"rel_l2": rel(u_host, U), "rel_l2_physical": rel(u_host[0][p, p], U[0][p, p]),
               "complex64_only": {"krylov": "BiCGSTAB", "rel_l2": rel(u32, U), "relres": st32[0]["relres"], "iters": st32[0]["iters"],
                                  "converged": bool(st32[0]["converged"]), "bar": 1e-4},
               "note": "the timed solve stops at relres 1e-6, so its error is about cond(B) x 1e-6; the parity "
                       "tests solve to 1e-10 and meet 1e-6"}

    if rank == 0:
        line = {
            "metric": "helmholtz_solves_per_s", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + ("_gardner_density" if args.density else ""), "grid": f"{model.nx}x{model.nz} padded ({mdl.Px}x{mdl.Pz} physical)",
                       "unknowns": n, "precision": "complex64 inner, FP64 residual/refinement",
                       "krylov": ("BiCGSTAB" if args.krylov == "bicgstab" else
                                  f"FGMRES({args.restart}, {GS_NAME[args.reorth]})") +
                                 " + shifted-Laplace Galerkin MG (V-cycle above the first level where k h of the "
                                 "shortest wavelength reaches 0.7, F-cycle from there; the first level with at most "
                                 "1200 nodes solved by its dense inverse), beta=(1,0.5)",
                       "inner_tol": args.inner_tol, "restart": args.restart if args.krylov == "fgmres" else None,
                       "coarse": args.coarse,
                       "tiles": {"restrict": tiles[:model.nlevels], "prolong": tiles[24:24 + model.nlevels],
                                 "by": "helm_autotune at 1 right-hand side"} if tiles else "library defaults",
                       "levels": model.nlevels, "l2": "flushed between timed steps (258 MB write)",
                       "parallelism": f"replicas x{world}"},
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "iters": stats_all[-1]["iters"], "outer_its": stats_all[-1]["outer_its"],
            "dense_level": stats_all[-1]["dense_level"],
            "relres": stats_all[-1]["relres"], "converged": conv,
            "fp64_plain": fp64, "other_krylov": alt,
            "speedup_vs_fp64": (value / world) / fp64["solves_per_s"] if fp64 else None,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(f_host.nbytes),
                    "d2h_bytes_per_step": int(u_host.nbytes), "ms": float(np.mean(e2e_ms))},
            "roofline": roof, "clocks": clocks, "gpu_launches": int(launches), "cpu_baseline": cpu,
            "err_vs_oracle": err,
            "batched_solves_per_s": legs["batched"]["solves_per_s"] if "batched" in legs else None,
            "gn_iters_per_s": legs["gauss_newton"]["iters_per_s"] if "gauss_newton" in legs else None,
            "legs": legs,
        }
        print(json.dumps(line), flush=True)
    model.close()
    ctx.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_batched(args):
    """64 shots x 5 frequencies (3..7 Hz) on the 401 x 201 layered model, one call (--tune: autotuned tiles)."""
    import torch

    from paper_1712_08743_gb300 import _lib, api, build

    build.build()
    _lib.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = api.Context(0, stream)
    r = batched_leg(api, _lib, ctx, stream, steps=args.steps, tune=args.tune, inner_tol=args.inner_tol,
                    krylov=args.krylov)
    print(json.dumps({"metric": "helmholtz_solves_per_s", "value": r["solves_per_s"], "unit": "solves/s", **r}),
          flush=True)
    ctx.close()


def run_gn(args):
    """One Gauss-Newton iteration of the gradient case (see gn_leg)."""
    import torch

    from paper_1712_08743_gb300 import _lib, api, build

    build.build()
    _lib.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = api.Context(0, stream)
    r = gn_leg(api, ctx, steps=args.steps, cg=args.cg)
    print(json.dumps({"metric": "gauss_newton_iterations_per_s", "value": r["iters_per_s"], "unit": "iterations/s",
                      **r}), flush=True)
    ctx.close()


def run_fwi(args):
    """The Gauss-Newton inversion loop on the gradient case (401 x 201, 32 shots,
    201 receivers, 3..6 Hz, lambda = 1e-3, smoothed start): `--fwi-strategy`
    sequential (one frequency at a time from the lowest, as in the paper's 2D
    example) or simultaneous (all at once, as in its 1D example), `--gn` Gauss-Newton
    iterations per group of `--cg` CG iterations each, with backtracking. Reports
    accepted iterations per second, the misfit history and the model error."""
    import torch

    from paper_1712_08743_gb300 import _lib, api, build
    from synth import models

    build.build()
    _lib.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = api.Context(0, stream)
    true, start = models.c4_models()
    om = true.omegas
    d_obs = observed_data(api, ctx, true)
    opts = dict(tol=1e-6, precision="mixed")
    lam = 1e-3
    bounds = (1 / 4500.0, 1 / 1400.0)

    def run(strategy, gn):
        t0 = time.perf_counter()
        m, hist, st = api.helm_fwi_run(ctx, start.slowness, start.h, om, start.sources, start.receivers, d_obs, lam,
                                       strategy=strategy, gn_iters=gn, cg_iters=args.cg, max_halvings=4,
                                       m_bounds=bounds, npml=start.npml, alpha_max=start.alpha_max, opts=opts)
        return m, hist, st, time.perf_counter() - t0

    for _ in range(max(args.warmup, 0)):
        run("simultaneous", 1)
    results = [run(args.fwi_strategy, args.gn) for _ in range(max(args.steps, 1))]
    m, hist, st, _ = results[-1]
    wall = float(np.mean([r[3] for r in results]))
    ngroups = len(om) if args.fwi_strategy == "sequential" else 1
    accepted = len(hist) - ngroups
    err0 = float(np.linalg.norm(start.slowness - true.slowness))
    print(json.dumps({"metric": "fwi_gauss_newton_iterations_per_s", "workload": "fwi_401x201_32shots_4f",
                      "strategy": args.fwi_strategy, "value": accepted / wall, "unit": "iterations/s",
                      "wall_s": wall, "accepted_iterations": accepted, "groups": ngroups, "gn_per_group": args.gn,
                      "cg_iters": args.cg, "misfit_history": [float(x) for x in hist],
                      "model_error_rel": float(np.linalg.norm(m - true.slowness)) / err0, "status": int(st)}),
          flush=True)
    ctx.close()


def run_ablation(args):
    """Preconditioner ablation on the batched case's model (401 x 201 physical,
    h = 10 m), one surface source, 3, 5 and 7 Hz: Krylov iterations and time to
    relres 1e-6 with the shifted-Laplace multigrid preconditioner at shift
    beta = (1, 0.5) and at the paper's (1, 1), and without a preconditioner."""
    import torch

    from paper_1712_08743_gb300 import _lib, api, build
    from synth import models

    build.build()
    _lib.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = api.Context(0, stream)
    mdl = models.c3_model()
    model = api.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    src = mdl.sources[len(mdl.sources) // 2: len(mdl.sources) // 2 + 1]
    kry = {"bicgstab": _lib.HELM_KRYLOV_BICGSTAB, "fgmres": _lib.HELM_KRYLOV_FGMRES}[args.krylov]
    rows = []
    for f_hz in (3.0, 5.0, 7.0):
        om = np.array([2 * np.pi * f_hz])
        for name, extra in (("MG beta=(1,0.5)", dict(beta=(1.0, 0.5))), ("MG beta=(1,1)", dict(beta=(1.0, 1.0))),
                            ("none", dict(precond=_lib.HELM_PRECOND_NONE))):
            opts = dict(tol=1e-6, precision="mixed", krylov=kry, restart=30, max_it=40000, **extra)
            api.helm_solve(model, om, src, opts=opts)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st, status = api.helm_solve(model, om, src, opts=opts)
            dt = time.perf_counter() - t0
            rows.append({"f_hz": f_hz, "preconditioner": name, "iters": st[0]["iters"], "ms": 1e3 * dt,
                         "converged": bool(st[0]["converged"]), "relres": st[0]["relres"]})
    print(json.dumps({"metric": "krylov_iterations", "workload": "ablation_401x201_1src_3-7Hz",
                      "krylov": args.krylov, "rows": rows}), flush=True)
    model.close()
    ctx.close()


def serve_stream(api, ctx, n: int, sizes, opts, rate: float, seed: int = 5):
    """Submits serving requests 0..n-1 (each generated just before it is due) at Poisson
    arrivals of `rate` per second (rate <= 0: all at once) through helm_submit; a poller
    thread collects every result in submission order (helm_poll) and releases it. Returns
    per-request records and the wall time from the first submission to the last completion."""
    import queue
    import threading as th

    from synth import models

    q = queue.Queue()
    recs = [None] * n
    t_sub = [0.0] * n

    def poller():
        for _ in range(n):
            i, t, N, f = q.get()
            res = api.helm_poll(ctx, t, -1, copy_u=False)
            recs[i] = {"N": N, "f_hz": f, "status": int(res.status), "latency_ms": res.latency_ms,
                       "queue_ms": res.queue_ms, "batch": res.batch_size, "iters": res.stats["iters"],
                       "relres": res.stats["relres"], "shift_switched": res.stats["shift_switched"]}
            api.helm_release(ctx, t)

    pt = th.Thread(target=poller)
    pt.start()
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    due = t0
    for i in range(n):
        r = models.c5_request(i, sizes=sizes)
        if rate > 0:
            due += rng.exponential(1.0 / rate)
            time.sleep(max(0.0, due - time.perf_counter()))
        t_sub[i] = time.perf_counter()
        t = api.helm_submit(ctx, r.slowness, r.h, r.omegas[0], r.sources[0], opts=opts)
        q.put((i, t, int(r.Px), float(r.omegas[0] / (2 * np.pi))))
    pt.join()
    t_end = max(t_sub[i] + 1e-3 * recs[i]["latency_ms"] for i in range(n))
    return recs, t_end - t0


def serve_summary(recs, wall):
    lat = [r["latency_ms"] for r in recs]
    return {"requests": len(recs), "solves_per_s": len(recs) / wall, "wall_s": wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "converged": sum(r["status"] == 0 for r in recs),
            "shift_switched": sum(bool(r["shift_switched"]) for r in recs),
            "mean_batch": float(np.mean([r["batch"] for r in recs])),
            "not_ok": [r for r in recs if r["status"] != 0]}


def run_serving(args):
    """The serving workload: a Poisson stream of solve requests of mixed grid sizes (128^2 ..
    1024^2) and frequencies (2..25 Hz, ten points per wavelength at 1500 m/s) on random layered
    models, served with continuous batching. First the saturated throughput (requests submitted
    all at once), then one stream per arrival rate rho x saturated (--rates), each reporting
    solves/s and p50/p99 latency; beside them the same kind of requests solved one after another
    in plain FP64 (--seq-requests of them)."""
    import torch

    from paper_1712_08743_gb300 import _lib, api, build
    from synth import models

    build.build()
    ctx = api.Context(0)
    sizes = tuple(int(x) for x in args.serve_sizes.split(","))
    kry = _lib.HELM_KRYLOV_FGMRES if args.krylov == "fgmres" else _lib.HELM_KRYLOV_BICGSTAB
    shift = {} if args.serve_beta2 is None else dict(beta2=args.serve_beta2)
    opts = dict(tol=1e-6, precision="mixed", krylov=kry, max_it=20000, reorth=REORTH[args.reorth], **shift)
    api.helm_serve_config(ctx, max_batch=16, max_slots=4)
    # warm-up: one request of each size through the server
    for N in sizes:
        warm = models.c5_request(0, sizes=(N,))
        t = api.helm_submit(ctx, warm.slowness, warm.h, warm.omegas[0], warm.sources[0], opts=opts)
        api.helm_poll(ctx, t, -1, copy_u=False)
        api.helm_release(ctx, t)
    # saturated throughput: every request queued at once
    nsat = min(args.requests, args.sat_requests)
    recs, wall = serve_stream(api, ctx, nsat, sizes, opts, rate=0.0)
    sat = serve_summary(recs, wall)
    rows = []
    for rho in (float(x) for x in args.rates.split(",")):
        rate = rho * sat["solves_per_s"] if args.rate <= 0 else args.rate
        with ClockSampler(0) as clk:
            recs, wall = serve_stream(api, ctx, args.requests, sizes, opts, rate=rate)
        row = {"rho": rho, "arrival_rate": rate, **serve_summary(recs, wall), "clocks": clk.summary()}
        rows.append(row)
    # sequential plain FP64 of the first requests of the same stream
    o64 = dict(tol=1e-6, precision="fp64", krylov=kry, max_it=20000, reorth=REORTH[args.reorth], **shift)
    t_seq = []
    for i in range(min(args.seq_requests, args.requests)):
        r = models.c5_request(i, sizes=sizes)
        mm = api.helm_create_model(ctx, r.slowness, r.h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.helm_solve(mm, r.omegas, r.sources, opts=o64)
        t_seq.append(time.perf_counter() - t0)
        mm.close()
    seq = {"requests": len(t_seq), "solves_per_s": len(t_seq) / float(np.sum(t_seq)),
           "p50_ms": 1e3 * float(np.percentile(t_seq, 50)), "p99_ms": 1e3 * float(np.percentile(t_seq, 99))}
    print(json.dumps({"metric": "helmholtz_solves_per_s",
                      "workload": f"serving_{args.requests}req_{min(sizes)}-{max(sizes)}",
                      "krylov": args.krylov, "shift": [1.0, args.serve_beta2 if args.serve_beta2 is not None else 0.5],
                      "unit": "solves/s", "saturated": sat, "rates": rows, "sequential_fp64": seq,
                      "sizes": {str(n): sum(models.c5_request(i, sizes=sizes).Px == n for i in range(args.requests))
                                for n in sizes} if args.requests <= 200 else None}), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.krylov is None:
        args.krylov = "fgmres" if args.workload in ("single", "serving") and not args.kernels_only else "bicgstab"
    if args.impl == "reference":
        run_reference(args)
    elif args.kernels_only:
        run_kernels_only(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "gn":
        run_gn(args)
    elif args.workload == "fwi":
        run_fwi(args)
    elif args.workload == "ablation":
        run_ablation(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
