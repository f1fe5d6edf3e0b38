"""GPU parity at the full sizes of the configured workloads, in the launch
configuration the benchmark uses.

* Single large case (1041 x 1041 padded, 15 Hz): the mixed-precision FGMRES and
  BiCGSTAB solves against the oracle's sparse-LU wavefield, and the FP64 true
  residual recomputed on the CPU with the oracle's operator.
* Batched case (320 right-hand sides, 441 x 241 padded): the true residual of
  sampled right-hand sides with the oracle's operator, and oracle wavefields
  for a few of them.
* Gradient case (32 shots x 4 frequencies, 201 receivers): gradient against the
  oracle's adjoint gradient (1e-5) and central differences of the GPU misfit on
  20 random cells (seed 44) with a non-negligible gradient (1e-2: the differences
  of a misfit built from iterative solves are noise-limited; the oracle
  comparison is the pin).
Tolerances: wavefield 1e-6 (FP64-refined), gradient 1e-5 (relative L2).
"""
import numpy as np
import pytest

import oracle
from synth import models

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import paper_1712_08743_gb300 as hg

    hg.load(build_if_missing=True)
    return hg


@pytest.fixture(scope="module")
def ctx(hg):
    c = hg.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def true_relres(mdl, omega, u, F):
    m_pad = oracle.pad_slowness(mdl.slowness, mdl.npml)
    alpha = oracle.damping_profile(mdl.Px, mdl.Pz, mdl.npml, mdl.alpha_max)
    B = oracle.operator(m_pad, mdl.h, omega, alpha)
    return float(np.linalg.norm(F - B @ u.ravel()) / np.linalg.norm(F))


@pytest.mark.timeout(1200)
def test_single_large_case_matches_oracle(hg, ctx):
    mdl = models.c2_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    ref = oracle.solve_fields(mdl.slowness, mdl.h, mdl.omegas[0], mdl.sources, mdl.npml, mdl.alpha_max)[0]
    F = oracle.point_sources(model.nx, model.nz, mdl.h, mdl.sources + mdl.npml)[0]
    for krylov in (hg.HELM_KRYLOV_FGMRES, hg.HELM_KRYLOV_BICGSTAB):
        u, st, status = hg.helm_solve(model, mdl.omegas, mdl.sources,
                                      opts=dict(tol=1e-10, precision="mixed", krylov=krylov, max_it=20000))
        assert status == hg.HELM_OK, st
        assert true_relres(mdl, mdl.omegas[0], u[0], F) < 2e-10
        assert rel(u[0], ref) < 1e-6, (krylov, rel(u[0], ref))
    # at the benchmark tolerance the true residual recomputed on the CPU meets 1e-6
    u, st, status = hg.helm_solve(model, mdl.omegas, mdl.sources,
                                  opts=dict(tol=1e-6, precision="mixed", krylov=hg.HELM_KRYLOV_FGMRES))
    assert status == hg.HELM_OK and true_relres(mdl, mdl.omegas[0], u[0], F) <= 1.0001e-6
    model.close()


@pytest.mark.timeout(1200)
def test_single_large_case_in_the_benchmark_configuration(hg, ctx):
    """The exact options the benchmark times: FGMRES(10) with one classical Gram-Schmidt
    pass, inner reduction 5e-2 per refinement step, mixed precision, the default coarse end
    (the first level with at most 1200 nodes solved by its dense inverse). At tol 1e-10 the
    wavefield matches the oracle's sparse LU to 1e-6; at the benchmark's tol 1e-6 the FP64
    true residual recomputed on the CPU meets 1e-6. The shared-memory tail variant of the
    cycle gives the same wavefield."""
    mdl = models.c2_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    ref = oracle.solve_fields(mdl.slowness, mdl.h, mdl.omegas[0], mdl.sources, mdl.npml, mdl.alpha_max)[0]
    F = oracle.point_sources(model.nx, model.nz, mdl.h, mdl.sources + mdl.npml)[0]
    bench = dict(precision="mixed", krylov=hg.HELM_KRYLOV_FGMRES, restart=10, reorth=hg.HELM_REORTH_NEVER,
                 inner_tol=5e-2, max_it=20000)
    u, st, status = hg.helm_solve(model, mdl.omegas, mdl.sources, opts=dict(tol=1e-10, **bench))
    assert status == hg.HELM_OK and st[0]["dense_level"] > 0, st
    assert rel(u[0], ref) < 1e-6, rel(u[0], ref)
    u, st, status = hg.helm_solve(model, mdl.omegas, mdl.sources, opts=dict(tol=1e-6, **bench))
    assert status == hg.HELM_OK and st[0]["relres"] <= 1e-6
    assert true_relres(mdl, mdl.omegas[0], u[0], F) <= 1.0001e-6
    u, st, status = hg.helm_solve(model, mdl.omegas, mdl.sources,
                                  opts=dict(tol=1e-10, coarse=hg.HELM_COARSE_TAIL, **bench))
    assert status == hg.HELM_OK and st[0]["dense_level"] == 0
    assert rel(u[0], ref) < 1e-6
    model.close()


@pytest.mark.timeout(1200)
def test_batched_case_residuals_and_oracle(hg, ctx):
    mdl = models.c3_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    om = np.repeat(mdl.omegas, len(mdl.sources))
    src = np.tile(mdl.sources, (len(mdl.omegas), 1))
    u, st, status = hg.helm_solve(model, om, src, opts=dict(tol=1e-6, precision="mixed"))
    assert status == hg.HELM_OK and all(s["converged"] for s in st)
    rng = np.random.default_rng(9)
    for k in rng.choice(len(om), 6, replace=False):
        F = oracle.point_sources(model.nx, model.nz, mdl.h, src[k:k + 1] + mdl.npml)[0]
        assert true_relres(mdl, om[k], u[k], F) <= 1.0001e-6
    # tighter solves of a few right-hand sides against oracle wavefields
    pick = [0, 100, 319]
    ut, _, status = hg.helm_solve(model, om[pick], src[pick], opts=dict(tol=1e-10, precision="mixed"))
    assert status == hg.HELM_OK
    for i, k in enumerate(pick):
        ref = oracle.solve_fields(mdl.slowness, mdl.h, om[k], src[k:k + 1], mdl.npml, mdl.alpha_max)[0]
        assert rel(ut[i], ref) < 1e-6
    model.close()


@pytest.mark.timeout(1800)
def test_gradient_case_matches_oracle_and_differences(hg, ctx):
    true, start = models.c4_models()
    lam = 1e-3
    om = true.omegas
    d_obs = np.stack([oracle.sample_receivers(
        oracle.solve_fields(true.slowness, true.h, w, true.sources, true.npml, true.alpha_max), true.receivers,
        true.npml) for w in om])
    opts = dict(tol=1e-10, precision="mixed")
    model = hg.helm_create_model(ctx, start.slowness, start.h, start.npml, start.alpha_max)
    J, g, dcal, st, status = hg.helm_adjoint_gradient(model, om, start.sources, start.receivers, d_obs, lam, opts)
    assert status == hg.HELM_OK
    Jr, gr = oracle.gradient(start.slowness, start.h, om, start.sources, start.receivers, d_obs, lam, start.npml,
                             start.alpha_max)
    assert abs(J - Jr) / Jr < 1e-8
    assert rel(g, gr) < 1e-5
    model.close()
    # central differences of the GPU misfit on random cells where the gradient is not
    # tiny (the misfit from iterative solves carries noise near 1e-10 relative, so the
    # differences are taken at 1e-3 of the cell's slowness and compared to 1e-2)
    rng = np.random.default_rng(44)
    big = np.argwhere(np.abs(g) >= 0.05 * np.max(np.abs(g)))
    cells = [tuple(int(v) for v in big[k]) for k in rng.choice(len(big), 20, replace=False)]
    for iz, ix in cells:
        e = 1e-3 * start.slowness[iz, ix]
        Js = []
        for sgn in (1, -1):
            mp = start.slowness.copy()
            mp[iz, ix] += sgn * e
            mm = hg.helm_create_model(ctx, mp, start.h, start.npml, start.alpha_max)
            Js.append(hg.helm_adjoint_gradient(mm, om, start.sources, start.receivers, d_obs, lam, opts)[0])
            mm.close()
        fd = (Js[0] - Js[1]) / (2 * e)
        assert abs(fd - g[iz, ix]) <= 1e-2 * abs(g[iz, ix]), ((iz, ix), fd, g[iz, ix])


@pytest.mark.timeout(1800)
@pytest.mark.parametrize("krylov", ["default", "fgmres"])
def test_serving_requests_that_stall_under_the_default_shift_converge(hg, ctx, krylov):
    """Four serving requests (1024^2 at 22.6, 12.6 and 6.6 Hz, 512^2 at 3.6 Hz: layered models
    with slow layers between fast ones) on which the default shift (1, 0.5) with Jacobi weight
    0.5 does not give a stable cycle: under the library defaults (and with FGMRES) the stall
    guard switches them to the paper's (1, 1) shift and each converges; the FP64 true residual,
    recomputed on the CPU, meets the tolerance."""
    opts = {}
    if krylov == "fgmres":
        opts.update(krylov=hg.HELM_KRYLOV_FGMRES)
    for i in (2, 15, 17, 26):
        r = models.c5_request(i)
        model = hg.helm_create_model(ctx, r.slowness, r.h)
        u, st, status = hg.helm_solve(model, r.omegas, r.sources, opts=opts)
        assert status == hg.HELM_OK and st[0]["converged"], (i, krylov, st)
        F = oracle.point_sources(model.nx, model.nz, r.h, r.sources + r.npml)[0]
        assert true_relres(r, r.omegas[0], u[0], F) <= 1.0001e-6
        model.close()
