"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (relative L2 unless stated): operator apply 1e-13 (FP64) / 2e-6 (FP32);
V-cycle 2e-5 (complex64 against a complex128 restatement); wavefields 1e-6 for
FP64 and FP64-refined solves, 1e-4 for pure complex64 solves; gradient 1e-5.
"""
import numpy as np
import pytest

import oracle
from oracle import multigrid as mg
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


# grids: the small plain case, a ragged one (partial tiles, odd/even levels), the batched case
GRIDS = [
    ("c1", lambda: models.c1_model()),
    ("ragged", lambda: models.Model("ragged", np.random.default_rng(11).uniform(1500, 3500, (23, 37)), 10.0,
                                    np.array([[5, 2]]), np.array([7.0]), npml=10)),
    ("c3", lambda: models.c3_model()),
]


@pytest.mark.parametrize("name,make", GRIDS)
def test_apply_matches_oracle_operator(hg, ctx, name, make):
    mdl = make()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    rng = np.random.default_rng(1)
    om = 2 * np.pi * np.array([3.0, 7.5])
    u = models.random_complex(rng, (2, model.nz, model.nx))
    m_pad = oracle.pad_slowness(mdl.slowness, mdl.npml)
    alpha = oracle.damping_profile(mdl.Px, mdl.Pz, mdl.npml, mdl.alpha_max)
    y64 = hg.helm_apply(model, om, u, hg.HELM_PREC_FP64)
    u32 = u.astype(np.complex64)
    y32 = hg.helm_apply(model, om, u32, hg.HELM_PREC_FP32)
    for k in range(2):
        B = oracle.operator(m_pad, mdl.h, om[k], alpha)
        ref = (B @ u[k].ravel()).reshape(model.nz, model.nx)
        assert rel(y64[k], ref) < 1e-13
        ref32 = (B @ u32[k].astype(np.complex128).ravel()).reshape(model.nz, model.nx)
        assert rel(y32[k], ref32) < 2e-6
    model.close()


@pytest.mark.parametrize("name,make", GRIDS)
def test_vcycle_matches_restatement(hg, ctx, name, make):
    mdl = make()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    rng = np.random.default_rng(2)
    om = 2 * np.pi * np.array([4.0, 6.0])
    r = models.random_complex(rng, (2, model.nz, model.nx), np.complex64)
    # default coarse end (for these few right-hand sides the first level with at most 1200
    # nodes solved by its dense inverse, one launch per step), the same cycle with its F-cycle
    # part in one persistent kernel, and the shared-memory tail over the whole hierarchy
    z_auto = {}
    for coarse, kind in [(None, "dense"), (hg.HELM_COARSE_FUSED, "dense"), (hg.HELM_COARSE_TAIL, "tail")]:
        for beta, wj in [((1.0, 0.5), 0.8), ((1.0, 1.0), 0.6)]:
            z = hg.helm_vcycle(model, om, r, beta, wj, coarse=coarse)
            m2 = oracle.pad_slowness(mdl.slowness, mdl.npml) ** 2
            assert len(mg.level_shapes(model.nx, model.nz)) == model.nlevels
            for k in range(2):
                V = mg.VCycle(m2, (mdl.h * om[k]) ** 2, beta, wj, coarse=kind)
                ref = V.apply(r[k].astype(np.complex128).ravel()).reshape(model.nz, model.nx)
                assert rel(z[k], ref) < 2e-5, (name, kind, beta, k, rel(z[k], ref))
            if coarse is None:
                z_auto[beta] = z
            elif coarse == hg.HELM_COARSE_FUSED:
                # the persistent kernel does each node's operations as the one-launch kernels do
                # (the compiler may contract them into fused multiply-adds differently: the two
                # agree to the rounding of complex64 arithmetic)
                assert rel(z, z_auto[beta]) < 1e-6, (name, beta, rel(z, z_auto[beta]))
    model.close()


@pytest.mark.parametrize("name,make", GRIDS)
def test_fused_prolongation_pairs_equal_separate_launches(hg, ctx, name, make):
    """Batches of at most 16 right-hand sides prolong two consecutive Galerkin levels in one
    launch (the finer level's correction recomputed in shared memory); larger batches launch
    them one by one. The same right-hand side alone and as the first of a batch of 17 (dense
    coarse end in both) must give the same cycle to complex64 rounding."""
    mdl = make()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    rng = np.random.default_rng(5)
    r = models.random_complex(rng, (1, model.nz, model.nx), np.complex64)
    om = 2 * np.pi * np.array([5.0])
    z1 = hg.helm_vcycle(model, om, r, (1.0, 0.5), 0.8, coarse=hg.HELM_COARSE_DENSE)
    z17 = hg.helm_vcycle(model, np.repeat(om, 17), np.repeat(r, 17, axis=0), (1.0, 0.5), 0.8,
                         coarse=hg.HELM_COARSE_DENSE)
    assert np.all(np.isfinite(z1))
    for k in (0, 16):
        assert rel(z17[k], z1[0]) < 1e-6, (name, k, rel(z17[k], z1[0]))
    model.close()


@pytest.mark.parametrize("coarse", [None, "dense"])
def test_large_batch_galerkin_kernels_equal_each_alone(hg, ctx, coarse):
    """Above 16 right-hand sides of one model the Galerkin kernels work on four per block and form
    each one's complex coefficients from the tile's real ones staged once. A batch of 20 with
    different frequencies (neighbours in a block differ) must give, for every member, the cycle
    of that right-hand side alone (the one-per-block kernels), to complex64 rounding; with the
    default coarse end the batch also takes the shared-memory tail, so only the dense end is
    compared member by member with the lone cycle, and the default end against the oracle cycle."""
    mdl = models.c3_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    rng = np.random.default_rng(9)
    om = 2 * np.pi * rng.uniform(3.0, 7.0, 20)
    r = models.random_complex(rng, (20, model.nz, model.nx), np.complex64)
    if coarse == "dense":
        z = hg.helm_vcycle(model, om, r, (1.0, 0.5), 0.8, coarse=hg.HELM_COARSE_DENSE)
        for k in (0, 1, 2, 3, 7, 19):
            z1 = hg.helm_vcycle(model, om[k:k + 1], r[k:k + 1], (1.0, 0.5), 0.8, coarse=hg.HELM_COARSE_DENSE)
            assert rel(z[k], z1[0]) < 1e-6, (k, rel(z[k], z1[0]))
    else:
        z = hg.helm_vcycle(model, om, r, (1.0, 0.5), 0.8)
        m2 = oracle.pad_slowness(mdl.slowness, mdl.npml) ** 2
        for k in (0, 5, 19):
            V = mg.VCycle(m2, (mdl.h * om[k]) ** 2, (1.0, 0.5), 0.8, coarse="tail")
            ref = V.apply(r[k].astype(np.complex128).ravel()).reshape(model.nz, model.nx)
            assert rel(z[k], ref) < 2e-5, (k, rel(z[k], ref))
    model.close()


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-6), ("mixed", 1e-10, 1e-6), ("fp32", 5e-5, 1e-4)])
def test_c1_wavefield_matches_oracle(hg, ctx, precision, tol, bound):
    mdl = models.c1_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    u, stats, st = hg.helm_solve(model, mdl.omegas, mdl.sources, opts=dict(tol=tol, precision=precision))
    ref = oracle.solve_fields(mdl.slowness, mdl.h, mdl.omegas[0], mdl.sources, mdl.npml, mdl.alpha_max)
    assert st == hg.HELM_OK and stats[0]["converged"] and stats[0]["relres"] <= tol, stats
    assert rel(u, ref) < bound, rel(u, ref)
    # physical part alone, as reported
    p = slice(mdl.npml, -mdl.npml)
    assert rel(u[0][p, p], ref[0][p, p]) < bound
    model.close()


@pytest.mark.parametrize("krylov", ["bicgstab", "fgmres"])
def test_unpreconditioned_solve_matches_oracle(hg, ctx, krylov):
    """The preconditioner-free path of the ablation solves the same system (more iterations)."""
    mdl = models.c1_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    ref = oracle.solve_fields(mdl.slowness, mdl.h, mdl.omegas[0], mdl.sources, mdl.npml, mdl.alpha_max)[0]
    kr = hg.HELM_KRYLOV_BICGSTAB if krylov == "bicgstab" else hg.HELM_KRYLOV_FGMRES
    u, st, status = hg.helm_solve(model, mdl.omegas, mdl.sources,
                                  opts=dict(tol=1e-10, precision="mixed", krylov=kr, restart=30, max_it=50000,
                                            precond=hg.HELM_PRECOND_NONE))
    assert status == hg.HELM_OK, st
    assert rel(u[0], ref) < 1e-6
    _, stp, _ = hg.helm_solve(model, mdl.omegas, mdl.sources, opts=dict(tol=1e-10, precision="mixed", krylov=kr))
    assert st[0]["iters"] > 2 * stp[0]["iters"]      # the preconditioner pays for itself
    model.close()


@pytest.mark.parametrize("reorth", ["always", "never", "ifneeded"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fgmres_matches_oracle_and_bicgstab(hg, ctx, precision, reorth):
    """Flexible GMRES (restart 20) with each Gram-Schmidt variant on the small case and
    a batched pair of the batched case: same wavefields as the oracle, and as BiCGSTAB,
    within the solve tolerance."""
    mdl = models.c1_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    ro = {"always": hg.HELM_REORTH_ALWAYS, "never": hg.HELM_REORTH_NEVER, "ifneeded": hg.HELM_REORTH_IFNEEDED}[reorth]
    opts = dict(tol=1e-10, precision=precision, krylov=hg.HELM_KRYLOV_FGMRES, restart=20, reorth=ro)
    u, stats, st = hg.helm_solve(model, mdl.omegas, mdl.sources, opts=opts)
    ref = oracle.solve_fields(mdl.slowness, mdl.h, mdl.omegas[0], mdl.sources, mdl.npml, mdl.alpha_max)
    assert st == hg.HELM_OK and stats[0]["converged"], stats
    assert rel(u, ref) < 1e-6
    model.close()
    m3 = models.c3_model()
    model = hg.helm_create_model(ctx, m3.slowness, m3.h, m3.npml, m3.alpha_max)
    om = m3.omegas[[0, 4]]
    src = m3.sources[[5, 40]]
    uf, sf, _ = hg.helm_solve(model, om, src, opts=opts)
    ub, sb, _ = hg.helm_solve(model, om, src, opts=dict(tol=1e-10, precision=precision))
    for k in range(2):
        assert sf[k]["converged"] and rel(uf[k], ub[k]) < 1e-6
    model.close()


def test_ragged_grid_general_rhs(hg, ctx):
    mdl = GRIDS[1][1]()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    rng = np.random.default_rng(3)
    F = models.random_complex(rng, (3, model.nz, model.nx))
    om = 2 * np.pi * np.array([2.0, 7.0, 13.0])
    for precision in ("fp64", "mixed"):
        u, stats, st = hg.helm_solve(model, om, f=F, opts=dict(tol=1e-11, precision=precision))
        for k in range(3):
            ref = oracle.solve_fields(mdl.slowness, mdl.h, om[k], None, mdl.npml, mdl.alpha_max,
                                      F=F[k].reshape(1, -1))[0]
            assert rel(u[k], ref) < 1e-6, (precision, k, rel(u[k], ref))
    model.close()


def test_degenerate_inputs(hg, ctx):
    """Degenerate cases of Eq. 3: a zero right-hand side gives u = 0 at once, also
    beside a non-zero one in the same batch; a frequency near zero (almost the
    Dirichlet Poisson problem) still matches the oracle; an empty batch is refused."""
    mdl = GRIDS[1][1]()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    F = np.zeros((2, model.nz, model.nx), np.complex128)
    F[1] = models.random_complex(np.random.default_rng(7), (model.nz, model.nx))
    om = 2 * np.pi * np.array([5.0, 0.05])
    for precision in ("fp64", "mixed"):
        u, stats, st = hg.helm_solve(model, om, f=F, opts=dict(tol=1e-10, precision=precision))
        assert st == hg.HELM_OK, stats
        assert np.all(u[0] == 0) and stats[0]["converged"] and stats[0]["relres"] == 0.0
        ref = oracle.solve_fields(mdl.slowness, mdl.h, om[1], None, mdl.npml, mdl.alpha_max,
                                  F=F[1].reshape(1, -1))[0]
        assert rel(u[1], ref) < 1e-6, (precision, rel(u[1], ref))
    with pytest.raises(hg.HelmError):
        hg.helm_solve(model, np.zeros(0), np.zeros((0, 2), np.int32))
    model.close()


def test_batch_equals_each_alone_and_oracle(hg, ctx):
    mdl = models.c3_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    shots = mdl.sources[[0, 31, 63]]
    om = np.repeat(mdl.omegas[[0, 4]], 3)
    src = np.tile(shots, (2, 1))
    opts = dict(tol=1e-10)
    ub, sb, _ = hg.helm_solve(model, om, src, opts=opts)
    for k in (0, 4):
        ua, sa, _ = hg.helm_solve(model, om[k:k + 1], src[k:k + 1], opts=opts)
        assert np.array_equal(ua[0], ub[k]) and sa[0]["iters"] == sb[k]["iters"]
    for k in (0, 5):
        ref = oracle.solve_fields(mdl.slowness, mdl.h, om[k], src[k:k + 1], mdl.npml, mdl.alpha_max)[0]
        assert rel(ub[k], ref) < 1e-6
    model.close()


def test_autotuned_tiles_give_the_same_wavefields(hg, ctx, tmp_path):
    """Every tile shape of the Galerkin kernels (and the autotuner's choice) gives the same
    wavefields; the cycle runs one launch per step so that every level uses the shapes."""
    from paper_1712_08743_gb300 import autotune

    mdl = models.c3_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    om = np.repeat(mdl.omegas[[1, 3]], 4)
    src = np.tile(mdl.sources[[3, 20, 41, 60]], (2, 1))
    opts = dict(tol=1e-9, coarse=hg.HELM_COARSE_DENSE)
    u0, _, _ = hg.helm_solve(model, om, src, opts=opts)
    tiles = autotune.autotune(model, len(om), float(om[0]), str(tmp_path / "t.json"))
    n = autotune.NTILES // 2
    assert len(tiles) == autotune.NTILES
    assert all(0 <= t <= 5 for t in tiles[:n]) and all(0 <= t <= 4 for t in tiles[n:]) and tiles[n] <= 1
    import ctypes as C
    for code in [None, 0, 2, 3, 4, 5]:
        if code is not None:   # the same shape code on every level (finest prolongation: 0 or 1;
            # restriction-only code 5: prolongation code 1)
            pc = min(code, 4) if code < 5 else 1
            arr = [code] * n + [min(pc, 1)] + [pc] * (n - 1)
            assert model.lib.helm_set_tiles(model.handle, (C.c_int * autotune.NTILES)(*arr)) == 0
        u1, st, _ = hg.helm_solve(model, om, src, opts=opts)
        assert all(s["converged"] for s in st)
        for k in range(len(om)):
            assert rel(u1[k], u0[k]) < 1e-6   # dot products sum in another order; tol 1e-9 solves
    bad = (C.c_int * autotune.NTILES)(*([6] * autotune.NTILES))
    assert model.lib.helm_set_tiles(model.handle, bad) == hg.HELM_E_INVALID
    model.close()


def test_not_converged_status_and_best_iterate(hg, ctx):
    mdl = models.c1_model()
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    u, stats, st = hg.helm_solve(model, mdl.omegas, mdl.sources, opts=dict(tol=1e-10, max_it=4, check_every=2))
    assert st == hg.HELM_E_NOT_CONVERGED
    assert not stats[0]["converged"] and 0 < stats[0]["iters"] <= 4 + 2 and 0 < stats[0]["relres"] < 1
    assert np.all(np.isfinite(u))
    model.close()


def test_invalid_arguments(hg, ctx):
    m = np.full((30, 30), 1 / 2000.0)
    m[3, 4] = np.nan
    with pytest.raises(hg.HelmError):
        hg.helm_create_model(ctx, m, 10.0)
    model = hg.helm_create_model(ctx, np.full((30, 30), 1 / 2000.0), 10.0, 10)
    with pytest.raises(hg.HelmError):
        hg.helm_solve(model, [2 * np.pi * 5], [[30, 0]])
    with pytest.raises(hg.HelmError):
        hg.helm_solve(model, [-1.0], [[3, 0]])
    with pytest.raises(hg.HelmError):
        hg.helm_solve(model, [2 * np.pi * 5], [[3, 0]], opts=dict(krylov=hg.HELM_KRYLOV_FGMRES, reorth=3))
    model.close()


def _small_fwi(seed=0):
    rng = np.random.default_rng(seed)
    Px, Pz, h, npml = 48, 32, 10.0, 10
    c_true = models.layered_model(rng, Px, Pz, h, 4)
    c0 = np.full_like(c_true, c_true.mean())
    src = np.array([[6, 1], [24, 1], [40, 1]])
    rec = np.array([[i, 1] for i in range(0, Px, 4)])
    om = 2 * np.pi * np.array([6.0, 9.0])
    d_obs = np.stack([oracle.sample_receivers(oracle.solve_fields(1 / c_true, h, w, src, npml), rec, npml) for w in om])
    return 1 / c0, h, npml, src, rec, om, d_obs


def test_gradient_matches_oracle_and_differences(hg, ctx):
    m0, h, npml, src, rec, om, d_obs = _small_fwi()
    lam = 1e-3
    model = hg.helm_create_model(ctx, m0, h, npml, 0.5)
    opts = dict(tol=1e-12)
    J, g, dcal, stats, st = hg.helm_adjoint_gradient(model, om, src, rec, d_obs, lam, opts)
    Jr, gr = oracle.gradient(m0, h, om, src, rec, d_obs, lam, npml)
    assert abs(J - Jr) / Jr < 1e-8
    assert rel(g, gr) < 1e-5
    # central differences of the GPU misfit at three cells (one on the edge); J from
    # solves at relres 1e-12 carries about 1e-12 relative error, which a difference of
    # 2e-4 relative steps magnifies to ~1e-4, so the steps are 1e-3 and 3e-3 (the
    # truncation error, O(step^2), stays near 1e-6) and the better one counts
    for (iz, ix) in [(0, 0), (10, 20), (31, 47)]:
        best = np.inf
        for step in (1e-3, 3e-3):
            e = step * m0[iz, ix]
            Js = []
            for sgn in (1, -1):
                mp = m0.copy()
                mp[iz, ix] += sgn * e
                mm = hg.helm_create_model(ctx, mp, h, npml, 0.5)
                Js.append(hg.helm_adjoint_gradient(mm, om, src, rec, d_obs, lam, opts)[0])
                mm.close()
            fd = (Js[0] - Js[1]) / (2 * e)
            best = min(best, abs(fd - g[iz, ix]) / abs(g[iz, ix]))
        assert best < 1e-4, ((iz, ix), best, g[iz, ix])
    model.close()


def test_gauss_newton_product_and_step_match_oracle(hg, ctx):
    """Eq. 8 without its second term and Eq. 9: the GPU Hessian-vector product against
    the oracle's (and its symmetry), and a 4-iteration CG step against the oracle's."""
    m0, h, npml, src, rec, om, d_obs = _small_fwi(2)
    lam = 1e2
    model = hg.helm_create_model(ctx, m0, h, npml, 0.5)
    opts = dict(tol=1e-11)
    J, dcal, state, _, st = hg.helm_fwi_forward(model, om, src, rec, d_obs, lam, opts)
    assert st == hg.HELM_OK
    g, st = hg.helm_fwi_backward(model, state, opts)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(m0.shape) * m0
    y = rng.standard_normal(m0.shape) * m0
    hx, st = hg.helm_gn_hvp(model, state, x, opts)
    assert st == hg.HELM_OK
    hy, _ = hg.helm_gn_hvp(model, state, y, opts)
    hx_ref = oracle.gn_hvp(m0, h, om, src, rec, lam, x, npml)
    assert rel(hx, hx_ref) < 1e-6
    assert abs(np.sum(x * hy) - np.sum(y * hx)) <= 1e-7 * abs(np.sum(x * hy))
    dm, relres, st = hg.helm_gn_step(model, state, g, 4, opts)
    dm_ref, rel_ref = oracle.gn_step(m0, h, om, src, rec, lam, g, 4, npml)
    assert rel(dm, dm_ref) < 1e-5
    np.testing.assert_allclose(relres, rel_ref, rtol=1e-4)
    assert relres[-1] < relres[0]
    # the step lowers the misfit of Eq. 4
    m1 = hg.helm_create_model(ctx, m0 + dm, h, npml, 0.5)
    J1 = hg.helm_adjoint_gradient(m1, om, src, rec, d_obs, lam, opts)[0]
    m1.close()
    assert J1 < J
    state.close()
    model.close()


@pytest.mark.parametrize("strategy", ["simultaneous", "sequential"])
def test_fwi_loop_matches_oracle(hg, ctx, strategy):
    """The Gauss-Newton inversion loop, all frequencies at once or lowest first: the
    same accepted steps, misfit history and final model as the oracle's loop, and a
    checkpoint for every accepted model."""
    m0, h, npml, src, rec, om, d_obs = _small_fwi(2)
    lam, bounds = 1e2, (1 / 4000.0, 1 / 1000.0)
    seen = []
    m, hist, st = hg.helm_fwi_run(ctx, m0, h, om, src, rec, d_obs, lam, strategy=strategy, gn_iters=2, cg_iters=4,
                                  max_halvings=3, m_bounds=bounds, npml=npml, opts=dict(tol=1e-11),
                                  checkpoint=lambda g, i, mm, J: seen.append((g, i, mm, J)))
    m_ref, hist_ref = oracle.fwi_run(m0, h, om, src, rec, d_obs, lam, strategy=strategy, gn_iters=2, cg_iters=4,
                                     max_halvings=3, m_bounds=bounds, npml=npml)
    assert st == hg.HELM_OK
    assert len(hist) == len(hist_ref) >= 3
    np.testing.assert_allclose(hist, hist_ref, rtol=1e-5)
    assert rel(m - m0, m_ref - m0) < 1e-4
    assert len(seen) == len(hist) and np.array_equal(seen[-1][2], m)
    assert [J for *_, J in seen] == list(hist)
    with pytest.raises(hg.HelmError):
        hg.helm_fwi_run(ctx, m0, h, om, src, rec, d_obs, 0.0, npml=npml)


def test_autograd_backward_runs_adjoint(hg, ctx):
    import torch

    from paper_1712_08743_gb300.autograd import FWIProblem, HelmFWI

    m0, h, npml, src, rec, om, d_obs = _small_fwi(1)
    prob = FWIProblem(ctx, h, om, src, rec, d_obs, 1e-3, npml, 0.5, dict(tol=1e-12))
    m = torch.tensor(m0, dtype=torch.float64, device="cuda", requires_grad=True)
    J = HelmFWI.apply(m, prob)
    J.backward(retain_graph=True)
    Jr, gr = oracle.gradient(m0, h, om, src, rec, d_obs, 1e-3, npml)
    assert abs(J.item() - Jr) / Jr < 1e-8
    assert rel(m.grad.cpu().numpy(), gr) < 1e-5
    # the forward's device state serves one backward: a second one through the same graph raises
    with pytest.raises(RuntimeError, match="backward ran already"):
        J.backward()


def test_served_results_equal_lone_solves(hg):
    """Each served result equals the lone helm_solve of its request within the wavefield bar
    (1e-6, solves to relres 1e-10). Not bit for bit: a batch whose member stalls continues with
    the (1, 1) shift as a whole (the stall guard), so a request can take another Krylov path in
    a batch than alone; both reach the tolerance."""
    ctx = hg.Context(0)
    hg.helm_serve_config(ctx, max_batch=4, max_slots=2)
    reqs = []
    for i in range(6):
        n = 64 if i % 2 == 0 else 96
        rng = np.random.default_rng(100 + i)
        f = float(rng.uniform(3, 8))
        h = 1500.0 / (12 * f)
        c = models.layered_model(rng, n, n, h, 5)
        reqs.append((1 / c, h, 2 * np.pi * f, (n // 2, 2)))
    opts = dict(tol=1e-10)
    tickets = [hg.helm_submit(ctx, m, h, w, s, opts=opts) for (m, h, w, s) in reqs]
    served = [hg.helm_poll(ctx, t, 120000) for t in tickets]
    for (m, h, w, s), res, t in zip(reqs, served, tickets):
        assert res is not None and res.status == hg.HELM_OK and res.latency_ms >= res.queue_ms >= 0
        model = hg.helm_create_model(ctx, m, h)
        u, st, _ = hg.helm_solve(model, [w], [s], opts=opts)
        assert rel(res.u, u[0]) < 1e-6, (rel(res.u, u[0]), res.stats, st[0])
        model.close()
        hg.helm_release(ctx, t)
    assert max(r.batch_size for r in served) >= 2
    ctx.close()


def test_served_requests_match_the_oracle(hg):
    """Requests of the serving workload's kind (a 128^2 and a 256^2 grid, layered models,
    ten points per wavelength) served together with a smaller one: each served wavefield
    matches the oracle's sparse-LU wavefield to 1e-6 (tol 1e-10)."""
    ctx = hg.Context(0)
    hg.helm_serve_config(ctx, max_batch=4, max_slots=2)
    reqs = [models.c5_request(i) for i in (6, 1)]          # 128^2 at 13.5 Hz, 256^2 at 9.9 Hz
    rng = np.random.default_rng(11)
    c = models.layered_model(rng, 64, 64, 20.0, 4)
    opts = dict(tol=1e-10, krylov=hg.HELM_KRYLOV_FGMRES, max_it=20000)
    tickets = [hg.helm_submit(ctx, r.slowness, r.h, r.omegas[0], r.sources[0], opts=opts) for r in reqs]
    tickets.append(hg.helm_submit(ctx, 1 / c, 20.0, 2 * np.pi * 5.0, (32, 2), opts=opts))
    served = [hg.helm_poll(ctx, t, 300000) for t in tickets]
    for r, res in zip(reqs, served):
        assert res is not None and res.status == hg.HELM_OK, (r.name, res and res.stats)
        ref = oracle.solve_fields(r.slowness, r.h, r.omegas[0], r.sources, 20, 0.5)[0]
        assert rel(res.u, ref) < 1e-6, (r.name, rel(res.u, ref))
    assert served[2] is not None and served[2].status == hg.HELM_OK
    for t in tickets:
        hg.helm_release(ctx, t)
    ctx.close()


def test_serving_refuses_what_cannot_fit(hg):
    ctx = hg.Context(0)
    hg.helm_serve_config(ctx, max_batch=4, max_slots=1, reserve_bytes=0, budget_bytes=1 << 20)
    m = np.full((200, 200), 1 / 2000.0)
    t = hg.helm_submit(ctx, m, 10.0, 2 * np.pi * 5, (100, 2))
    res = hg.helm_poll(ctx, t, 60000)
    assert res is not None and res.status == hg.HELM_E_NOMEM
    ctx.close()


# ------------------------------------------------ variable density (Eq. 1)
def _density(Pz, Px, seed=0):
    """Two density layers with a smooth lateral variation (values 0.7 .. 2.8)."""
    z = np.arange(Pz)[:, None] * np.ones((1, Px))
    return np.where(z < Pz // 2, 1.0, 2.5) + 0.3 * np.sin(np.arange(Px)[None, :] / 7.0 + seed)


def test_density_apply_and_cycle_match_oracle(hg, ctx):
    """Eq. 1 operator (FP64 and FP32) against the oracle's flux form, and one
    preconditioner cycle built on it against the oracle's restatement."""
    mdl = models.c1_model()
    rho = _density(mdl.Pz, mdl.Px)
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max, density=rho)
    rng = np.random.default_rng(3)
    om = 2 * np.pi * np.array([3.0, 7.5])
    u = models.random_complex(rng, (2, model.nz, model.nx))
    m_pad = oracle.pad_slowness(mdl.slowness, mdl.npml)
    rho_pad = oracle.pad_slowness(rho, mdl.npml)
    alpha = oracle.damping_profile(mdl.Px, mdl.Pz, mdl.npml, mdl.alpha_max)
    y64 = hg.helm_apply(model, om, u, hg.HELM_PREC_FP64)
    u32 = u.astype(np.complex64)
    y32 = hg.helm_apply(model, om, u32, hg.HELM_PREC_FP32)
    for k in range(2):
        B = oracle.operator(m_pad, mdl.h, om[k], alpha, rho_pad)
        assert rel(y64[k], (B @ u[k].ravel()).reshape(model.nz, model.nx)) < 1e-13
        ref32 = (B @ u32[k].astype(np.complex128).ravel()).reshape(model.nz, model.nx)
        assert rel(y32[k], ref32) < 2e-6
    r = models.random_complex(rng, (2, model.nz, model.nx), np.complex64)
    z = hg.helm_vcycle(model, om, r, (1.0, 0.5), 0.5)
    for k in range(2):
        V = mg.VCycle(m_pad ** 2, (mdl.h * om[k]) ** 2, (1.0, 0.5), 0.5, rho_pad=rho_pad)
        ref = V.apply(r[k].astype(np.complex128).ravel()).reshape(model.nz, model.nx)
        assert rel(z[k], ref) < 2e-5, (k, rel(z[k], ref))
    model.close()


@pytest.mark.parametrize("krylov,precision", [("bicgstab", "mixed"), ("fgmres", "mixed"), ("bicgstab", "fp64")])
def test_density_wavefield_matches_oracle(hg, ctx, krylov, precision):
    """Wavefield of Eq. 1 against the oracle's LU solve; a unit density reproduces the
    constant-density wavefield."""
    mdl = models.c1_model()
    rho = _density(mdl.Pz, mdl.Px, 1)
    kr = hg.HELM_KRYLOV_BICGSTAB if krylov == "bicgstab" else hg.HELM_KRYLOV_FGMRES
    opts = dict(tol=1e-10, precision=precision, krylov=kr, restart=20)
    model = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max, density=rho)
    u, stats, st = hg.helm_solve(model, mdl.omegas, mdl.sources, opts=opts)
    ref = oracle.solve_fields(mdl.slowness, mdl.h, mdl.omegas[0], mdl.sources, mdl.npml, mdl.alpha_max, rho_phys=rho)
    assert st == hg.HELM_OK and stats[0]["converged"], stats
    assert rel(u, ref) < 1e-6, rel(u, ref)
    model.close()
    m1 = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max, density=np.ones_like(rho))
    m0 = hg.helm_create_model(ctx, mdl.slowness, mdl.h, mdl.npml, mdl.alpha_max)
    u1 = hg.helm_solve(m1, mdl.omegas, mdl.sources, opts=opts)[0]
    u0 = hg.helm_solve(m0, mdl.omegas, mdl.sources, opts=opts)[0]
    assert rel(u1, u0) < 1e-8
    m1.close()
    m0.close()


def test_density_gradient_matches_oracle(hg, ctx):
    """Eq. 7 at a model with a density (the density enters B only) against the oracle."""
    m0, h, npml, src, rec, om, d_obs = _small_fwi(3)
    rho = _density(*m0.shape, 2)
    model = hg.helm_create_model(ctx, m0, h, npml, 0.5, density=rho)
    J, g, _, _, st = hg.helm_adjoint_gradient(model, om, src, rec, d_obs, 1e-3, dict(tol=1e-12))
    Jr, gr = oracle.gradient(m0, h, om, src, rec, d_obs, 1e-3, npml, rho_phys=rho)
    assert st == hg.HELM_OK
    assert abs(J - Jr) / Jr < 1e-8
    assert rel(g, gr) < 1e-5
    model.close()
    with pytest.raises(hg.HelmError):
        hg.helm_create_model(ctx, m0, h, npml, 0.5, density=-rho)
