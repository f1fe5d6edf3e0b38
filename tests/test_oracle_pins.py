"""Pins for the CPU oracle against facts that do not come from the oracle itself.

Each test ties one part of the oracle to mathematics or physics fixed
independently of its code: a discrete eigenpair of the 5-point Laplacian, a
matrix assembled node by node from Eq. 2, second-order convergence to a smooth
manufactured solution, the free-space Green's function, source-receiver
reciprocity, and finite differences / Taylor expansion of the misfit of Eq. 4.
The last tests plant plausible mistakes in the oracle and check that a pin
catches each one.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.special

import oracle
from oracle import helmholtz as H
from synth import models


def _rng(seed=0):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------- damping layer
def test_damping_profile_closed_form():
    Px, Pz, npml, amax = 7, 5, 4, 0.5
    a = oracle.damping_profile(Px, Pz, npml, amax)
    assert a.shape == (Pz + 8, Px + 8)
    assert np.all(a[npml:npml + Pz, npml:npml + Px] == 0.0)          # physical interior
    assert a[npml, 0] == pytest.approx(amax)                          # outermost node, d = npml
    assert a[npml, npml - 1] == pytest.approx(amax * (1 / npml) ** 2)  # first layer node, d = 1
    assert a[npml, npml + Px + 1] == pytest.approx(amax * (2 / npml) ** 2)
    assert a[0, 0] == pytest.approx(amax)                             # corner: max over axes
    assert a[1, 2] == pytest.approx(amax * (3 / npml) ** 2)
    assert np.max(a) == pytest.approx(amax)


# --------------------------------------------------------------------- operator
def test_operator_discrete_eigenpair():
    """With alpha = 0 and constant m, sin(p pi (i+1)/(n+1)) sin(q pi (k+1)/(n+1)) is an
    eigenvector of the Dirichlet 5-point Laplacian with eigenvalue
    (2 - 2 cos(p pi/(nx+1)) + 2 - 2 cos(q pi/(nz+1))) / h^2; the mass term subtracts
    omega^2 m^2 (Eq. 2)."""
    nx, nz, h, om, m = 13, 9, 7.0, 2 * np.pi * 3.0, 1 / 1800.0
    B = oracle.operator(np.full((nz, nx), m), h, om, np.zeros((nz, nx)))
    for p, q in [(1, 1), (3, 2), (nx, nz), (5, 8)]:
        i = np.arange(nx)
        k = np.arange(nz)
        v = np.outer(np.sin(q * np.pi * (k + 1) / (nz + 1)), np.sin(p * np.pi * (i + 1) / (nx + 1))).ravel()
        lam = (4 - 2 * np.cos(p * np.pi / (nx + 1)) - 2 * np.cos(q * np.pi / (nz + 1))) / h ** 2 - om ** 2 * m ** 2
        np.testing.assert_allclose(B @ v, lam * v, rtol=0, atol=1e-12 * np.abs(lam) * np.max(np.abs(v)) + 1e-18)


def _dense_by_loops(m_pad, h, om, alpha):
    """B assembled node by node: 4/h^2 - omega^2 m^2 (1 - j alpha) on the diagonal and
    -1/h^2 to each of the four neighbours that exist (Dirichlet ghosts elsewhere)."""
    nz, nx = m_pad.shape
    N = nx * nz
    B = np.zeros((N, N), np.complex128)
    for iz in range(nz):
        for ix in range(nx):
            r = iz * nx + ix
            B[r, r] = 4.0 / h ** 2 - om ** 2 * m_pad[iz, ix] ** 2 * (1 - 1j * alpha[iz, ix])
            for dx, dz in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                jx, jz = ix + dx, iz + dz
                if 0 <= jx < nx and 0 <= jz < nz:
                    B[r, jz * nx + jx] = -1.0 / h ** 2
    return B


def test_operator_matches_node_by_node_assembly_and_dense_solve():
    rng = _rng(1)
    Px, Pz, npml, h = 6, 8, 3, 10.0
    c = rng.uniform(1500, 3000, (Pz, Px))
    m_pad = oracle.pad_slowness(1 / c, npml)
    alpha = oracle.damping_profile(Px, Pz, npml, 0.5)
    om = 2 * np.pi * 11.0
    Bs = oracle.operator(m_pad, h, om, alpha).toarray()
    Bd = _dense_by_loops(m_pad, h, om, alpha)
    np.testing.assert_allclose(Bs, Bd, rtol=1e-15, atol=1e-20)
    # direct LU vs LAPACK dense solve, point source and random right-hand side
    src = np.array([[2, 1]])
    u = oracle.solve_fields(1 / c, h, om, src, npml, 0.5)[0].ravel()
    f = np.zeros(Bd.shape[0], complex)
    f[(1 + npml) * (Px + 2 * npml) + 2 + npml] = 1 / h ** 2
    ud = np.linalg.solve(Bd, f)
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-12
    F = models.random_complex(rng, (1, Bd.shape[0]))
    u2 = oracle.solve_fields(1 / c, h, om, src, npml, 0.5, F=F)[0].ravel()
    assert np.linalg.norm(u2 - np.linalg.solve(Bd, F[0])) / np.linalg.norm(u2) < 1e-12


def test_pad_is_edge_replication():
    m = np.arange(12.0).reshape(3, 4)
    p = oracle.pad_slowness(m, 2)
    assert p.shape == (7, 8)
    assert p[0, 0] == m[0, 0] and p[-1, -1] == m[-1, -1] and p[0, 5] == m[0, 3] and p[3, 0] == m[1, 0]
    np.testing.assert_array_equal(p[2:5, 2:6], m)


def test_manufactured_smooth_solution_second_order():
    """alpha = 0, constant m, u* = sin(pi x/L) sin(pi z/L) vanishing one node outside the
    grid: -Laplace u* - k^2 u* = (2 pi^2/L^2 - k^2) u*. The 5-point scheme converges at
    second order, so the error falls about 4x per halving of h (Eq. 2 with the
    standard finite-difference reading)."""
    L, c, f_hz = 1000.0, 2000.0, 1.5
    k2 = (2 * np.pi * f_hz / c) ** 2
    errs = []
    for n in (19, 39, 79):
        h = L / (n + 1)
        x = (np.arange(n) + 1) * h
        ustar = np.outer(np.sin(np.pi * x / L), np.sin(np.pi * x / L))
        F = ((2 * np.pi ** 2 / L ** 2 - k2) * ustar).reshape(1, -1)
        u = oracle.solve_fields(np.full((n, n), 1 / c), h, 2 * np.pi * f_hz, np.zeros((1, 2), int),
                                npml=0, F=F)[0]
        errs.append(np.max(np.abs(u - ustar)) / np.max(np.abs(ustar)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


def test_greens_function_far_from_source_and_layer():
    """Homogeneous medium: with the exp(+j omega t) convention that makes (1 - j alpha)
    absorbing, the outgoing solution of -Laplace G - k^2 G = delta is conj((j/4) H0^(1)(k r)).
    A thick layer keeps reflections small; agreement is limited by grid dispersion."""
    c, h, f_hz, Pn, npml = 2000.0, 5.0, 13.0, 121, 60     # about 31 points per wavelength
    mdl = models.homogeneous_model(Pn, Pn, h, c, [f_hz], [(Pn // 2, Pn // 2)], npml=npml, alpha_max=1.0)
    U = oracle.solve_fields(mdl.slowness, h, mdl.omegas[0], mdl.sources, npml, 1.0)[0]
    k = 2 * np.pi * f_hz / c
    iz, ix = np.meshgrid(np.arange(Pn), np.arange(Pn), indexing="ij")
    r = h * np.hypot(ix - Pn // 2, iz - Pn // 2)
    sel = (r >= 5 * h) & (r <= 40 * h)
    g = 0.25j * scipy.special.hankel1(0, k * r[sel])
    u = np.conj(U[npml:npml + Pn, npml:npml + Pn][sel])
    rel = np.abs(u - g) / np.abs(g)
    assert np.median(rel) < 0.03 and np.max(rel) < 0.08, (np.median(rel), np.max(rel))


def test_reciprocity_heterogeneous():
    """B is complex symmetric, so the field at x_r from a source at x_s equals the field
    at x_s from a source at x_r."""
    rng = _rng(2)
    Px, Pz, h = 30, 24, 10.0
    c = rng.uniform(1500, 3500, (Pz, Px))
    pts = np.array([[3, 2], [25, 2], [14, 20], [7, 11]])
    U = oracle.solve_fields(1 / c, h, 2 * np.pi * 9.0, pts, npml=8)
    d = oracle.sample_receivers(U, pts, 8)        # [src][rec]
    np.testing.assert_allclose(d, d.T, rtol=1e-10, atol=0)


# -------------------------------------------------------------------- gradient
def _small_fwi(seed=3):
    rng = _rng(seed)
    Px, Pz, h, npml = 24, 16, 10.0, 6
    c_true = rng.uniform(1800, 2600, (Pz, Px))
    c0 = np.full((Pz, Px), 2200.0)
    src = np.array([[3, 1], [12, 1], [20, 1]])
    rec = np.array([[i, 1] for i in range(0, Px, 3)])
    om = 2 * np.pi * np.array([9.0, 14.0])
    d_obs = np.stack([oracle.sample_receivers(oracle.solve_fields(1 / c_true, h, w, src, npml), rec, npml)
                      for w in om])
    return dict(m=1 / c0, h=h, omegas=om, src=src, rec=rec, d_obs=d_obs, lam=1e-3 * 2200.0 ** 2, npml=npml)


def test_gradient_central_differences():
    """The adjoint gradient equals central finite differences of J (Eq. 4) cell by cell,
    including edge cells whose value also fills the damping layer (E^T fold)."""
    p = _small_fwi()
    J, g = oracle.gradient(p["m"], p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"])
    assert J == pytest.approx(oracle.misfit(p["m"], p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"],
                                            p["lam"], p["npml"]), rel=1e-12)
    cells = [(0, 0), (0, 23), (15, 5), (7, 11), (3, 3), (15, 23)]
    for (iz, ix) in cells:
        m0 = p["m"][iz, ix]
        best = np.inf
        for rel_eps in (1e-3, 1e-4, 1e-5):
            e = rel_eps * m0
            mp = p["m"].copy(); mp[iz, ix] += e
            mm = p["m"].copy(); mm[iz, ix] -= e
            fd = (oracle.misfit(mp, p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"])
                  - oracle.misfit(mm, p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"])) / (2 * e)
            best = min(best, abs(fd - g[iz, ix]) / abs(g[iz, ix]))
        assert best < 1e-6, ((iz, ix), best)


def test_gradient_taylor_second_order():
    p = _small_fwi(5)
    J0, g = oracle.gradient(p["m"], p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"])
    dm = _rng(6).standard_normal(p["m"].shape) * p["m"] * 1e-2
    res = []
    for eps in (1.0, 0.5, 0.25):
        Je = oracle.misfit(p["m"] + eps * dm, p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"])
        res.append(abs(Je - J0 - eps * np.sum(g * dm)))
    assert 3.0 < res[0] / res[1] < 5.0 and 3.0 < res[1] / res[2] < 5.0, res


def test_adjoint_solve_dot_product():
    rng = _rng(7)
    Px, Pz, h, npml = 12, 10, 10.0, 4
    c = rng.uniform(1500, 3000, (Pz, Px))
    m_pad = oracle.pad_slowness(1 / c, npml)
    alpha = oracle.damping_profile(Px, Pz, npml, 0.5)
    fac = oracle.Factorised(m_pad, h, 2 * np.pi * 7.0, alpha)
    x = models.random_complex(rng, (1, m_pad.size))
    y = models.random_complex(rng, (1, m_pad.size))
    lhs = np.vdot(y, fac.solve(x))
    rhs = np.vdot(fac.solve_adjoint(y), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_fold_pad_sums_layer_onto_edge_cells():
    g = np.ones((4 + 6, 5 + 6))
    f = oracle.fold_pad(g, 3)
    assert f.sum() == g.sum()
    assert f[0, 0] == 16 and f[1, 1] == 1 and f[0, 2] == 4 and f[2, 0] == 4


# ------------------------------------------------------- planted mistakes are caught
def test_planted_mistakes_are_caught(monkeypatch):
    """Plant a sign error in the damping term and a wrong mass sign in the oracle; the
    Green's-function and eigenpair pins must fail for each."""
    good = H.operator

    def wrong_damping(m_pad, h, omega, alpha, rho_pad=None):
        return good(m_pad, h, omega, -alpha, rho_pad)

    monkeypatch.setattr(H, "operator", wrong_damping)
    with pytest.raises(AssertionError):
        test_greens_function_far_from_source_and_layer()

    def wrong_mass(m_pad, h, omega, alpha, rho_pad=None):
        return good(m_pad, h, 1j * omega, alpha, rho_pad)   # flips the sign of omega^2

    monkeypatch.setattr(H, "operator", wrong_mass)
    monkeypatch.setattr(oracle, "operator", wrong_mass)
    with pytest.raises(AssertionError):
        test_operator_discrete_eigenpair()


# ------------------------------------------------ variable density (Eq. 1)
def test_flux_laplacian_reduces_to_the_constant_density_operator():
    """rho = 1 gives the 5-point Laplacian of Eq. 2 exactly; rho = c scales it by c."""
    nz, nx = 7, 9
    lap = (sp.kron(sp.identity(nz), sp.diags([-np.ones(nx - 1), 2 * np.ones(nx), -np.ones(nx - 1)], [-1, 0, 1]))
           + sp.kron(sp.diags([-np.ones(nz - 1), 2 * np.ones(nz), -np.ones(nz - 1)], [-1, 0, 1]), sp.identity(nx)))
    assert abs(oracle.flux_laplacian(np.ones((nz, nx))) - lap).max() == 0.0
    assert abs(oracle.flux_laplacian(np.full((nz, nx), 2.5)) - 2.5 * lap).max() < 1e-14


def test_flux_laplacian_energy_by_loops():
    """u^T G u = sum over edges of rho_e |u_i - u_j|^2 (harmonic-mean rho_e) plus
    rho_i |u_i|^2 for every edge to a ghost node outside the grid, summed here edge by
    edge; G is symmetric."""
    rng = _rng(21)
    nz, nx = 5, 6
    rho = rng.uniform(0.5, 3.0, (nz, nx))
    u = rng.standard_normal((nz, nx))
    G = oracle.flux_laplacian(rho)
    assert abs(G - G.T).max() == 0.0
    e = 0.0
    for iz in range(nz):
        for ix in range(nx):
            for dz, dx in ((0, 1), (1, 0), (0, -1), (-1, 0)):
                jz, jx = iz + dz, ix + dx
                if 0 <= jz < nz and 0 <= jx < nx:
                    if (dz, dx) in ((0, 1), (1, 0)):          # each interior edge once
                        re = 2 * rho[iz, ix] * rho[jz, jx] / (rho[iz, ix] + rho[jz, jx])
                        e += re * (u[iz, ix] - u[jz, jx]) ** 2
                else:
                    e += rho[iz, ix] * u[iz, ix] ** 2
    assert float(u.ravel() @ (G @ u.ravel())) == pytest.approx(e, rel=1e-13)


def test_flux_laplacian_exact_across_a_density_jump():
    """With the density jump midway between two rows, -(rho u')' = 0 has the
    piecewise-linear solution of constant flux; the harmonic-mean edge makes the
    discrete operator vanish on it at every interior node (an arithmetic mean would
    not)."""
    nz, nx, k = 12, 5, 5                       # rows 0..k have rho1, rows k+1.. rho2
    rho1, rho2, q = 1.0, 4.0, 0.7
    z = np.arange(nz, dtype=float)
    zi = k + 0.5
    u_z = np.where(z <= zi, q * z / rho1, q * zi / rho1 + q * (z - zi) / rho2)
    rho = np.where(z[:, None] <= zi, rho1, rho2) * np.ones((nz, nx))
    u = np.repeat(u_z[:, None], nx, axis=1)
    r = (oracle.flux_laplacian(rho) @ u.ravel()).reshape(nz, nx)
    assert np.abs(r[1:-1, 1:-1]).max() < 1e-13
    # the arithmetic mean across the jump would leave a residual on the row above it
    ra = 0.5 * (rho1 + rho2)
    r_arith = rho1 * (u_z[k] - u_z[k - 1]) + ra * (u_z[k] - u_z[k + 1])
    assert abs(r_arith) > 0.5 * q


def test_density_gradient_central_differences():
    """With a density the slowness gradient keeps its form (rho enters B only) and
    still equals central differences of J."""
    p = _small_fwi()
    rho = _rng(22).uniform(1.0, 2.5, p["m"].shape)
    J, g = oracle.gradient(p["m"], p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"],
                           rho_phys=rho)
    for (iz, ix) in [(0, 0), (7, 11), (15, 23)]:
        e = 1e-4 * p["m"][iz, ix]
        mp = p["m"].copy(); mp[iz, ix] += e
        mm = p["m"].copy(); mm[iz, ix] -= e
        fd = (oracle.misfit(mp, p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"], rho_phys=rho)
              - oracle.misfit(mm, p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"],
                              rho_phys=rho)) / (2 * e)
        assert abs(fd - g[iz, ix]) / abs(g[iz, ix]) < 1e-6, ((iz, ix), fd, g[iz, ix])
