"""Pins for the CPU restatement of the multigrid preconditioner (oracle/multigrid.py).

The restatement is checked against facts independent of its code: full weighting
is a quarter of the transpose of bilinear interpolation, interpolation is exact
for linear functions, the V-cycle used as a stationary iteration converges to
the direct solution of M u = f, and damped Jacobi damps the checkerboard mode.
"""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import multigrid as mg
from synth import models


def test_level_shapes_rule():
    assert mg.level_shapes(141, 141)[-1] == (8, 8)
    assert mg.level_shapes(441, 241) == [(441, 241), (220, 120), (110, 60), (55, 30), (27, 15), (13, 7)]
    assert mg.level_shapes(1041, 1041)[-1] == (8, 8)
    s = mg.level_shapes(1064, 1064)
    assert all(a[0] // 2 == b[0] for a, b in zip(s, s[1:]))


def test_full_weighting_is_quarter_transpose_of_bilinear():
    for nx, nz in [(9, 7), (10, 8), (17, 12), (6, 11)]:
        P = mg.prolongation(nx, nz).toarray()
        R = mg.full_weighting(nx, nz).toarray()
        np.testing.assert_allclose(R, P.T / 4.0, rtol=0, atol=1e-15)


def test_bilinear_reproduces_linear_functions():
    nx, nz = 21, 15
    nxc, nzc = nx // 2, nz // 2
    Xc, Zc = np.meshgrid(2 * np.arange(nxc) + 1.0, 2 * np.arange(nzc) + 1.0)
    a, b, c = 0.3, -1.7, 2.2
    u = mg.prolongation(nx, nz) @ (a + b * Xc + c * Zc).ravel()
    X, Z = np.meshgrid(np.arange(nx, dtype=float), np.arange(nz, dtype=float))
    exact = a + b * X + c * Z
    inner = (X >= 1) & (X <= 2 * nxc - 1) & (Z >= 1) & (Z <= 2 * nzc - 1)
    np.testing.assert_allclose(u.reshape(nz, nx)[inner], exact[inner], rtol=0, atol=1e-12)


def test_galerkin_coarse_operator_closed_form():
    """For constant coefficients, P^T M P of the grid-scaled 5-point Laplacian with bilinear
    P is the textbook 9-point stencil (1/4)[-1 -2 -1; -2 12 -2; -1 -2 -1], and P^T diag(c) P is
    c times the tensor square of the 1D stencil [1/4, 3/2, 1/4] (interior nodes)."""
    nx = nz = 41
    c = 3.7e-7
    V = mg.VCycle(np.full((nz, nx), c), 0.0)                      # hw2 = 0: pure Laplacian
    M1 = V.M[1].toarray()
    n1 = nx // 2
    i = (n1 // 2) * n1 + n1 // 2
    lap = {(0, 0): 3.0, (1, 0): -0.5, (0, 1): -0.5, (1, 1): -0.25, (-1, 1): -0.25}
    for (dx, dz), v in lap.items():
        assert abs(M1[i, i + dz * n1 + dx] - v) < 1e-14
        assert abs(M1[i, i - dz * n1 - dx] - v) < 1e-14
    P = mg.prolongation(nx, nz)
    K1 = (P.T @ (c * P)).toarray() / c
    one = {0: 1.5, 1: 0.25, -1: 0.25}
    for dz in (-1, 0, 1):
        for dx in (-1, 0, 1):
            assert abs(K1[i, i + dz * n1 + dx] - one[dx] * one[dz]) < 1e-14


def test_tail_level_rule():
    assert mg.tail_level(mg.level_shapes(1041, 1041)) == 3      # 130 x 130 = 16900 nodes
    assert mg.tail_level(mg.level_shapes(441, 241)) == 2        # 110 x 60
    assert mg.tail_level(mg.level_shapes(141, 141)) == 1        # 70 x 70


def test_vcycle_iteration_converges_to_direct_solution():
    rng = np.random.default_rng(4)
    mdl = models.c1_model()
    m_pad = np.pad(mdl.slowness, 20, mode="edge")
    hw2 = (mdl.h * mdl.omegas[0]) ** 2
    V = mg.VCycle(m_pad ** 2, hw2, beta=(1.0, 0.5))
    M = V.M[0]
    f = models.random_complex(rng, M.shape[0])
    exact = spla.spsolve(M.tocsc(), f)
    u = np.zeros_like(f)
    errs = []
    for _ in range(200):
        u = u + V.apply(f - M @ u)
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    assert errs[-1] < 1e-6, errs[::20]
    # contracting until round-off
    assert all(b < a for a, b in zip(errs[::20], errs[20::20]) if a > 1e-12)


def test_jacobi_damps_checkerboard():
    nx = nz = 33
    m2 = np.full((nz, nx), (1 / 2000.0) ** 2)
    M = mg.shifted_laplacian(m2, (10.0 * 2 * np.pi * 5.0) ** 2, complex(1.0, -0.5))
    D = M.diagonal()
    X, Z = np.meshgrid(np.arange(nx), np.arange(nz))
    e = ((-1.0) ** (X + Z)).ravel().astype(complex)
    e2 = e - 0.8 * (M @ e) / D       # error propagation of one sweep for M u = 0
    assert np.linalg.norm(e2) < 0.7 * np.linalg.norm(e)


def test_fcycle_level_rule():
    """The F-cycle starts at the first level where the shortest wavelength has
    k h >= 0.7, never later than the node-count level: 1041^2 at h = 5 m, 15 Hz and
    1950 m/s gives k h = 0.48 on level 1, 0.97 on level 2 and 1.93 on level 3."""
    shapes = mg.level_shapes(1041, 1041)
    hw2 = (5.0 * 2 * np.pi * 15.0) ** 2
    assert mg.tail_level(shapes) == 3
    assert mg.fcycle_level(shapes, hw2, 1 / 1950.0) == 2
    assert mg.fcycle_level(shapes, hw2 / 100, 1 / 1950.0) == 3     # 1.5 Hz: capped by the node count
    assert mg.fcycle_level(shapes, hw2 * 4, 1 / 1950.0) == 1        # 30 Hz: k h = 0.97 on level 1


def test_density_cycle_converges_to_direct_solution():
    """With a density (Eq. 1) the finest operator is the flux form; the Galerkin
    hierarchy built from it still gives a convergent stationary iteration, and a unit
    density leaves the cycle exactly as without one."""
    rng = np.random.default_rng(5)
    mdl = models.c1_model()
    m_pad = np.pad(mdl.slowness, 20, mode="edge")
    nz, nx = m_pad.shape
    z = np.arange(nz)[:, None] * np.ones((1, nx))
    rho = np.where(z < nz // 2, 1.0, 2.5) + 0.3 * np.sin(np.arange(nx)[None, :] / 7.0)
    hw2 = (mdl.h * mdl.omegas[0]) ** 2
    V = mg.VCycle(m_pad ** 2, hw2, beta=(1.0, 0.5), rho_pad=rho)
    M = V.M[0]
    f = models.random_complex(rng, M.shape[0])
    exact = spla.spsolve(M.tocsc(), f)
    u = np.zeros_like(f)
    for _ in range(200):
        u = u + V.apply(f - M @ u)
    assert np.linalg.norm(u - exact) / np.linalg.norm(exact) < 1e-6
    V1 = mg.VCycle(m_pad ** 2, hw2, beta=(1.0, 0.5), rho_pad=np.ones_like(rho))
    V0 = mg.VCycle(m_pad ** 2, hw2, beta=(1.0, 0.5))
    assert np.array_equal(V1.apply(f), V0.apply(f))


def test_dense_level_rule():
    """With a complex shift the first level below the finest with at most 1200 nodes is
    solved exactly (32^2 for 1041^2, 27 x 15 for 441 x 241, 17^2 for the padded small case);
    without the imaginary part of the shift the coarsest level is."""
    hw2 = (5.0 * 2 * np.pi * 15.0) ** 2
    shapes = mg.level_shapes(1041, 1041)
    first = next(l for l in range(1, len(shapes)) if shapes[l][0] * shapes[l][1] <= 1200)
    assert shapes[first] == (32, 32) and first == 5
    assert mg.level_shapes(441, 241)[4] == (27, 15)
    small = mg.VCycle(np.full((141, 141), (1 / 2000.0) ** 2), hw2, beta=(1.0, 0.5))
    assert small.shapes[small.exact] == (17, 17)
    assert mg.VCycle(np.full((141, 141), (1 / 2000.0) ** 2), hw2, beta=(1.0, 0.0)).exact == len(small.shapes) - 1


def test_dense_level_is_solved_exactly_and_the_cycle_converges():
    """The level the dense coarse end solves returns M_l^{-1} f, checked against a dense
    LAPACK solve of the assembled level matrix (not the oracle's own sparse LU), and the
    cycle with that coarse end, used as a stationary iteration, converges to the direct
    solution of M u = f like the cycle with the coarsest level exact."""
    rng = np.random.default_rng(7)
    mdl = models.c1_model()
    m_pad = np.pad(mdl.slowness, 20, mode="edge")
    hw2 = (mdl.h * mdl.omegas[0]) ** 2
    V = mg.VCycle(m_pad ** 2, hw2, beta=(1.0, 0.5), coarse="dense")
    T = mg.VCycle(m_pad ** 2, hw2, beta=(1.0, 0.5), coarse="tail")
    assert V.exact < T.exact
    Ml = V.M[V.exact].toarray()
    g = models.random_complex(rng, Ml.shape[0])
    e = V.cycle(g, V.exact, "V")
    assert np.linalg.norm(e - np.linalg.solve(Ml, g)) < 1e-12 * np.linalg.norm(e)
    M = V.M[0]
    f = models.random_complex(rng, M.shape[0])
    exact = spla.spsolve(M.tocsc(), f)
    for cyc in (V, T):
        u = np.zeros_like(f)
        for _ in range(200):
            u = u + cyc.apply(f - M @ u)
        assert np.linalg.norm(u - exact) < 1e-6 * np.linalg.norm(exact)
    # one application differs between the two coarse ends (the dense one is exact lower down)
    assert np.linalg.norm(V.apply(f) - T.apply(f)) > 1e-8 * np.linalg.norm(T.apply(f))


def test_second_coarse_correction_right_hand_side():
    """The F-cycle's second coarse correction at level l solves for
    P^T (f - M_l (wj D^-1 f + P e)), e the first correction. Because the coarse operator
    is the Galerkin product P^T M_l P and the restriction is P^T, this equals
    f_{l+1} - M_{l+1} e with f_{l+1} = P^T (f - M_l wj D^-1 f) (level l + 1 data only),
    and it vanishes when the first correction solved level l + 1 exactly. The CUDA cycle
    uses both facts (it forms the right-hand side on level l + 1 and does nothing above
    the dense level); here they are checked on the oracle's assembled operators against
    the textbook form, which the oracle's cycle keeps."""
    rng = np.random.default_rng(11)
    mdl = models.c1_model()
    m_pad = np.pad(mdl.slowness, 20, mode="edge")
    hw2 = (mdl.h * mdl.omegas[0]) ** 2
    V = mg.VCycle(m_pad ** 2, hw2, beta=(1.0, 0.5), omega_jacobi=0.5, coarse="dense")
    for l in range(V.exact):
        M, P, Mc = V.M[l], V.P[l], V.M[l + 1]
        D = M.diagonal()
        f = models.random_complex(rng, M.shape[0])
        e = models.random_complex(rng, Mc.shape[0])
        u1 = V.wj * f / D
        fc = P.T @ (f - M @ u1)
        textbook = P.T @ (f - M @ (u1 + P @ e))
        assert np.linalg.norm(textbook - (fc - Mc @ e)) < 1e-12 * np.linalg.norm(textbook), l
        if l + 1 == V.exact:
            e_exact = V.cycle(fc, l + 1, "V")
            r2 = P.T @ (f - M @ (u1 + P @ e_exact))
            assert np.linalg.norm(r2) < 1e-12 * np.linalg.norm(fc)
    # a planted mistake is seen: the identity fails if the coarse operator is not P^T M P
    M, P = V.M[0], V.P[0]
    e = models.random_complex(rng, P.shape[1])
    wrong = 1.01 * V.M[1]
    assert np.linalg.norm(P.T @ (M @ (P @ e)) - wrong @ e) > 1e-3 * np.linalg.norm(wrong @ e)
