"""Pins for the oracle's Gauss-Newton Hessian-vector product and step (Eq. 8, Eq. 9)
against facts that do not come from that code: symmetry, central differences of the
oracle gradient where the data residual vanishes (there the Gauss-Newton and full
Hessians coincide), central differences of the receiver data (v^T H v = 2|Jac v|^2 +
2 lam |v|^2), a dense solve of H assembled column by column, and a planted mistake."""
import numpy as np
import pytest

import oracle
from oracle import gauss_newton as GN


def _tiny(seed=11, at_truth=False):
    rng = np.random.default_rng(seed)
    Px, Pz, h, npml = 10, 8, 10.0, 4
    c_true = rng.uniform(1800, 2600, (Pz, Px))
    m_true = 1 / c_true
    m0 = m_true if at_truth else np.full((Pz, Px), 1 / 2200.0)
    src = np.array([[2, 1], [7, 1]])
    rec = np.array([[i, 1] for i in range(0, Px, 2)])
    om = 2 * np.pi * np.array([12.0, 19.0])
    d_obs = np.stack([oracle.sample_receivers(oracle.solve_fields(m_true, h, w, src, npml), rec, npml) for w in om])
    return dict(m=m0, h=h, omegas=om, src=src, rec=rec, d_obs=d_obs, lam=1e-3 * 2200.0 ** 2 * 1e-3, npml=npml)


def _hvp(p, v):
    return GN.gn_hvp(p["m"], p["h"], p["omegas"], p["src"], p["rec"], p["lam"], v, p["npml"])


def _grad(p, m):
    return oracle.gradient(m, p["h"], p["omegas"], p["src"], p["rec"], p["d_obs"], p["lam"], p["npml"])[1]


def _data(p, m):
    return np.stack([oracle.sample_receivers(oracle.solve_fields(m, p["h"], w, p["src"], p["npml"]), p["rec"],
                                             p["npml"]) for w in p["omegas"]])


def test_gn_hessian_is_symmetric_positive():
    p = _tiny()
    rng = np.random.default_rng(1)
    x = rng.standard_normal(p["m"].shape) * p["m"]
    y = rng.standard_normal(p["m"].shape) * p["m"]
    hx, hy = _hvp(p, x), _hvp(p, y)
    assert abs(np.sum(x * hy) - np.sum(y * hx)) <= 1e-10 * abs(np.sum(x * hy))
    assert np.sum(x * hx) > 0 and np.sum(y * hy) > 0


def test_gn_equals_gradient_differences_at_zero_residual():
    """With d_obs = P u(m) the residual is zero, the second term of Eq. 8 vanishes and
    H v is the directional derivative of the gradient."""
    p = _tiny(at_truth=True)
    v = np.random.default_rng(2).standard_normal(p["m"].shape) * p["m"]
    hv = _hvp(p, v)
    best = np.inf
    for eps in (1e-3, 1e-4):
        fd = (_grad(p, p["m"] + eps * v) - _grad(p, p["m"] - eps * v)) / (2 * eps)
        best = min(best, np.linalg.norm(fd - hv) / np.linalg.norm(hv))
    assert best < 1e-6, best


def test_gn_quadratic_form_matches_data_differences():
    """v^T H v = 2 |Jac v|^2 + 2 lam |v|^2 with Jac v from central differences of the data."""
    p = _tiny()
    v = np.random.default_rng(3).standard_normal(p["m"].shape) * p["m"]
    q = float(np.sum(v * _hvp(p, v)))
    eps = 1e-4
    jv = (_data(p, p["m"] + eps * v) - _data(p, p["m"] - eps * v)) / (2 * eps)
    ref = 2.0 * float(np.sum(np.abs(jv) ** 2)) + 2.0 * p["lam"] * float(np.sum(v * v))
    assert abs(q - ref) / ref < 1e-6, (q, ref)


def test_gn_step_matches_dense_solve():
    p = _tiny()
    p["lam"] = 1e4          # condition number ~1e3, so n CG iterations converge in floating point
    n = p["m"].size
    H = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n); e[k] = 1.0
        H[:, k] = _hvp(p, e.reshape(p["m"].shape)).ravel()
    g = _grad(p, p["m"])
    ref = np.linalg.solve(H, -g.ravel())
    dm, rel = GN.gn_step(p["m"], p["h"], p["omegas"], p["src"], p["rec"], p["lam"], g, n, p["npml"])
    assert rel[0] == 1.0 and rel[-1] < 1e-6
    assert np.linalg.norm(dm.ravel() - ref) / np.linalg.norm(ref) < 1e-5


def test_gn_planted_mistake_is_caught(monkeypatch):
    """Drop the damping factor (1 - j alpha) from the Born source: the zero-residual
    difference pin must fail (the perturbation reaches the layer through E)."""
    good = GN.gn_hvp

    def no_damping(m_phys, h, omegas, src, rec, lam, dm, npml=20, alpha_max=0.5):
        return good(m_phys, h, omegas, src, rec, lam, dm, npml, 0.0) if alpha_max else good(
            m_phys, h, omegas, src, rec, lam, dm, npml, alpha_max)

    monkeypatch.setattr(GN, "gn_hvp", no_damping)
    with pytest.raises(AssertionError):
        test_gn_equals_gradient_differences_at_zero_residual()


def _smooth_tiny(Px=10, Pz=8, amp=100.0):
    """A smooth background with a slow Gaussian anomaly; the background is the start."""
    h, npml = 10.0, 4
    X, Z = np.meshgrid(np.arange(Px) * h, np.arange(Pz) * h)
    c_bg = 2000.0 + 8.0 * Z
    c_true = c_bg - amp * np.exp(-((X - 5 * Px) ** 2 + (Z - 5 * Pz) ** 2) / (2 * 20.0 ** 2))
    return h, npml, 1 / c_bg, 1 / c_true


def test_fwi_loop_first_step_is_the_dense_gauss_newton_update():
    """One iteration of the oracle's inversion loop (no halving) on a smooth model is
    m0 + dm with dm the dense solve of H dm = -g (H assembled column by column), and it
    is kept because it lowers the misfit of Eq. 4, evaluated here directly."""
    h, npml, m0, m_true = _smooth_tiny()
    src = np.array([[2, 1], [7, 1]])
    rec = np.array([[i, 1] for i in range(0, m0.shape[1], 2)])
    om = 2 * np.pi * np.array([12.0, 19.0])
    d_obs = np.stack([oracle.sample_receivers(oracle.solve_fields(m_true, h, w, src, npml), rec, npml) for w in om])
    p = dict(m=m0, h=h, omegas=om, src=src, rec=rec, d_obs=d_obs, lam=1e2, npml=npml)   # CG converges in n steps
    n = m0.size
    H = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n); e[k] = 1.0
        H[:, k] = _hvp(p, e.reshape(m0.shape)).ravel()
    dm = np.linalg.solve(H, -_grad(p, m0).ravel()).reshape(m0.shape)
    m1, hist = GN.fwi_run(m0, h, om, src, rec, d_obs, p["lam"], strategy="simultaneous", gn_iters=1, cg_iters=n,
                          max_halvings=0, m_bounds=(1e-9, 1.0), npml=npml)
    J0 = oracle.misfit(m0, h, om, src, rec, d_obs, p["lam"], npml)
    Jt = oracle.misfit(m0 + dm, h, om, src, rec, d_obs, p["lam"], npml)
    assert Jt < J0
    assert hist[0] == pytest.approx(J0, rel=1e-12)
    assert len(hist) == 2 and hist[1] == pytest.approx(Jt, rel=1e-6)
    # n CG iterations leave a relative residual near 5e-8; with cond(H) near 1e3 the
    # step then agrees with the dense solve to about 5e-5
    assert np.linalg.norm(m1 - (m0 + dm)) / np.linalg.norm(dm) < 2e-4


def test_fwi_loop_sequential_goes_lowest_first_and_recovers_the_model():
    """Sequential use of the frequencies (the paper's 2D example): the first group is
    the lowest frequency whatever the input order, and the inversion moves the model
    towards the one that made the data and lowers the misfit over all frequencies."""
    Px, Pz, h, npml = 16, 12, 10.0, 4
    X, Z = np.meshgrid(np.arange(Px) * h, np.arange(Pz) * h)
    c_bg = 2000.0 + 8.0 * Z
    c_true = c_bg - 250.0 * np.exp(-((X - 80.0) ** 2 + (Z - 60.0) ** 2) / (2 * 25.0 ** 2))
    src = np.array([[2, 1], [8, 1], [13, 1]])
    rec = np.array([[i, 1] for i in range(Px)])
    om = 2 * np.pi * np.array([20.0, 11.0])                 # given highest first
    d_obs = np.stack([oracle.sample_receivers(oracle.solve_fields(1 / c_true, h, w, src, npml), rec, npml)
                      for w in om])
    lam = 1e-4
    m0 = 1 / c_bg
    m, hist = GN.fwi_run(m0, h, om, src, rec, d_obs, lam, strategy="sequential", gn_iters=3, cg_iters=6,
                         max_halvings=4, m_bounds=(1 / 4000.0, 1 / 1000.0), npml=npml)
    J_low = oracle.misfit(m0, h, om[1:], src, rec, d_obs[1:], lam, npml)
    assert hist[0] == pytest.approx(J_low, rel=1e-12)
    assert len(hist) >= 3
    m_true = 1 / c_true
    assert np.linalg.norm(m - m_true) < 0.8 * np.linalg.norm(m0 - m_true)
    J_all0 = oracle.misfit(m0, h, om, src, rec, d_obs, lam, npml)
    J_all = oracle.misfit(m, h, om, src, rec, d_obs, lam, npml)
    assert J_all < 0.5 * J_all0
