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
