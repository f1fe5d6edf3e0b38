"""CPU restatement of the Gauss-Newton step of Eq. 9 (complex128, sparse LU).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA Gauss-Newton
Hessian-vector product and step; never by the product path.

Eq. 8 writes the Hessian of the misfit of Eq. 4 as Re[G^T G + alpha I] plus a
second-order term that Gauss-Newton drops. With the misfit
J(m) = sum |P u(m) - d_obs|^2 + lam |m|^2 of this package (lam is the paper's
regulariser weight alpha), the Gauss-Newton Hessian is

    H = 2 Re[Jac^H Jac] + 2 lam I,     Jac dm = P B^{-1} [2 omega^2 m (1 - j alpha) u (E dm)],

Jac the Jacobian of the receiver data with respect to the physical slowness
(E copies a physical perturbation into the damping layer). H dm takes one
"Born" solve and one adjoint solve per shot and frequency: the two extra
modellings per iteration the paper counts (Section "Full waveform inversion in
the space-frequency domain", the paragraph after Eq. 9). The step solves
H dm = -g by conjugate gradients, as the paper does because H is dense.
"""
from __future__ import annotations

import numpy as np

from .helmholtz import Factorised, damping_profile, fold_pad, pad_slowness, point_sources


def gn_hvp(m_phys, h, omegas, src_phys, rec_phys, lam, dm, npml=20, alpha_max=0.5):
    """H dm for the Gauss-Newton Hessian at m_phys (physical [Pz][Px] arrays)."""
    m_phys = np.asarray(m_phys, np.float64)
    Pz, Px = m_phys.shape
    m_pad = pad_slowness(m_phys, npml)
    dm_pad = pad_slowness(np.asarray(dm, np.float64), npml)          # E dm: the same edge replication
    alpha = damping_profile(Px, Pz, npml, alpha_max).ravel()
    nz, nx = m_pad.shape
    src_pad = np.asarray(src_phys).reshape(-1, 2) + npml
    rec_pad = np.asarray(rec_phys).reshape(-1, 2) + npml
    rec_flat = rec_pad[:, 1] * nx + rec_pad[:, 0]
    h_pad = np.zeros(nz * nx)
    for om in omegas:
        fac = Factorised(m_pad, h, om, alpha.reshape(nz, nx))
        U = fac.solve(point_sources(nx, nz, h, src_pad))                 # forward fields [ns][N]
        born = 2.0 * om ** 2 * m_pad.ravel() * (1.0 - 1j * alpha) * dm_pad.ravel() * U
        dU = fac.solve(born)                                             # Born fields
        dd = dU[:, rec_flat]                                             # Jac dm at the receivers
        adj = np.zeros_like(U)
        for s in range(U.shape[0]):
            np.add.at(adj[s], rec_flat, dd[s])                           # P^T (Jac dm)
        w = fac.solve_adjoint(adj)                                       # B^{-H} P^T Jac dm
        h_pad += 4.0 * om ** 2 * m_pad.ravel() * np.sum(np.real((1.0 - 1j * alpha) * U * np.conj(w)), axis=0)
    return fold_pad(h_pad.reshape(nz, nx), npml) + 2.0 * lam * np.asarray(dm, np.float64)


def gn_step(m_phys, h, omegas, src_phys, rec_phys, lam, grad, iters, npml=20, alpha_max=0.5):
    """(dm, relative residuals) after `iters` conjugate-gradient iterations on
    H dm = -grad from dm = 0."""
    g = np.asarray(grad, np.float64)
    dm = np.zeros_like(g)
    r = -g.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    g0 = np.sqrt(rr)
    rel = [1.0]
    for _ in range(iters):
        if rr == 0.0:
            rel.append(0.0)
            continue
        hp = gn_hvp(m_phys, h, omegas, src_phys, rec_phys, lam, p, npml, alpha_max)
        a = rr / float(np.sum(p * hp))
        dm += a * p
        r -= a * hp
        rr_new = float(np.sum(r * r))
        rel.append(np.sqrt(rr_new) / g0)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return dm, np.array(rel)


def fwi_run(m0, h, omegas, src_phys, rec_phys, d_obs, lam, strategy="sequential", gn_iters=2, cg_iters=5,
            max_halvings=4, m_bounds=(1 / 6000.0, 1 / 1000.0), npml=20, alpha_max=0.5):
    """The Gauss-Newton inversion loop the paper's examples run (Section
    "Examples"): all frequencies at once ("simultaneous", its 1D example) or one
    at a time from the lowest, each starting from the previous model
    ("sequential", its 2D example). Each iteration: the gradient of Eq. 7 at the
    current model, the step dm of Eq. 9 by `cg_iters` CG iterations, then m + t dm
    (clipped to m_bounds) for the first t in 1, 1/2, ... (at most `max_halvings`
    halvings) whose misfit is below the current one; a group ends early when no
    t lowers it (the paper prints no line search: this backtracking is a reading).
    d_obs: [nf][ns][nrec]. Returns (m, J history): each group's J at its start and
    after every accepted iteration."""
    from .helmholtz import gradient, misfit

    omegas = np.asarray(omegas, np.float64)
    d_obs = np.asarray(d_obs, np.complex128)
    m = np.asarray(m0, np.float64).copy()
    if strategy == "simultaneous":
        groups = [list(range(len(omegas)))]
    else:
        groups = [[f] for f in np.argsort(omegas, kind="stable")]
    hist = []
    for grp in groups:
        om, d = omegas[grp], d_obs[grp]
        J = misfit(m, h, om, src_phys, rec_phys, d, lam, npml, alpha_max)
        hist.append(J)
        for _ in range(gn_iters):
            _, g = gradient(m, h, om, src_phys, rec_phys, d, lam, npml, alpha_max)
            dm, _ = gn_step(m, h, om, src_phys, rec_phys, lam, g, cg_iters, npml, alpha_max)
            t, accepted = 1.0, False
            for _ in range(max_halvings + 1):
                trial = np.clip(m + t * dm, m_bounds[0], m_bounds[1])
                Jt = misfit(trial, h, om, src_phys, rec_phys, d, lam, npml, alpha_max)
                if Jt < J:
                    m, J, accepted = trial, Jt, True
                    break
                t *= 0.5
            if not accepted:
                break
            hist.append(J)
    return m, np.array(hist)
