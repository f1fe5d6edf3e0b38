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
