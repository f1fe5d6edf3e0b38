"""Plain, slow, obviously correct CPU oracle (complex128) for the 2D damped Helmholtz path.

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg; never by the product path.

What it computes (Kazemi, "Application of shifted-Laplace preconditioners for
heterogeneous Helmholtz equation - part 2: Full waveform inversion"):

* Eq. 2:  -Laplace(u) - omega^2 m^2 (1 - j alpha) u = f, m = 1/c the real slowness;
          with a density, Eq. 1:  -div(rho grad u) - omega^2 m^2 (1 - j alpha) u = f
          (rho as the paper writes it, multiplying the gradient), in 5-point flux
          form with harmonic-mean edge densities.
* Eq. 3:  the finite-difference matrix form  B u = f.
* Eq. 4:  J(m) = sum |u_obs - u_cal(m)|^2 + lambda |m|^2 over shots, receivers
          and frequencies (the paper's regulariser weight is also called alpha;
          here it is ``lam``).
* Eq. 7:  the gradient of J, formed with one adjoint solve per shot/frequency
          instead of the sensitivity matrix G.

Readings where the paper is silent (each also listed in the design notes):

* The discretisation is the standard second-order 5-point Laplacian on a
  uniform grid (h equal in x and z) with homogeneous Dirichlet ghosts one node
  outside the padded grid; the absorbing boundary is the damping term alpha of
  Eq. 2 inside an ``npml``-node layer on all four sides.
* alpha = alpha_max * (d / npml)^2 at a layer node d nodes from the physical
  edge (d = npml at the outermost node), max over the two axes in corners, 0 in
  the physical interior.
* The slowness in the layer copies the nearest physical value (map E); the
  gradient is taken with respect to the physical cells, so layer contributions
  are summed onto the edge cells (E^T).
* A point source of unit amplitude is f = 1/h^2 at its node.
* Eq. 7 omits the factor 2 and leaves the sign implicit; the exact derivative of
  the discrete J is used:
      dJ/dm_i = 4 omega^2 m_i Re[(1 - j alpha_i) u_i conj(lambda_i)] + 2 lam m_i,
      lambda = B^{-H} P^T (P u - d_obs).

The operator is assembled with scipy.sparse Kronecker sums of 1D second
differences; solves use SuperLU (``scipy.sparse.linalg.splu``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# --------------------------------------------------------------------------- model
def pad_slowness(m_phys: np.ndarray, npml: int) -> np.ndarray:
    """Extend the physical slowness [Pz][Px] into the damping layer by copying the
    nearest physical value (map E). The paper's Eq. 2 lives on the padded grid."""
    return np.pad(np.asarray(m_phys, dtype=np.float64), npml, mode="edge")


def damping_profile(Px: int, Pz: int, npml: int, alpha_max: float) -> np.ndarray:
    """alpha of Eq. 2 on the padded grid [Pz+2npml][Px+2npml].

    d = distance in nodes from the physical edge (0 inside), alpha = alpha_max (d/npml)^2,
    the larger of the x and z values in the corners.
    """
    nx, nz = Px + 2 * npml, Pz + 2 * npml
    alpha = np.zeros((nz, nx))
    if npml == 0:
        return alpha
    for iz in range(nz):
        dz = max(npml - iz, iz - (npml + Pz - 1), 0)
        for ix in range(nx):
            dx = max(npml - ix, ix - (npml + Px - 1), 0)
            d = max(dx, dz)
            alpha[iz, ix] = alpha_max * (d / npml) ** 2
    return alpha


def _second_difference(n: int) -> sp.csr_matrix:
    """1D tridiag(-1, 2, -1): minus the second difference with Dirichlet ghosts."""
    e = np.ones(n)
    return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], format="csr")


def flux_laplacian(rho_pad: np.ndarray) -> sp.csr_matrix:
    """h^2 times -div(rho grad) of Eq. 1 in 5-point flux form on the padded grid:
    row i holds sum_e rho_e on the diagonal and -rho_e for the neighbour across edge
    e, with rho_e the harmonic mean 2 rho_i rho_j / (rho_i + rho_j) of the two nodes.
    An edge to a node outside the grid (zero Dirichlet ghost) takes rho_i."""
    rho = np.asarray(rho_pad, np.float64)
    nz, nx = rho.shape
    N = nz * nx
    idx = np.arange(N).reshape(nz, nx)
    diag = np.zeros((nz, nx))
    rows, cols, vals = [], [], []
    for axis in (0, 1):                                   # z edges, then x edges
        a = rho[:-1, :] if axis == 0 else rho[:, :-1]
        b = rho[1:, :] if axis == 0 else rho[:, 1:]
        re = 2.0 * a * b / (a + b)
        ia = idx[:-1, :] if axis == 0 else idx[:, :-1]
        ib = idx[1:, :] if axis == 0 else idx[:, 1:]
        rows += [ia.ravel(), ib.ravel()]
        cols += [ib.ravel(), ia.ravel()]
        vals += [-re.ravel(), -re.ravel()]
        if axis == 0:
            diag[:-1, :] += re
            diag[1:, :] += re
        else:
            diag[:, :-1] += re
            diag[:, 1:] += re
    # edges to the ghost nodes around the grid
    diag[0, :] += rho[0, :]
    diag[-1, :] += rho[-1, :]
    diag[:, 0] += rho[:, 0]
    diag[:, -1] += rho[:, -1]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def operator(m_pad: np.ndarray, h: float, omega: float, alpha: np.ndarray, rho_pad=None) -> sp.csc_matrix:
    """B of Eq. 3 for Eq. 2 on the padded grid, unknowns ordered x fastest.

    B = (I_z (x) L_x + L_z (x) I_x) / h^2 - diag(omega^2 m^2 (1 - j alpha)),
    or, with a density (Eq. 1), flux_laplacian(rho) / h^2 - diag(...).
    """
    nz, nx = m_pad.shape
    if rho_pad is None:
        lap = sp.kron(sp.identity(nz), _second_difference(nx)) + sp.kron(_second_difference(nz), sp.identity(nx))
    else:
        lap = flux_laplacian(rho_pad)
    mass = (omega ** 2) * (m_pad ** 2) * (1.0 - 1j * alpha)
    B = lap.astype(np.complex128) / (h * h) - sp.diags(mass.ravel())
    return sp.csc_matrix(B)


def point_sources(nx: int, nz: int, h: float, src_pad: np.ndarray) -> np.ndarray:
    """Right-hand sides [ns][nz*nx]: a unit-amplitude point source is f = 1/h^2 at
    its node (the discrete delta). ``src_pad`` holds padded-grid (ix, iz)."""
    src_pad = np.asarray(src_pad).reshape(-1, 2)
    F = np.zeros((len(src_pad), nz * nx), np.complex128)
    for s, (ix, iz) in enumerate(src_pad):
        F[s, iz * nx + ix] = 1.0 / (h * h)
    return F


class Factorised:
    """One sparse LU factorisation of B(m, omega), reused for every right-hand side
    of that frequency (the paper models its data with a direct LU solve, Examples section)."""

    def __init__(self, m_pad: np.ndarray, h: float, omega: float, alpha: np.ndarray, rho_pad=None):
        self.shape = m_pad.shape
        self.B = operator(m_pad, h, omega, alpha, rho_pad)
        self.lu = spla.splu(self.B, permc_spec="MMD_AT_PLUS_A")

    def solve(self, F: np.ndarray) -> np.ndarray:
        """u = B^{-1} f for each row of F [k][N]."""
        F = np.atleast_2d(F)
        return self.lu.solve(np.ascontiguousarray(F.T)).T.copy()

    def solve_adjoint(self, F: np.ndarray) -> np.ndarray:
        """lambda = B^{-H} f for each row of F [k][N]."""
        F = np.atleast_2d(F)
        return self.lu.solve(np.ascontiguousarray(F.T), trans="H").T.copy()


def solve_fields(m_phys: np.ndarray, h: float, omega: float, src_phys: np.ndarray,
                 npml: int = 20, alpha_max: float = 0.5, F: np.ndarray | None = None, rho_phys=None) -> np.ndarray:
    """Wavefields u = B^{-1} f (Eq. 3) on the padded grid, one per source: [ns][nz][nx].

    ``src_phys`` holds physical-grid (ix, iz) node indices; ``F`` (optional,
    [k][nz*nx]) replaces the point sources by explicit right-hand sides; ``rho_phys``
    (optional, [Pz][Px]) is the density of Eq. 1, padded like the slowness.
    """
    Pz, Px = m_phys.shape
    m_pad = pad_slowness(m_phys, npml)
    alpha = damping_profile(Px, Pz, npml, alpha_max)
    nz, nx = m_pad.shape
    if F is None:
        F = point_sources(nx, nz, h, np.asarray(src_phys).reshape(-1, 2) + npml)
    rho_pad = None if rho_phys is None else pad_slowness(rho_phys, npml)
    fac = Factorised(m_pad, h, omega, alpha, rho_pad)
    return fac.solve(F).reshape(-1, nz, nx)


def sample_receivers(U: np.ndarray, rec_phys: np.ndarray, npml: int) -> np.ndarray:
    """d_cal = P u (Eq. 4): the wavefield at the receiver nodes. U is [..., nz, nx]."""
    rec = np.asarray(rec_phys).reshape(-1, 2) + npml
    return U[..., rec[:, 1], rec[:, 0]]


def fold_pad(g_pad: np.ndarray, npml: int) -> np.ndarray:
    """E^T: sum each layer node's value onto the physical cell it copies."""
    nz, nx = g_pad.shape
    Pz, Px = nz - 2 * npml, nx - 2 * npml
    g = np.zeros((Pz, Px))
    for iz in range(nz):
        pz = min(max(iz - npml, 0), Pz - 1)
        for ix in range(nx):
            px = min(max(ix - npml, 0), Px - 1)
            g[pz, px] += g_pad[iz, ix]
    return g


def misfit(m_phys, h, omegas, src_phys, rec_phys, d_obs, lam, npml=20, alpha_max=0.5, rho_phys=None) -> float:
    """J(m) of Eq. 4: sum over frequencies, shots and receivers of |d_cal - d_obs|^2
    plus lam * sum over physical cells of m^2. d_obs is [nf][ns][nrec]."""
    J = 0.0
    for f_i, om in enumerate(omegas):
        U = solve_fields(m_phys, h, om, src_phys, npml, alpha_max, rho_phys=rho_phys)
        r = sample_receivers(U, rec_phys, npml) - d_obs[f_i]
        J += float(np.sum(np.abs(r) ** 2))
    return J + lam * float(np.sum(np.asarray(m_phys, float) ** 2))


def gradient(m_phys, h, omegas, src_phys, rec_phys, d_obs, lam, npml=20, alpha_max=0.5, rho_phys=None):
    """(J, dJ/dm) for Eq. 4 by the adjoint method behind Eq. 7.

    Per frequency: u = B^{-1} f per shot; r_d = P u - d_obs; J += |r_d|^2;
    lambda = B^{-H} P^T r_d; g_pad += 4 omega^2 m Re[(1 - j alpha) u conj(lambda)].
    Then g = E^T g_pad + 2 lam m over physical cells. Returns (J, g [Pz][Px]).
    A density (Eq. 1) enters B only: the slowness derivative is the same.
    """
    m_phys = np.asarray(m_phys, np.float64)
    Pz, Px = m_phys.shape
    m_pad = pad_slowness(m_phys, npml)
    alpha = damping_profile(Px, Pz, npml, alpha_max)
    nz, nx = m_pad.shape
    src_pad = np.asarray(src_phys).reshape(-1, 2) + npml
    rec_pad = np.asarray(rec_phys).reshape(-1, 2) + npml
    rec_flat = rec_pad[:, 1] * nx + rec_pad[:, 0]
    J = 0.0
    g_pad = np.zeros(nz * nx)
    rho_pad = None if rho_phys is None else pad_slowness(rho_phys, npml)
    for f_i, om in enumerate(omegas):
        fac = Factorised(m_pad, h, om, alpha, rho_pad)
        U = fac.solve(point_sources(nx, nz, h, src_pad))          # [ns][N]
        r = U[:, rec_flat] - d_obs[f_i]                            # [ns][nrec]
        J += float(np.sum(np.abs(r) ** 2))
        adj = np.zeros_like(U)
        for s in range(U.shape[0]):
            np.add.at(adj[s], rec_flat, r[s])                      # P^T r_d
        lam_f = fac.solve_adjoint(adj)                             # B^{-H} P^T r_d
        w = (1.0 - 1j * alpha.ravel())
        g_pad += 4.0 * om ** 2 * m_pad.ravel() * np.sum(np.real(w * U * np.conj(lam_f)), axis=0)
    g = fold_pad(g_pad.reshape(nz, nx), npml) + 2.0 * lam * m_phys
    J += lam * float(np.sum(m_phys ** 2))
    return J, g
