"""CPU restatement of the shifted-Laplace multigrid preconditioner (complex128).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA V-cycle; never by the
product path.

The paper preconditions its Krylov data-modelling engine with a shifted-Laplace
operator (Section "Full waveform inversion in the space-frequency domain", the
paragraph after Eq. 9; shift "1 + j" in Section "Examples"). It does not say how
the preconditioner is inverted. The reading used here, which the CUDA path
implements, is one geometric multigrid V(1,1)-cycle per application:

* M_l = 4 - (neighbours) - (h_l omega)^2 m_l^2 (beta1 - j beta2), the grid-scaled
  5-point shifted Laplacian on level l (no damping term), zero Dirichlet ghosts.
* Level l + 1 has floor(n/2) nodes per axis; coarse node I sits on fine node 2I+1;
  h_{l+1} = 2 h_l; coarse m^2 by injection. Coarsening stops once a level has at
  most 128 nodes or an axis has fewer than 4; the coarsest level is solved exactly.
* Pre-smoothing: one damped-Jacobi sweep from a zero guess, u = w_J D^-1 f.
* Restriction: full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] of the residual, times 4
  because the coarse grid-scaled system carries h_{l+1}^2 = 4 h_l^2.
* Prolongation: bilinear interpolation, then one post-smoothing Jacobi sweep.

Operators are explicit scipy.sparse matrices assembled node by node, so the
restatement shares nothing with the fused CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

COARSE_MAX = 128


def level_shapes(nx: int, nz: int):
    shapes = [(nx, nz)]
    while shapes[-1][0] * shapes[-1][1] > COARSE_MAX and shapes[-1][0] >= 4 and shapes[-1][1] >= 4:
        shapes.append((shapes[-1][0] // 2, shapes[-1][1] // 2))
    return shapes


def shifted_laplacian(m2: np.ndarray, hw2: float, beta: complex) -> sp.csr_matrix:
    """Grid-scaled M on one level: diagonal 4 - hw2 m^2 beta, -1 to each existing neighbour."""
    nz, nx = m2.shape
    rows, cols, vals = [], [], []
    for iz in range(nz):
        for ix in range(nx):
            r = iz * nx + ix
            rows.append(r); cols.append(r); vals.append(4.0 - hw2 * m2[iz, ix] * beta)
            for dx, dz in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                jx, jz = ix + dx, iz + dz
                if 0 <= jx < nx and 0 <= jz < nz:
                    rows.append(r); cols.append(jz * nx + jx); vals.append(-1.0)
    return sp.csr_matrix((np.asarray(vals, complex), (rows, cols)), shape=(nx * nz, nx * nz))


def prolongation(nxf: int, nzf: int) -> sp.csr_matrix:
    """Bilinear interpolation from the coarse level (floor(n/2) per axis, node I on fine
    2I+1) to the fine level; coarse values outside the coarse grid are zero."""
    nxc, nzc = nxf // 2, nzf // 2

    def weights(j, nc):
        if j % 2 == 1:
            return [((j - 1) // 2, 1.0)]
        return [(I, 0.5) for I in (j // 2 - 1, j // 2) if 0 <= I < nc]

    rows, cols, vals = [], [], []
    for jz in range(nzf):
        for jx in range(nxf):
            for Iz, wz in weights(jz, nzc):
                for Ix, wx in weights(jx, nxc):
                    if 0 <= Ix < nxc:
                        rows.append(jz * nxf + jx); cols.append(Iz * nxc + Ix); vals.append(wz * wx)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nxf * nzf, nxc * nzc))


def full_weighting(nxf: int, nzf: int) -> sp.csr_matrix:
    """(1/16)[1 2 1; 2 4 2; 1 2 1] centred on fine node (2I+1, 2K+1); fine nodes outside
    the grid contribute zero."""
    nxc, nzc = nxf // 2, nzf // 2
    rows, cols, vals = [], [], []
    for K in range(nzc):
        for I in range(nxc):
            for dz in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    jx, jz = 2 * I + 1 + dx, 2 * K + 1 + dz
                    if 0 <= jx < nxf and 0 <= jz < nzf:
                        rows.append(K * nxc + I); cols.append(jz * nxf + jx)
                        vals.append((2 - abs(dx)) * (2 - abs(dz)) / 16.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nxc * nzc, nxf * nzf))


class VCycle:
    """One V(1,1)-cycle approximating M^{-1} for grid-scaled (h omega)^2 = hw2."""

    def __init__(self, m2_pad: np.ndarray, hw2: float, beta=(1.0, 0.5), omega_jacobi: float = 0.8):
        nz, nx = m2_pad.shape
        self.wj = omega_jacobi
        bt = complex(beta[0], -beta[1])
        self.M, self.P, self.R, self.shapes = [], [], [], level_shapes(nx, nz)
        m2 = np.asarray(m2_pad, float)
        for l, (lx, lz) in enumerate(self.shapes):
            self.M.append(shifted_laplacian(m2, hw2 * 4.0 ** l, bt))
            if l + 1 < len(self.shapes):
                self.P.append(prolongation(lx, lz))
                self.R.append(full_weighting(lx, lz))
                m2 = m2[1::2, 1::2][: lz // 2, : lx // 2]
        self.coarse = spla.splu(sp.csc_matrix(self.M[-1]))

    def apply(self, f: np.ndarray, level: int = 0) -> np.ndarray:
        """z = V(f) for a flat complex vector on `level`."""
        if level == len(self.M) - 1:
            return self.coarse.solve(f)
        M = self.M[level]
        D = M.diagonal()
        u = self.wj * f / D
        r = f - M @ u
        e = self.apply(4.0 * (self.R[level] @ r), level + 1)
        u = u + self.P[level] @ e
        return u + self.wj * (f - M @ u) / D
