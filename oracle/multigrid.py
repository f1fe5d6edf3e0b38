"""CPU restatement of the shifted-Laplace multigrid preconditioner (complex128).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA preconditioner; never
by the product path.

The paper preconditions its Krylov data-modelling engine with a shifted-Laplace
operator (Section "Full waveform inversion in the space-frequency domain", the
paragraph after Eq. 9; shift "1 + j" in Section "Examples"). It does not say how
the preconditioner is inverted. The reading used here, which the CUDA path
implements, is one multigrid cycle per application:

* Finest level: M_0 = 4 - (neighbours) - (h omega)^2 m^2 (beta1 - j beta2), the
  grid-scaled 5-point shifted Laplacian (no damping term), zero Dirichlet ghosts;
  with a density (Eq. 1) the 5-point flux form of -div(rho grad) in its place.
* Level l + 1 has floor(n/2) nodes per axis; coarse node I sits on fine node
  2I+1. Coarsening stops once a level has at most 128 nodes or an axis has
  fewer than 4.
* Coarse operators are Galerkin products M_{l+1} = P^T M_l P with P bilinear
  interpolation; restriction is P^T (full weighting times 4).
* Smoother: damped Jacobi (default weight 0.5), one sweep before (from a zero
  guess) and one after each coarse correction.
* Cycle: a V-cycle on the levels above lf; from lf down, an F-cycle whose
  second coarse correction is a V-cycle; the coarsest level is solved exactly.
  With coarse="dense" (the library's default when beta2 != 0) the first level
  l >= 1 with at most 1200 nodes is solved exactly instead, and the cycle does
  not descend below it; coarse="tail" keeps the full hierarchy.
  lf (>= 1) is the first level whose spacing 2^l h gives k h >= 0.7 for the
  shortest wavelength (h omega 2^l m_max >= 0.7: fewer than about 9 nodes per
  wavelength), and no later than the first level with at most 24576 nodes.

Operators are explicit scipy.sparse matrices (Galerkin products by sparse
matrix multiplication), so the restatement shares nothing with the fused CUDA
kernels.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

COARSE_MAX = 128
TAIL_MAX = 24576
DENSE_MAX = 1200


def level_shapes(nx: int, nz: int):
    shapes = [(nx, nz)]
    while shapes[-1][0] * shapes[-1][1] > COARSE_MAX and shapes[-1][0] >= 4 and shapes[-1][1] >= 4:
        shapes.append((shapes[-1][0] // 2, shapes[-1][1] // 2))
    return shapes


def shifted_laplacian(m2: np.ndarray, hw2: float, beta: complex, rho=None) -> sp.csr_matrix:
    """Grid-scaled M on one level: diagonal 4 - hw2 m^2 beta, -1 to each existing neighbour;
    with a density (Eq. 1) the oracle's flux-form operator minus hw2 m^2 beta."""
    if rho is not None:
        from .helmholtz import flux_laplacian
        return (flux_laplacian(rho).astype(complex) - sp.diags(hw2 * beta * np.asarray(m2, float).ravel())).tocsr()
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


def tail_level(shapes) -> int:
    """First level (>= 1) with at most TAIL_MAX nodes: the F-cycle starts there."""
    for l in range(1, len(shapes)):
        if shapes[l][0] * shapes[l][1] <= TAIL_MAX:
            return l
    return len(shapes) - 1


FCYCLE_KH = 0.7


def fcycle_level(shapes, hw2: float, m_max: float) -> int:
    """First level of the F-cycle: the first l >= 1 with sqrt(hw2) 2^l m_max >= 0.7,
    at most tail_level(shapes) (hw2 = (h omega)^2 on the finest level)."""
    cap = tail_level(shapes)
    for l in range(1, cap):
        if np.sqrt(hw2) * 2.0 ** l * m_max >= FCYCLE_KH:
            return l
    return cap


class VCycle:
    """One preconditioner application approximating M^{-1} for grid-scaled (h omega)^2 = hw2."""

    def __init__(self, m2_pad: np.ndarray, hw2: float, beta=(1.0, 0.5), omega_jacobi: float = 0.5, rho_pad=None,
                 coarse: str = "dense"):
        nz, nx = m2_pad.shape
        self.wj = omega_jacobi
        bt = complex(beta[0], -beta[1])
        self.shapes = level_shapes(nx, nz)
        self.lt = fcycle_level(self.shapes, hw2, float(np.sqrt(np.max(m2_pad))))
        self.M = [shifted_laplacian(np.asarray(m2_pad, float), hw2, bt, rho_pad)]
        self.P = []
        for l, (lx, lz) in enumerate(self.shapes[:-1]):
            P = prolongation(lx, lz)
            self.P.append(P)
            self.M.append((P.T @ self.M[-1] @ P).tocsr())
        # the level solved exactly: the coarsest, or (coarse="dense", beta2 != 0) the first
        # level l >= 1 with at most DENSE_MAX nodes
        self.exact = len(self.M) - 1
        if coarse == "dense" and beta[1] != 0:
            self.exact = next(l for l in range(1, len(self.shapes)) if self.shapes[l][0] * self.shapes[l][1] <= DENSE_MAX)
        elif coarse not in ("dense", "tail"):
            raise ValueError(coarse)
        self.coarse = spla.splu(sp.csc_matrix(self.M[self.exact]))

    def cycle(self, f: np.ndarray, level: int, kind: str) -> np.ndarray:
        """kind 'V' or 'F' from `level` with a zero initial guess."""
        if level == self.exact:
            return self.coarse.solve(f)
        M, P = self.M[level], self.P[level]
        D = M.diagonal()
        u = self.wj * f / D
        sub = "F" if kind == "F" else ("F" if level + 1 == self.lt else "V")
        u = u + P @ self.cycle(P.T @ (f - M @ u), level + 1, sub)
        if kind == "F":
            u = u + P @ self.cycle(P.T @ (f - M @ u), level + 1, "V")
        return u + self.wj * (f - M @ u) / D

    def apply(self, f: np.ndarray) -> np.ndarray:
        """z = cycle(f) on the finest level: V above lt, F from lt down."""
        return self.cycle(f, 0, "F" if self.lt == 0 else "V")
