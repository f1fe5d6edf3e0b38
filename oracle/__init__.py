"""CPU complex128 oracle for the shifted-Laplace Helmholtz path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or link
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA library; both sides take their inputs from ``synth``.

The oracle is the plain definition of what the method computes: the exact
discrete solution ``u = B^{-1} f`` of Eq. 2/3 by a direct sparse LU
factorisation (the paper, too, makes its observed data with a finite-difference
solve by LU factorisation, Examples section), and the exact derivative of the discrete
misfit of Eq. 4 by the adjoint formula behind Eq. 7.
"""
from .helmholtz import (  # noqa: F401
    damping_profile,
    flux_laplacian,
    fold_pad,
    gradient,
    misfit,
    operator,
    pad_slowness,
    point_sources,
    sample_receivers,
    solve_fields,
    Factorised,
)
from .gauss_newton import fwi_run, gn_hvp, gn_step  # noqa: F401,E402
