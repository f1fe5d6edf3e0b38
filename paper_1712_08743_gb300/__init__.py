"""GB300-native shifted-Laplace Helmholtz solver and FWI gradient (arXiv 1712.08743).

The compute path is the CUDA library ``_build/libhelm.so`` behind the C ABI of
``include/helm.h``; this package is its Python binding (same names).
"""
from ._lib import (  # noqa: F401
    HELM_E_BUSY, HELM_E_CUDA, HELM_E_INVALID, HELM_E_NOMEM, HELM_E_NOT_CONVERGED, HELM_E_TIMEOUT, HELM_OK,
    HELM_PENDING, HELM_KRYLOV_BICGSTAB, HELM_KRYLOV_FGMRES, HELM_PREC_FP32, HELM_PREC_FP64, HELM_PREC_MIXED,
    HELM_FWI_SEQUENTIAL, HELM_FWI_SIMULTANEOUS, HELM_PRECOND_MG, HELM_PRECOND_NONE, HELM_REORTH_ALWAYS,
    HELM_REORTH_IFNEEDED, HELM_REORTH_NEVER, HELM_COARSE_AUTO, HELM_COARSE_DENSE, HELM_COARSE_FUSED, HELM_COARSE_TAIL, HelmError, load,
)
from .api import (  # noqa: F401
    Context, Model, helm_adjoint_gradient, helm_apply, helm_create_model, helm_ctx_create, helm_ctx_destroy,
    helm_default_opts, helm_destroy_model, helm_fwi_backward, helm_fwi_forward, helm_fwi_run, helm_gn_hvp,
    helm_gn_step, helm_poll, helm_release, helm_serve_config, helm_solve, helm_submit, helm_vcycle,
)
