"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package draws velocity models, acquisition geometry and random vectors. It
holds none of the method's arithmetic (no operator, no solver, no gradient), so
that both sides of every parity check can take their inputs from it without
sharing any of the computation being checked.
"""
from .models import (  # noqa: F401
    Model,
    c1_model,
    c2_model,
    c3_model,
    c4_models,
    c5_request,
    homogeneous_model,
    random_complex,
    layered_model,
)
