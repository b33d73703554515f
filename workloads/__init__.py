"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 4).

This package only builds matrices, coordinates, right-hand sides and random
fields.  It holds none of the hybrid factorization's arithmetic (no scaling,
pivoting, Krylov or Schur step), so the CPU oracle and the CUDA path can both
draw their inputs from it without sharing any of the method.
"""
from .gen import (  # noqa: F401
    CsrSystem,
    diffusion2d,
    stokes3d,
    stokes3d_ldu,
    row_sign_form,
    elasticity3d,
    darcy2d,
    batched_systems,
    adjoint_diffusion2d,
    diffusion2d_structure,
    consistent_rhs,
    config_system,
)
