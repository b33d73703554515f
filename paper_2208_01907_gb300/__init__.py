"""GB300-native hybrid sparse factorization (arXiv 2208.01907, Alg. 1 and Alg. 2).

The compute path is libhf.so (hand-written CUDA for sm_103a behind a C ABI,
include/hf.h); this package only marshals arguments to it.
"""
from .hf import (  # noqa: F401
    HybridFactor, HFError, default_opts, lib, LIB_PATH, EXPORTED,
    HF_PREC_MIXED, HF_PREC_FP64, HF_PREC_FP32, HF_OK, HF_ERR_NOT_CONVERGED,
    factorize_batched, schur_batched, solve_batched,
)
