"""GB300 (sm_103a) implementation of ChASE for pseudo-hermitian BSE Hamiltonians
(arXiv 2601.10557): a CUDA library with a C ABI (include/chase_bse.h) and this
thin Python binding."""
from ._lib import (ChaseBSEError, FP64, MIXED_BF16X3, MIXED_BF16X6, MIXED_FP16X3, alloc_count, BSEEigvals, eigvals, filter, grad, lib, rayleigh_ritz,
                   residuals, solve, strerror, LIB_PATH, EXPORTS, launch_count, has_mixed, dgemm_sliced,
                   trim_memory)

__all__ = ["ChaseBSEError", "FP64", "MIXED_BF16X3", "MIXED_BF16X6", "MIXED_FP16X3", "alloc_count", "BSEEigvals", "eigvals", "filter", "grad", "lib",
           "rayleigh_ritz", "residuals", "solve", "strerror", "LIB_PATH", "EXPORTS", "launch_count", "has_mixed",
           "dgemm_sliced", "trim_memory"]
