"""GB300 (sm_103a) implementation of ChASE for pseudo-hermitian BSE Hamiltonians
(arXiv 2601.10557): a CUDA library with a C ABI (include/chase_bse.h) and this
thin Python binding."""
from ._lib import (ChaseBSEError, FP64, FP64_TC, MIXED_BF16X3, MIXED_BF16X6, MIXED_FP16X3, BSEEigvals,
                   alloc_count, degrees, dgemm_sliced, eig_general, eigh, eigvals, filter, filter_cols,
                   gemm_time, gemm_timer, grad, h2_blocks, filter_h2, has_mixed, launch_count, lib, rayleigh_ritz,
                   rayleigh_ritz_fallback, residuals, set_wait_limit, solve, strerror, trim_memory, LIB_PATH,
                   EXPORTS)

__all__ = ["ChaseBSEError", "FP64", "FP64_TC", "MIXED_BF16X3", "MIXED_BF16X6", "MIXED_FP16X3", "BSEEigvals",
           "alloc_count", "degrees", "dgemm_sliced", "eig_general", "eigh", "eigvals", "filter", "filter_cols",
           "gemm_time", "gemm_timer", "grad", "h2_blocks", "filter_h2", "has_mixed", "launch_count", "lib", "rayleigh_ritz",
           "rayleigh_ritz_fallback", "residuals", "set_wait_limit", "solve", "strerror", "trim_memory",
           "LIB_PATH", "EXPORTS"]
