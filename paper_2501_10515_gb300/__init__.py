"""GB300 ASCC / PLASCC amplitude-residual library (Python binding of libascc).

The binding only marshals arguments: every step of the residual, the update
and the iteration runs in libascc's CUDA kernels.  Importing the package does
not load the library; `load()` (called by the first Context) does, and fails
loudly when libascc.so has not been built.
"""
from .binding import (ASCC_FP64, ASCC_FP64_TC, ASCC_MIXED_BF16, AsccError, Context, Excitation,
                      Server, Options, Profile, Result, TwoAnsatzResult, default_options,
                      gemm_fp64_tc, gemm_split_bf16, gemm_split_bf16_noalloc, load, symbols,
                      autotuned_classes, t3p_plan_check, selftest_bounded_wait)

__all__ = ["ASCC_FP64", "ASCC_FP64_TC", "ASCC_MIXED_BF16", "AsccError", "Context", "Excitation",
           "Server", "Options", "Profile", "Result", "default_options", "gemm_fp64_tc",
           "gemm_split_bf16", "gemm_split_bf16_noalloc", "load", "symbols", "TwoAnsatzResult",
           "autotuned_classes", "t3p_plan_check", "selftest_bounded_wait"]
