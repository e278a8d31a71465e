"""GB300-native apply of a butterfly factorization (Li, Yang, Martin, Ho, Ying,
"Butterfly Factorization", arXiv 1502.01379).

The compute path is the CUDA library libbfly.so (csrc/, C ABI in
include/bfly.h); ``capi`` is its thin Python binding.  There is no CPU
fallback: loading raises if the library is missing.
"""
from .capi import (BF_C64, BF_C128, BF_ERR_CORRUPT, BF_ERR_CUDA, BF_ERR_INVALID, BF_ERR_NOMEM, BF_ERR_TIMEOUT,
                   BF_ERR_UNSUPPORTED, BF_OK, BfError, Plan, bf_apply, bf_apply_adjoint, bf_factor_file_check,
                   bf_factor_file_save, bf_plan_create_from_file,
                   bf_plan_check, bf_plan_create, bf_plan_destroy, bf_plan_device_bytes,
                   bf_plan_kernel_times, bf_plan_set_precision, bf_plan_set_profiling, bf_quad_apply, bf_quad_check,
                   bf_quad_create, bf_quad_destroy, bf_quad_device_bytes, bf_quad_set_precision, bf_status_string,
                   load)

__all__ = [
    "BF_C64", "BF_C128", "BF_OK", "BF_ERR_INVALID", "BF_ERR_CUDA", "BF_ERR_NOMEM", "BF_ERR_UNSUPPORTED",
    "BF_ERR_TIMEOUT", "BF_ERR_CORRUPT", "BfError", "Plan", "bf_factor_file_save", "bf_factor_file_check",
    "bf_plan_create_from_file", "bf_apply", "bf_apply_adjoint", "bf_plan_check",
    "bf_plan_create", "bf_plan_destroy", "bf_plan_device_bytes", "bf_plan_kernel_times",
    "bf_plan_set_profiling", "bf_plan_set_precision", "bf_status_string", "load", "bf_quad_create",
    "bf_quad_apply", "bf_quad_check", "bf_quad_set_precision", "bf_quad_device_bytes", "bf_quad_destroy",
]
