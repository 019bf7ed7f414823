"""GB300-native batched rigid-body kinematics and dynamics (sm_103a CUDA).

The public entry points mirror the C ABI in include/frax.h:
frax_model_create, frax_fk, frax_jacobian, frax_rnea, frax_crba, frax_aba, frax_aba_articulated,
frax_rnea_vjp, frax_aba_vjp, frax_ltdl_solve, frax_ltdl_inverse, frax_osc, frax_rnea_ext, frax_aba_ext, frax_fk_jvp, frax_rnea_jvp,
frax_aba_jvp, plus the autograd wrappers RneaFn / AbaFn.
"""

from .frax import (AbaFn, FraxError, Model, RneaFn, aba, frax_aba, frax_aba_articulated, frax_aba_vjp, frax_crba, frax_fk,
                   frax_jacobian, frax_last_error, frax_ltdl_inverse, frax_ltdl_solve, frax_model_create, frax_osc, frax_rnea_ext, frax_aba_ext,
                   frax_fk_jvp, frax_rnea_jvp, frax_aba_jvp, frax_fk_scan, frax_fp32_probe, frax_rnea, frax_rnea_vjp,
                   frax_serve_batch_noalloc, frax_version, lib, rnea)

__all__ = [
    "AbaFn", "FraxError", "Model", "RneaFn", "aba", "frax_aba", "frax_aba_articulated", "frax_aba_vjp", "frax_crba", "frax_fk",
    "frax_jacobian", "frax_last_error", "frax_ltdl_inverse", "frax_ltdl_solve", "frax_model_create", "frax_osc", "frax_rnea_ext", "frax_aba_ext",
    "frax_fk_jvp", "frax_rnea_jvp", "frax_aba_jvp", "frax_fk_scan", "frax_rnea", "frax_rnea_vjp",
    "frax_fp32_probe", "frax_serve_batch_noalloc", "frax_version",
    "lib", "rnea",
]
