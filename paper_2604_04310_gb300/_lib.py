"""ctypes declarations of libfrax.so (the C ABI in include/frax.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfrax.so")

c_f = ctypes.POINTER(ctypes.c_float)
c_i32 = ctypes.POINTER(ctypes.c_int32)
c_d = ctypes.POINTER(ctypes.c_double)
c_int = ctypes.c_int
c_i64 = ctypes.c_int64
c_vp = ctypes.c_void_p

# name -> (restype, argtypes)
SIGNATURES = {
    "frax_model_create": (c_int, [c_int, c_i32, c_i32, c_d, c_d, c_d, c_d, ctypes.POINTER(c_vp)]),
    "frax_model_destroy": (c_int, [c_vp]),
    "frax_model_dims": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "frax_model_kind": (c_int, [c_vp, ctypes.POINTER(c_int)]),
    "frax_model_set_tree_path": (c_int, [c_vp, c_int]),
    "frax_fk": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp]),
    "frax_jacobian": (c_int, [c_vp, c_i64, c_i64, c_vp, c_int, c_i32, c_vp, c_vp, c_vp]),
    "frax_rnea": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_crba": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "frax_aba": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_aba_articulated": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_debug_inject_fault": (c_int, [c_int, c_int]),
    "frax_fp32_probe": (c_int, [c_int, c_int, c_int, c_vp, ctypes.POINTER(ctypes.c_double), c_vp]),
    "frax_rnea_vjp": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_aba_vjp": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_ltdl_solve": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "frax_ltdl_inverse": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp]),
    "frax_rnea_ext": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_aba_ext": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_fk_scan": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp]),
    "frax_fk_jvp": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_int, c_vp, c_vp, c_vp]),
    "frax_rnea_jvp": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_aba_jvp": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_osc": (c_int, [c_vp, c_int, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "frax_server_create": (c_int, [c_i64, ctypes.c_double, ctypes.POINTER(c_vp)]),
    "frax_server_add_model": (c_int, [c_vp, c_vp, ctypes.POINTER(c_int)]),
    "frax_server_submit": (c_int, [c_vp, c_int, c_int, c_i64, ctypes.POINTER(c_vp), ctypes.POINTER(c_i64)]),
    "frax_server_poll": (c_int, [c_vp, c_i64, ctypes.POINTER(c_int)]),
    "frax_server_wait_any": (c_int, [c_vp, ctypes.c_double, ctypes.POINTER(c_i64)]),
    "frax_server_collect": (c_int, [c_vp, c_i64, ctypes.POINTER(c_vp), ctypes.POINTER(ctypes.c_double)]),
    "frax_server_info": (c_int, [c_vp, c_vp]),
    "frax_server_destroy": (c_int, [c_vp, c_int, ctypes.c_double]),
    "frax_server_replay": (c_int, [c_vp, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_i64),
                                   ctypes.POINTER(c_vp), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_vp),
                                   ctypes.POINTER(ctypes.c_double), ctypes.c_double]),
    "frax_serve_batch_noalloc": (c_int, [c_vp, c_int, c_vp]),
    "frax_last_error": (ctypes.c_char_p, []),
    "frax_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libfrax.so once and declares every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it first (python -m paper_2604_04310_gb300.build). "
            "This package has no CPU or Python fallback.")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
