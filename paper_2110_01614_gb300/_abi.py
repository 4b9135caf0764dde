"""ctypes declarations of the nsdf C ABI (include/nsdf.h).

Argument marshalling only: every computation happens inside libnsdf.so.
Loading fails loudly when the library has not been built; there is no
fallback path.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnsdf.so")

NSDF_OK = 0
NSDF_ERR_INVALID_ARG = 1
NSDF_ERR_MISALIGNED = 2
NSDF_ERR_NOT_LOADED = 3
NSDF_ERR_OOM = 4
NSDF_ERR_CUDA = 5
NSDF_ERR_UNSUPPORTED = 6
NSDF_ERR_TIMEOUT = 7
NSDF_ERR_TOO_LARGE = 8

NSDF_FP32 = 0
NSDF_BF16 = 1
NSDF_FP16 = 2
NSDF_RAW_GRADIENT = 1


class nsdf_arch(ctypes.Structure):
    _fields_ = [("in_dim", ctypes.c_int), ("width", ctypes.c_int),
                ("n_hidden", ctypes.c_int), ("skip_layer", ctypes.c_int),
                ("beta", ctypes.c_float), ("activation", ctypes.c_int),
                ("ff_freqs", ctypes.c_int)]


NSDF_ACT_SOFTPLUS = 0
NSDF_ACT_RELU = 1


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_ST = ctypes.c_int

# name -> (restype, argtypes); every symbol include/nsdf.h declares
SIGNATURES = {
    "nsdf_num_params": (ctypes.c_size_t, [ctypes.POINTER(nsdf_arch)]),
    "nsdf_create": (_ST, [ctypes.POINTER(nsdf_arch), ctypes.c_int, ctypes.c_int,
                          ctypes.POINTER(ctypes.c_void_p)]),
    "nsdf_destroy": (_ST, [_P]),
    "nsdf_load_weights": (_ST, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int, _P]),
    "nsdf_query": (_ST, [_P, _P, _I64, _P, ctypes.c_uint32, _P]),
    "nsdf_collide": (_ST, [_P, _P, _I64, ctypes.c_float, _P, _P, _P, _P, _P]),
    "nsdf_collide_noalloc": (_ST, [_P, _P, _I64, ctypes.c_float, _P, _P, _P, _P, _P]),
    "nsdf_backward": (_ST, [_P, _P, _I64, _P, _P, _P, _P, _P]),
    "nsdf_query_grouped": (_ST, [_P, _P, _P, _P, _I64, ctypes.c_float, _P, _P, _P]),
    "nsdf_query_grouped_T": (_ST, [_P, _P, _P, _P, _I64, ctypes.c_float, _P, _P, _P, _P]),
    "nsdf_l1_grad": (_ST, [_P, _P, _I64, _P, _P, _P, _P]),
    "nsdf_autotune_grouped": (_ST, [_P, _P, _P, _P, _I64, ctypes.c_float, _P, _P, _P,
                                    ctypes.POINTER(ctypes.c_int)]),
    "nsdf_set_grouped_config": (_ST, [_P, ctypes.c_int, ctypes.c_int]),
    "nsdf_mesh_sdf": (_ST, [_P, _I64, _P, _I64, _P, _I64, _P, _P]),
    "nsdf_cloth_step": (_ST, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, _P]),
    "nsdf_sync_status": (_ST, [_P, _P]),
    "nsdf_status_string": (ctypes.c_char_p, [_ST]),
    "nsdf_voxel_build": (_ST, [_P, _I64, _P, _I64, ctypes.c_int, _P, _P, _P, _P]),
    "nsdf_voxel_collide": (_ST, [_P, ctypes.c_int, _P, _P, _P, _I64, ctypes.c_float, _P, _P, _P,
                                 _P]),
    "nsdf_debug_inject": (_ST, [_P, ctypes.c_int, ctypes.c_longlong]),
    "nsdf_debug_noalloc_limit": (_ST, [ctypes.c_size_t]),
    "nsdf_debug_fp32_fma_peak": (_ST, [ctypes.POINTER(ctypes.c_double), _P]),
    "nsdf_debug_tc16_one_cta": (_ST, [ctypes.c_int]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libnsdf.so once; raises if it is missing (build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"nsdf CUDA library not found at {path}; build it with "
            "`python -m paper_2110_01614_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
