"""ctypes declarations of the C ABI in include/mps.h (argument marshalling only).

The shared library is built in-tree by ``build.py``; if it is missing this
module raises ImportError: there is no fallback implementation.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmps_gb300.so")

MPS_OK = 0
MPS_E_ARG = -1
MPS_E_NOMEM = -2
MPS_E_CUDA = -3
MPS_E_TIMEOUT = -4
MPS_E_STATE = -5
MPS_E_UNSUPPORTED = -6

MPS_PREC_FP64 = 0
MPS_PREC_MIXED = 1
MPS_POLICY_CANON = 0
MPS_POLICY_LOCAL = 1
MPS_TRUNC_QRCP = 0
MPS_TRUNC_SVD = 1
MPS_TRUNC_RQRCP = 2
MPS_HOST_C128 = 0
MPS_HOST_C64 = 1
MPS_FLAG_PROFILE = 1
MPS_FLAG_TENSOR_CORES = 2
MPS_FLAG_AUTOTUNE = 4
MPS_FLAG_NO_GRAPH = 8
MPS_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024

KCLASS = ["theta", "panel", "update", "norms", "formq", "split", "other", "canon", "svd"]

ERROR_NAMES = {0: "MPS_OK", -1: "MPS_E_ARG", -2: "MPS_E_NOMEM", -3: "MPS_E_CUDA",
               -4: "MPS_E_TIMEOUT", -5: "MPS_E_STATE", -6: "MPS_E_UNSUPPORTED"}


class mps_c128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class mps_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("policy", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("panel_width", ctypes.c_int),
                ("wait_timeout_s", ctypes.c_double), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p), ("flags", ctypes.c_int),
                ("debug_barrier_extra", ctypes.c_int), ("debug_max_ctas", ctypes.c_int),
                ("truncation", ctypes.c_int), ("sketch_seed", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class mps_tune_result(ctypes.Structure):
    _fields_ = [("panel_width", ctypes.c_int), ("panel_ctas", ctypes.c_int), ("candidates", ctypes.c_int),
                ("ms", ctypes.c_double), ("default_ms", ctypes.c_double)]


class mps_kstat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double), ("alg_flops", ctypes.c_double)]


KCLASS_COUNT = 9

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "mps_version": (_I, []),
    "mps_selftest_gemm": (_I, [_I, _I, _I, _I, _I, _I, _I, _I, _I, _I, ctypes.c_uint,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "mps_config_init": (None, [ctypes.POINTER(mps_config)]),
    "mps_create": (_I, [ctypes.POINTER(_P), _I, _I]),
    "mps_create_ex": (_I, [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(mps_config)]),
    "mps_destroy": (_I, [_P]),
    "mps_apply_1q": (_I, [_P, _I, ctypes.POINTER(mps_c128)]),
    "mps_apply_2q": (_I, [_P, _I, ctypes.POINTER(mps_c128), _I]),
    "mps_swap": (_I, [_P, _I, _I]),
    "mps_apply_2q_routed": (_I, [_P, _I, _I, ctypes.POINTER(mps_c128), _I]),
    "mps_apply_layer": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(mps_c128), _I, _I]),
    "mps_permute": (_I, [_P, ctypes.POINTER(_I), _I, ctypes.POINTER(ctypes.c_longlong)]),
    "mps_permute_layers": (_I, [_P, ctypes.POINTER(_I), _I, ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(_I)]),
    "mps_amplitude": (_I, [_P, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(mps_c128)]),
    "mps_fidelity_estimate": (_I, [_P, ctypes.POINTER(ctypes.c_double)]),
    "mps_overlap": (_I, [_P, _P, ctypes.POINTER(mps_c128)]),
    "mps_bond_dims": (_I, [_P, ctypes.POINTER(_I)]),
    "mps_get_site": (_I, [_P, _I, _I, _P, ctypes.c_size_t]),
    "mps_set_site": (_I, [_P, _I, _I, _I, _I, _P]),
    "mps_set_centre": (_I, [_P, _I]),
    "mps_get_centre": (_I, [_P, ctypes.POINTER(_I)]),
    "mps_move_centre": (_I, [_P, _I]),
    "mps_discarded_weight": (_I, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "mps_svd_last_stats": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong)]),
    "mps_apply_mpo": (_I, [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(mps_c128), _I]),
    "mps_set_stream": (_I, [_P, _P]),
    "mps_sync": (_I, [_P]),
    "mps_last_error": (ctypes.c_char_p, [_P]),
    "mps_kernel_stats": (_I, [_P, ctypes.POINTER(mps_kstat)]),
    "mps_kernel_stats_reset": (_I, [_P]),
    "mps_layer_stats": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(_I)]),
    "mps_two_site_workspace": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "mps_two_site_apply": (_I, [_I, _I, _I, _I, _I, _P, _P, ctypes.POINTER(mps_c128), _P, _P,
                                _P, _P, ctypes.c_size_t, _P]),
    "mps_two_site_apply_noalloc": (_I, [_I, _I, _I, _I, _I, _P, _P, ctypes.POINTER(mps_c128), _P, _P,
                                        _P, _P]),
    "mps_debug_raw_wait": (_I, [_I, ctypes.c_double]),
    "mps_tune_two_site": (_I, [_I, _I, _I, _I, _I, _I, ctypes.POINTER(mps_tune_result)]),
    "mps_last_split_pivots": (_I, [_P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
}

CHECKED_LIB_PATH = os.path.join(HERE, "_build_checked", "libmps_gb300_checked.so")

_lib = None
_checked = None


def _open(path):
    if not os.path.exists(path):
        raise ImportError("%s not built; run paper_2505_06119_gb300/build.py or __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path=LIB_PATH):
    global _lib
    if _lib is None:
        _lib = _open(path)
    return _lib


def load_checked():
    """The bounds-checking build of the library (compiled with -DMPS_BOUNDS_CHECK)."""
    global _checked
    if _checked is None:
        _checked = _open(CHECKED_LIB_PATH)
    return _checked
