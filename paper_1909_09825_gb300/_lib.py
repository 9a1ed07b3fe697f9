"""ctypes loader for the in-tree libfgt1d.so (argument marshalling only).

The product path has no fallback: if the shared library is missing or fails to
load, every call raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfgt1d.so")

FGT1D_OK = 0
FGT1D_EINVAL = 1
FGT1D_EUNSUPPORTED = 2
FGT1D_ENONFINITE = 3
FGT1D_ENOMEM = 4
FGT1D_ETIMEOUT = 5
FGT1D_ECUDA = 6
FGT1D_EWORKSPACE = 7
FGT1D_ETOOLARGE = 8
FGT1D_FP64 = 0
FGT1D_FP32 = 1
FGT1D_EXACT_SELF = 2
FGT1D_F32X2 = 4
MAX_TERMS = 8
MAX_N = 16

_lib = None

# name -> (restype, argtypes); mirrors include/fgt1d.h
_P, _I, _I64, _D, _U, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint, ctypes.c_size_t
SIGNATURES = {
    "fgt1d_soe_cf": (_I, [_I, _P, _P, _P, _P, _P, _P]),
    "fgt1d_plan_create": (_I, [_D, _D, _U, _P]),
    "fgt1d_plan_create_soe": (_I, [_D, _I, _P, _P, _P, _P, _U, _P]),
    "fgt1d_plan_info": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fgt1d_plan_destroy": (None, [_P]),
    "fgt1d_workspace_size": (_I, [_P, _I64, _I64, _P]),
    "fgt1d_execute": (_I, [_P, _P, _I64, _P, _P, _I64, _P, _P, _SZ, _P]),
    "fgt1d_execute_profiled": (_I, [_P, _P, _I64, _P, _P, _I64, _P, _P, _SZ, _P, _P]),
    "fgt1d_workspace_size_host": (_I, [_P, _I64, _I64, _P]),
    "fgt1d_execute_host": (_I, [_P, _P, _I64, _P, _P, _I64, _P, _P, _SZ, _P]),
    "fgt1d_execute_host_async": (_I, [_P, _P, _I64, _P, _P, _I64, _P, _P, _SZ, _P]),
    "fgt1d_execute_noalloc": (_I, [_P, _P, _I64, _P, _P, _I64, _P, _P]),
    "fgt1d_batched_workspace_size": (_I, [_P, _I, _I64, _I64, _P]),
    "fgt1d_execute_batched": (_I, [_P, _I, _P, _P, _P, _P, _I64, _P, _P, _I64, _P, _P, _SZ, _P]),
    "fgt1d_backward_workspace_size": (_I, [_P, _I64, _I64, _P]),
    "fgt1d_backward": (_I, [_P, _P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "fgt1d_sort_workspace_size": (_I, [_I64, _I64, _P]),
    "fgt1d_sort_merged": (_I, [_P, _I64, _P, _I64, _P, _P, _SZ, _P]),
    "fgt1d_self_workspace_size": (_I, [_P, _I64, _P]),
    "fgt1d_execute_self": (_I, [_P, _P, _I64, _P, _P, _P, _SZ, _P]),
    "fgt1d_geometry_workspace_size": (_I, [_P, _I64, _I64, _P]),
    "fgt1d_geometry_bind": (_I, [_P, _P, _I64, _P, _I64, _P, _SZ, _P]),
    "fgt1d_geometry_apply": (_I, [_P, _I64, _I64, _P, _P, _P, _SZ, _P]),
    "fgt1d_plan_set_tile": (_I, [_P, _I]),
    "fgt1d_plan_get_tile": (_I, [_P, _P]),
    "fgt1d_autotune": (_I, [_P, _I, _P, _P, _P, _P, _I64, _P, _P, _I64, _P, _P, _SZ, _I, _P, _P, _P]),
    "fgt1d_segment_execute": (_I, [_P, _P, _I64, _P, _P, _I64, _P, _P, _P, _SZ, _P]),
    "fgt1d_segment_compose": (_I, [_P, _I, _I, _P, _P]),
    "fgt1d_segment_apply": (_I, [_P, _I64, _I64, _P, _P, _P, _SZ, _P]),
    "fgt1d_measure_peaks": (_I, [_P, _P]),
    "fgt1d_check": (_I, [_P, _SZ, _P]),
    "fgt1d_strerror": (ctypes.c_char_p, [_I]),
    "fgt1d_version": (_I, []),
}


def lib():
    """Load libfgt1d.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libfgt1d.so not built: run __graft_entry__.build() or paper_1909_09825_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class FGTError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = lib().fgt1d_strerror(code).decode()
        super().__init__("%s: %s (status %d)" % (where, msg, code) if where else "%s (status %d)" % (msg, code))


def check(code, where=""):
    if code != FGT1D_OK:
        raise FGTError(code, where)
