"""ctypes binding of libse (include/se.h): argument marshalling only.

Every function here has the name and argument order of the C entry point it
calls.  Device arrays are passed as torch CUDA tensors (their data pointers),
host arrays as numpy arrays.  There is no CPU fallback: if the library has not
been built, or no CUDA device is present, calls raise.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libse.so")

SE_OK = 0
SE_WARN_NONNEUTRAL = 1
SE_ERR_ARG = -1
SE_ERR_CUDA = -2
SE_ERR_NOMEM = -3
SE_ERR_UNSUPPORTED = -4
SE_ERR_CUFFT = -5
SE_ERR_NONFINITE = -6
SE_FP64 = 0
SE_FP32 = 1
SE_FP32_PLAIN = 2
SE_QUANTITY_POTENTIAL = 0
SE_QUANTITY_ENERGY = 1
SE_QUANTITY_FORCE = 2
SE_FORCE_ANALYTIC = 0
SE_FORCE_IK = 1
SE_PROBE_FP32_FMA = 0
SE_PROBE_FP64_FMA = 1
SE_PROBE_SMEM_ATOMIC_U32 = 2
SE_PROBE_SMEM_ATOMIC_F32 = 3

# name -> (restype, argtypes)
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "se_plan_create": (_i, [ctypes.POINTER(_vp), _i64, _d, _d, _i, _i]),
    "se_plan_destroy": (_i, [_vp]),
    "se_plan_set_precision": (_i, [_vp, _i]),
    "se_plan_set_shape": (_i, [_vp, _d, _i]),
    "se_plan_set_prefactor": (_i, [_vp, _d]),
    "se_plan_set_stream": (_i, [_vp, _vp]),
    "se_plan_set_tuning": (_i, [_vp, _i, _i]),
    "se_plan_set_force_mode": (_i, [_vp, _i]),
    "se_plan_get_params": (_i, [_vp, _dp]),
    "se_spread": (_i, [_vp, _vp, _vp]),
    "se_scale": (_i, [_vp, _vp]),
    "se_gather": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "se_energy_force": (_i, [_vp, _vp, _vp, _dp, _vp, _vp]),
    "se_adjoint": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "se_energy_force_host": (_i, [_vp, _vp, _vp, _dp, _vp, _vp]),
    "se_copy_grid": (_i, [_vp, _i, _vp]),
    "se_self_energy": (_i, [_vp, _vp, _i64, _dp]),
    "se_evaluate": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "se_plan_get_status": (_i, [_vp, ctypes.POINTER(_i)]),
    "se_plan_set_graph": (_i, [_vp, _i]),
    "se_plan_set_timing": (_i, [_vp, _i]),
    "se_plan_get_timing": (_i, [_vp, _dp, _i, ctypes.POINTER(_i64), _i]),
    "se_spread_noalloc": (_i, [_vp, _vp, _i64, _d, _d, _i, _i, _vp, _vp]),
    "se_batch_create": (_i, [ctypes.POINTER(_vp), _i, _vp, _vp, _vp, _d, _i]),
    "se_batch_destroy": (_i, [_vp]),
    "se_batch_set_stream": (_i, [_vp, _vp]),
    "se_batch_set_prefactor": (_i, [_vp, _d]),
    "se_batch_set_tile": (_i, [_vp, _i]),
    "se_batch_set_graph": (_i, [_vp, _i]),
    "se_batch_evaluate": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "se_batch_grid_energy": (_i, [_vp, _vp]),
    "se_batch_get_status": (_i, [_vp, ctypes.POINTER(_i)]),
    "se_batch_set_timing": (_i, [_vp, _i]),
    "se_batch_get_timing": (_i, [_vp, _dp, _i, ctypes.POINTER(_i64), _i]),
    "se_batch_autotune": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_i),
                               ctypes.POINTER(ctypes.c_float)]),
    "se_real_create": (_i, [ctypes.POINTER(_vp), _i64, _d, _d, _d]),
    "se_real_destroy": (_i, [_vp]),
    "se_real_set_precision": (_i, [_vp, _i]),
    "se_real_set_prefactor": (_i, [_vp, _d]),
    "se_real_set_stream": (_i, [_vp, _vp]),
    "se_real_get_cells": (_i, [_vp, ctypes.POINTER(_i)]),
    "se_real_set_reach": (_i, [_vp, _i]),
    "se_real_evaluate": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i]),
    "se_select_params": (_i, [_i, _d, _d, _d, _d, _d, _dp, ctypes.POINTER(_i),
                              ctypes.POINTER(_i), _dp]),
    "se_select_support": (_i, [_d, _d]),
    "se_lambert_w0": (_d, [_d]),
    "se_strerror": (ctypes.c_char_p, [_i]),
    "se_probe_peak": (_i, [_i, ctypes.POINTER(_d)]),
    "se_version": (_i, []),
}

_lib = None


class SEError(RuntimeError):
    def __init__(self, status, where):
        super().__init__("%s: %s (status %d)" % (where, strerror(status), status))
        self.status = status


def load(path=None):
    """Load libse.so (raises OSError with a clear message if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError("libse.so not built (%s); run __graft_entry__.build() or "
                      "python paper_1712_04718_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(status):
    try:
        return load().se_strerror(int(status)).decode()
    except OSError:
        return "status %d" % status


def check(status, where):
    """Raise SEError for a negative status; return the status otherwise."""
    if status < 0:
        raise SEError(status, where)
    return status
