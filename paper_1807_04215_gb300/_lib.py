"""ctypes view of libgridspt.so (include/gridspt.h). Argument marshalling only."""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgridspt.so")

c_void_p = ctypes.c_void_p
c_int32 = ctypes.c_int32
c_size_t = ctypes.c_size_t
c_double = ctypes.c_double


class GridsptDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_max", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("form", ctypes.c_int32), ("box", ctypes.c_double), ("kcut_lin", ctypes.c_double),
                ("kcut_nl", ctypes.c_double), ("truncate", ctypes.c_int32), ("accum", ctypes.c_int32)]


class GridsptCosmo(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("h", ctypes.c_double), ("n_s", ctypes.c_double),
                ("sigma8", ctypes.c_double), ("gamma", ctypes.c_double)]


class GridsptKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


# name -> (restype, argtypes); the status enum is an int
SIGNATURES = {
    "gridspt_plan_create": (c_int32, [ctypes.POINTER(GridsptDesc), ctypes.POINTER(c_void_p)]),
    "gridspt_plan_destroy": (c_int32, [c_void_p]),
    "gridspt_workspace_size": (c_int32, [c_void_p, ctypes.POINTER(c_size_t)]),
    "gridspt_linear_amplitude": (c_int32, [ctypes.POINTER(GridsptCosmo), ctypes.POINTER(c_double)]),
    "gridspt_make_linear_field": (c_int32, [c_void_p, ctypes.POINTER(GridsptCosmo),
                                            ctypes.POINTER(ctypes.c_uint64), c_void_p, c_void_p]),
    "gridspt_run_orders": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gridspt_c2r": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "gridspt_r2c": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "gridspt_power_workspace_size": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_size_t)]),
    "gridspt_power": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, ctypes.POINTER(c_double),
                                c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gridspt_power_noalloc": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, ctypes.POINTER(c_double),
                                        c_void_p, c_void_p, c_void_p]),
    "gridspt_bispectrum_workspace_size": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_size_t)]),
    "gridspt_bispectrum": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, ctypes.POINTER(c_double),
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gridspt_growth_factor": (c_int32, [ctypes.POINTER(GridsptCosmo), c_double, ctypes.POINTER(c_double)]),
    "gridspt_sum_orders": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_double, c_void_p,
                                     c_void_p]),
    "gridspt_cross_correlation_workspace_size": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_size_t)]),
    "gridspt_cross_correlation": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, ctypes.POINTER(c_double),
                                            c_void_p, c_void_p, c_size_t, c_void_p]),
    "gridspt_bispectrum_triple": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                            ctypes.POINTER(c_double), c_void_p, c_void_p, c_void_p, c_size_t,
                                            c_void_p]),
    "gridspt_batch_create": (c_int32, [ctypes.POINTER(c_void_p), c_int32, ctypes.POINTER(c_void_p),
                                       ctypes.POINTER(c_int32), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                       ctypes.POINTER(c_size_t), ctypes.POINTER(c_void_p)]),
    "gridspt_batch_launch": (c_int32, [c_void_p, c_void_p]),
    "gridspt_multi_create": (c_int32, [ctypes.POINTER(c_void_p), c_int32, ctypes.POINTER(c_void_p),
                                       ctypes.POINTER(c_int32), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                       ctypes.POINTER(c_size_t), ctypes.POINTER(c_void_p)]),
    "gridspt_run_orders_multi": (c_int32, [c_void_p, c_void_p]),
    "gridspt_multi_destroy": (c_int32, [c_void_p]),
    "gridspt_batch_destroy": (c_int32, [c_void_p]),
    "gridspt_autotune_scratch_size": (c_int32, [c_void_p, ctypes.POINTER(c_size_t)]),
    "gridspt_autotune": (c_int32, [c_void_p, c_void_p, c_size_t, ctypes.POINTER(c_int32), c_void_p]),
    "gridspt_set_tuning": (c_int32, [c_void_p, ctypes.POINTER(c_int32)]),
    "gridspt_get_tuning": (c_int32, [c_void_p, ctypes.POINTER(c_int32)]),
    "gridspt_mlp_param_count": (c_int32, [c_int32, c_int32, c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "gridspt_mlp_forward": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p, c_int32, c_void_p,
                                      c_void_p, c_void_p]),
    "gridspt_mlp_backward_workspace_size": (c_int32, [c_int32, c_int32, c_int32, c_int32, ctypes.POINTER(c_size_t)]),
    "gridspt_mlp_backward": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p, c_int32, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gridspt_mlp_mse": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.c_int64, c_void_p, c_void_p, c_void_p]),
    "gridspt_mlp_adam": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                   ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   c_void_p]),
    "gridspt_mlp_convert": (c_int32, [c_void_p, c_void_p, c_int32, ctypes.c_int64, c_void_p]),
    "gridspt_check": (c_int32, [c_void_p, c_void_p]),
    "gridspt_selftest_bounded_wait": (c_int32, [c_void_p, c_void_p]),
    "gridspt_profile_begin": (c_int32, []),
    "gridspt_profile_end": (c_int32, [ctypes.POINTER(GridsptKernelStat), c_int32, ctypes.POINTER(c_int32)]),
    "gridspt_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path=LIB_PATH):
    """Load the library (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgridspt.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GridsptError(RuntimeError):
    def __init__(self, name, status, msg):
        super().__init__(f"{name} failed with status {status}: {msg}")
        self.status = status


def check(name, status):
    if status != 0:
        raise GridsptError(name, status, _lib.gridspt_last_error().decode(errors="replace"))
