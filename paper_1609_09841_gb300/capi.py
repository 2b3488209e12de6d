"""ctypes declarations of libhermite's C ABI (include/hermite.h).

Argument marshalling only: every step of the half step runs in the CUDA
library.  Importing this module loads libhermite.so and raises if it is
missing -- there is no fallback implementation."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhermite.so")
DEBUG_LIB_PATH = os.path.join(_HERE, "libhermite_debug.so")

HERMITE_OK = 0
HERMITE_EINVAL = -1
HERMITE_ENOMEM = -2
HERMITE_ECUDA = -3
HERMITE_EUNSUPPORTED = -4
HERMITE_EUNSTABLE = -5
HERMITE_ETIMEOUT = -6
HERMITE_ENONFINITE = -7
HERMITE_ENOCONV = -8

HERMITE_FP64 = 0
HERMITE_FP32 = 1
HERMITE_3XTF32 = 2
HERMITE_SPLITBF16 = 3
HERMITE_HYBRID64 = 4
HERMITE_HYBRIDDF = 5
HERMITE_REMAINDER = 6
HERMITE_STATE_FP64 = 0
HERMITE_STATE_FP32 = 1
HERMITE_AUTO = 0
HERMITE_FUSED = 1
HERMITE_SPLIT = 2

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EUNSUPPORTED",
                -5: "EUNSTABLE", -6: "ETIMEOUT", -7: "ENONFINITE", -8: "ENOCONV"}


class HermiteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def load_library(path=LIB_PATH):
    """ctypes handle of a libhermite build (the release library by default;
    the debug build is libhermite_debug.so beside it), with every signature
    declared."""
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not built ({path}); run paper_1609_09841_gb300/build.py")
    lib = ctypes.CDLL(path)
    P, I, D, U, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint, ctypes.c_size_t
    IP, DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "hermite_plan": (I, [ctypes.POINTER(P), I, IP, DP, D, D, I, I, I]),
        "hermite_plan_taylor": (I, [ctypes.POINTER(P), I, IP, DP, D, D, I, I, I, I]),
        "hermite_step": (I, [P, P, P, I, P]),
        "hermite_adjoint_step": (I, [P, P, P, I, P]),
        "hermite_error": (I, [P, P, P, U, DP, P]),
        "hermite_state_elems": (S, [P]),
        "hermite_stability_limit": (D, [I]),
        "hermite_stability_limit_taylor": (D, [I, I]),
        "hermite_adv_plan": (I, [ctypes.POINTER(P), I, IP, DP, DP, D, I, I, I, I]),
        "hermite_adv_stability_limit": (D, [I, I]),
        "hermite_symbol_radius": (I, [I, I, D, DP, D, DP, DP]),
        "hermite_max_dt": (I, [I, I, D, DP, I, DP]),
        "hermite_max_radius": (I, [I, I, D, DP, D, I, DP]),
        "hermite_adv_max_radius": (I, [I, I, DP, DP, D, I, DP]),
        "hermite_adv_symbol_radius": (I, [I, I, DP, DP, D, DP, DP]),
        "hermite_adv_max_dt": (I, [I, I, DP, DP, I, DP]),
        "hermite_plan_operator": (I, [P, DP]),
        "hermite_destroy": (None, [P]),
        "hermite_step_dc": (I, [P, P, P, I, P]),
        "hermite_schedule_count": (I, [P]),
        "hermite_set_taylor_order": (I, [P, I]),
        "hermite_taylor_order": (I, [P]),
        "hermite_step_split_static": (I, [P, P, P, I, P]),
        "hermite_static_workspace_bytes": (S, []),
        "hermite_batch_plan": (I, [ctypes.POINTER(P), I, IP, IP, DP, DP, DP, I, I]),
        "hermite_batch_elems": (S, [P, I]),
        "hermite_batch_set_schedule": (I, [P, IP]),
        "hermite_batch_set_tiles": (I, [P, IP]),
        "hermite_batch_tile_shape": (I, [I, I, IP, IP]),
        "hermite_batch_step": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P), I, P]),
        "hermite_batch_run": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P), I, P]),
        "hermite_set_schedule": (I, [P, I, I]),
        "hermite_dot": (I, [P, P, P, DP, P]),
        "hermite_device_status": (I, [P, IP, P]),
        "hermite_inject_alloc_failure": (I, [ctypes.c_longlong, ctypes.c_longlong]),
        "hermite_debug_build": (I, []),
        "hermite_debug_status": (I, [P, IP, ctypes.POINTER(ctypes.c_ulonglong), P]),
        "hermite_debug_selftest": (I, [P, P, P, I, D, P]),
        "hermite_debug_wait_drill": (I, [P, P, P, I, P]),
        "hermite_record": (I, [P, P, P, I, P, P]),
        "hermite_inject": (I, [P, P, P, I, P, P]),
        "hermite_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load_library()


def last_error():
    return lib.hermite_last_error().decode()


def check(code):
    if code != HERMITE_OK:
        raise HermiteError(code, last_error())
    return code
