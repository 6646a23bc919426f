"""ctypes loader of libtaser.so.  There is no fallback: if the library is missing the
import fails loudly, because every step of the detector runs in its CUDA kernels.

TASER_LIBRARY=debug in the environment loads the bounds-checked libtaser_debug.so
instead (same ABI; see taser_debug_report in include/taser.h)."""
import ctypes
import os

_LIBDIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib")
VARIANT = os.environ.get("TASER_LIBRARY", "release")
if VARIANT not in ("release", "debug"):
    raise ImportError("TASER_LIBRARY must be 'release' or 'debug' (got %r)" % VARIANT)
LIB_PATH = os.path.join(_LIBDIR, "libtaser_debug.so" if VARIANT == "debug" else "libtaser.so")

_c_i32, _c_i64, _c_f32, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p

# name -> (restype, argtypes); must match include/taser.h
SIGNATURES = {
    "taser_problem_size": (_c_i32, [_c_i32, _c_i32]),
    "taser_status_string": (ctypes.c_char_p, [_c_i32]),
    "taser_last_error": (ctypes.c_char_p, []),
    "taser_build_T": (_c_i32, [_c_i32, _c_i64, _c_i32, _c_i32, _vp, _vp, _c_f32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "taser_step_size": (_c_i32, [_c_i64, _c_i32, _vp, _c_i32, _c_f32, _vp, _vp, _vp]),
    "taser_detect": (_c_i32, [_c_i64, _c_i32, _vp, _vp, _vp, _c_i32, _c_i32, _c_i32, _vp, _vp, _vp, _vp]),
    "taser_detect_monitored": (_c_i32, [_c_i64, _c_i32, _vp, _vp, _vp, _c_i32, _c_i32, _c_i32, _c_f32, _vp, _vp,
                                        _vp, _vp, _vp]),
    "taser_host_workspace_bytes": (ctypes.c_size_t, [_c_i32, _c_i64, _c_i32, _c_i32]),
    "taser_run_host": (_c_i32, [_c_i32, _c_i64, _c_i32, _c_i32, _vp, _vp, _c_f32, _c_i32, _c_i32, _c_i32, _vp,
                                ctypes.c_size_t, _vp, _vp, _vp]),
    "taser_run_host_static": (_c_i32, [_c_i32, _c_i64, _c_i32, _c_i32, _vp, _vp, _c_f32, _c_i32, _c_i32, _c_i32,
                                       _vp, _vp, _vp]),
    "taser_unfolded_forward": (_c_i32, [_c_i64, _c_i32, _vp, _vp, _vp, _vp, _c_i32, _c_i32, _c_i32, _vp, _vp, _vp,
                                        _vp]),
    "taser_unfolded_backward": (_c_i32, [_c_i64, _c_i32, _vp, _vp, _vp, _vp, _c_i32, _c_i32, _c_i32, _vp, _vp, _vp,
                                         _vp, _vp]),
    "taser_uneven_workspace_bytes": (ctypes.c_size_t, [_c_i64]),
    "taser_detect_uneven": (_c_i32, [_c_i64, _vp, _vp, _vp, _vp, _c_i32, _c_i32, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                     _vp, _vp]),
    "taser_debug_report": (_c_i32, [_vp, _vp, _vp]),
    "taser_debug_drop_copy": (_c_i32, [_c_i64, _c_i32]),
}


class UnevenTuning(ctypes.Structure):
    """taser_uneven_tuning of include/taser.h."""
    _fields_ = [("blocks_per_sm", ctypes.c_int32 * 4), ("pop", ctypes.c_int32 * 4)]

# Capacity of the library's static device scratch (include/taser.h).
STATIC_SCRATCH_BYTES = 64 << 20

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "%s not found; build it with paper_1609_01797_gb300.build.build(%s) "
                "(the detector has no CPU fallback)" % (LIB_PATH, "debug=True" if VARIANT == "debug" else ""))
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


class TaserError(RuntimeError):
    def __init__(self, status, where):
        l = lib()
        msg = "%s failed: %s (%s)" % (where, l.taser_status_string(status).decode(),
                                      l.taser_last_error().decode())
        super().__init__(msg)
        self.status = status


def check(status, where):
    if status != 0:
        raise TaserError(status, where)
