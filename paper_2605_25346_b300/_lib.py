"""ctypes binding of the C ABI in include/diffreach.h (argument marshalling only).

Every function keeps the C name.  Loading fails loudly when the in-tree library is
missing: there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdiffreach.so")

DR_OK = 0
DR_ERR_ARG, DR_ERR_SHAPE, DR_ERR_STATE, DR_ERR_OOM, DR_ERR_CUDA, DR_ERR_TIMEOUT, DR_ERR_NONFINITE = -1, -2, -3, -4, -5, -6, -7
DR_F32, DR_F64 = 0, 1
DR_SLOPE_ADAPTIVE, DR_SLOPE_CHORD, DR_SLOPE_ZERO, DR_SLOPE_USER = 0, 1, 2, 3
DR_PREC_AUTO, DR_PREC_SIMT, DR_PREC_TF32X3 = 0, 1, 2
DR_STATUS_NONFINITE, DR_STATUS_INFEASIBLE, DR_STATUS_MARGIN = 1, 2, 4
DR_KT_GEMM_ALL, DR_KT_GEMM_CHAIN, DR_KT_GEMM_FINAL, DR_KT_GEMM_OTHER, DR_KT_GEMM_REVERSE = 0, 1, 2, 3, 4

# every symbol the header declares
EXPORTS = [
    "dr_create", "dr_destroy", "dr_load_controller", "dr_load_dynamics", "dr_set_boxes", "dr_set_splits",
    "dr_set_horizon", "dr_set_step_offsets", "dr_get_shift_gradient", "dr_set_options", "dr_compute_bounds", "dr_get_objective", "dr_optimize_slopes",
    "dr_backward", "dr_get_weight_gradient", "dr_get_alpha", "dr_set_alpha", "dr_get_beta", "dr_set_beta", "dr_kernel_launches", "dr_graph_replays", "dr_kernel_timing", "dr_gemm_tuning_report", "dr_last_error",
    "dr_slope_gradient_static", "dr_tf32x3_gemm", "dr_check_wait_expiry",
]


class dr_split(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int32), ("layer", ctypes.c_int32), ("neuron", ctypes.c_int32), ("sign", ctypes.c_int32)]


class dr_static_args(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("widths", ctypes.c_int32 * 9), ("W", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("e", ctypes.c_void_p), ("D", ctypes.c_int64),
                ("H", ctypes.c_int32), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("alpha", ctypes.c_void_p),
                ("margin_rho", ctypes.c_double), ("dalpha", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("stream", ctypes.c_void_p)]


class dr_options(ctypes.Structure):
    _fields_ = [("slope_mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("margin_rho", ctypes.c_double),
                ("chunk_domains", ctypes.c_int64), ("mem_cap_bytes", ctypes.c_int64),
                ("box_margin", ctypes.c_double), ("tuning", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("timing", ctypes.c_int32), ("rigorous", ctypes.c_int32),
                ("weight_grad", ctypes.c_int32), ("reverse", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libdiffreach.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run paper_2605_25346_b300/build.py (no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dp, fp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
    sig = {
        "dr_create": (i32, [ctypes.POINTER(vp), i32, vp]),
        "dr_destroy": (None, [vp]),
        "dr_load_controller": (i32, [vp, i32, vp, vp, vp, i32]),
        "dr_load_dynamics": (i32, [vp, i32, i32, dp, dp, dp]),
        "dr_set_boxes": (i32, [vp, i64, dp, dp, i32]),
        "dr_set_splits": (i32, [vp, vp, vp, fp]),
        "dr_set_horizon": (i32, [vp, i32]),
        "dr_set_step_offsets": (i32, [vp, dp, i32]),
        "dr_get_shift_gradient": (i32, [vp, dp, i32]),
        "dr_set_options": (i32, [vp, ctypes.POINTER(dr_options)]),
        "dr_compute_bounds": (i32, [vp, dp, dp, dp, dp, vp, i32]),
        "dr_get_objective": (i32, [vp, dp, i32]),
        "dr_optimize_slopes": (i32, [vp, i32, ctypes.c_double, ctypes.c_double, dp]),
        "dr_backward": (i32, [vp, dp, dp, fp, fp, i32]),
        "dr_get_weight_gradient": (i32, [vp, dp, dp, i32]),
        "dr_get_alpha": (i32, [vp, fp, i32]),
        "dr_set_alpha": (i32, [vp, fp, i32]),
        "dr_get_beta": (i32, [vp, fp, i32]),
        "dr_set_beta": (i32, [vp, fp, i32]),
        "dr_kernel_launches": (i64, [vp]),
        "dr_graph_replays": (i64, [vp]),
        "dr_gemm_tuning_report": (i64, [ctypes.c_char_p, i64]),
        "dr_kernel_timing": (i32, [vp, i32, i64, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
        "dr_last_error": (ctypes.c_char_p, [vp]),
        "dr_slope_gradient_static": (i32, [ctypes.POINTER(dr_static_args)]),
        "dr_tf32x3_gemm": (i32, [i32, i32, i32, vp, vp, vp, vp]),
        "dr_check_wait_expiry": (i32, [ctypes.c_double]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class DiffReachError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def check(ctx, code: int):
    if code != DR_OK:
        msg = load().dr_last_error(ctx)
        raise DiffReachError(code, msg.decode() if msg else "")
    return code
