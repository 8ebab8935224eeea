"""ctypes declarations of the C ABI in include/epic.h (argument marshalling
only: every step of the imaging and calibration runs in libepic.so)."""
from __future__ import annotations

import ctypes as ct
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libepic.so")

# epic_status
EPIC_OK = 0
STATUS_NAMES = {
    0: "EPIC_OK", 1: "EPIC_ERR_INVALID_ARG", 2: "EPIC_ERR_GRID_TOO_SMALL", 3: "EPIC_ERR_CUDA",
    4: "EPIC_ERR_OOM", 5: "EPIC_ERR_NUMERIC", 6: "EPIC_ERR_TIMEOUT", 7: "EPIC_ERR_UNSUPPORTED",
    8: "EPIC_ERR_STATE",
}
EPIC_KERNEL_GAUSSIAN, EPIC_KERNEL_TOPHAT = 0, 1
EPIC_IN_CI4, EPIC_IN_COMPLEX64 = 0, 1
EPIC_PREC_FP32, EPIC_PREC_FP16, EPIC_PREC_BF16 = 0, 1, 2
EPIC_PATH_AUTO, EPIC_PATH_FUSED, EPIC_PATH_UNFUSED, EPIC_PATH_CLUSTER, EPIC_PATH_PIPED = 0, 1, 2, 3, 4

# every exported entry point, as declared in include/epic.h
EXPORTS = [
    "epic_plan_create", "epic_plan_destroy", "epic_plan_set_stream", "epic_plan_get_info",
    "epic_set_gains", "epic_image", "epic_image_host", "epic_image_host_static",
    "epical_configure", "epical_update", "epical_average_channels",
    "epic_plan_sync", "epical_get_gains", "epical_get_state", "epical_set_state",
    "epic_plan_get_grid_table", "epic_unpack_ci4", "epic_last_error",
    "epic_set_gains_device", "epic_image_backward", "epic_autotune", "epic_graph_capture",
    "epic_graph_launch", "epic_measure_fma_peak", "epical_configure_pixels",
    "epical_get_direction_gains", "epic_visibilities", "epic_visibility_solve", "epical_fit_bandpass",
    "epic_set_phase_centre", "epic_plan_set_wait_limit", "epic_plan_set_adjoint_precision",
]

c_dp = ct.POINTER(ct.c_double)
c_fp = ct.POINTER(ct.c_float)
c_ip = ct.POINTER(ct.c_int)
c_u8p = ct.POINTER(ct.c_ubyte)


class PlanDesc(ct.Structure):
    _fields_ = [
        ("n_ant", ct.c_int), ("ant_xy_m", c_dp),
        ("n_chan", ct.c_int), ("freq_hz", c_dp),
        ("grid_n", ct.c_int), ("cell_wavelengths", ct.c_double),
        ("kernel", ct.c_int), ("kernel_support", ct.c_int), ("kernel_param", ct.c_double),
        ("input", ct.c_int), ("voltage_scale", c_fp),
        ("flags", c_u8p),
        ("precision", ct.c_int),
        ("cuda_stream", ct.c_void_p),
        ("path", ct.c_int),
        ("workspace_bytes", ct.c_size_t),
        ("kernel_param_ant", c_dp),
        ("batch_persistent", ct.c_int),
    ]


class PlanInfo(ct.Structure):
    _fields_ = [
        ("n_ant", ct.c_int), ("n_chan", ct.c_int), ("grid_n", ct.c_int),
        ("kernel_support", ct.c_int), ("window_rows", ct.c_int),
        ("cal_kx", ct.c_int), ("cal_ky", ct.c_int), ("ctas", ct.c_int),
        ("units_per_chan", ct.c_int), ("smem_bytes", ct.c_size_t),
        ("frames_pending", ct.c_longlong), ("iteration", ct.c_longlong),
        ("path", ct.c_int), ("batch_time", ct.c_int),
    ]


class TuneResult(ct.Structure):
    _fields_ = [
        ("path", ct.c_int), ("units_target", ct.c_int), ("batch_time", ct.c_int),
        ("cols_target", ct.c_int), ("ms_default", ct.c_double), ("ms_best", ct.c_double),
        ("candidates", ct.c_int), ("row_table", ct.c_int), ("row_frames", ct.c_int),
        ("batch_persistent", ct.c_int),
    ]


class EpicError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None) -> ct.CDLL:
    """Load libepic.so (built by build.py) and declare its signatures.
    Raises if the library is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libepic.so not built ({path}); run __graft_entry__.build()")
    lib = ct.CDLL(path)
    P = ct.c_void_p
    sig = {
        "epic_plan_create": [ct.POINTER(P), ct.POINTER(PlanDesc)],
        "epic_plan_destroy": [P],
        "epic_plan_set_stream": [P, P],
        "epic_plan_get_info": [P, ct.POINTER(PlanInfo)],
        "epic_set_gains": [P, c_dp],
        "epic_image": [P, P, ct.c_longlong, P, ct.c_int],
        "epic_image_host": [P, P, ct.c_longlong, P, ct.c_int],
        "epic_image_host_static": [P, P, ct.c_longlong, P, ct.c_int],
        "epical_configure": [P, ct.c_double, ct.c_double, ct.c_int, c_dp, ct.c_double, c_dp],
        "epical_update": [P, P, P],
        "epical_average_channels": [P, ct.c_int, ct.c_int],
        "epic_plan_sync": [P, c_ip],
        "epical_get_gains": [P, c_dp],
        "epical_get_state": [P, P, ct.POINTER(ct.c_size_t)],
        "epical_set_state": [P, P, ct.c_size_t],
        "epic_plan_get_grid_table": [P, c_ip, c_dp],
        "epic_unpack_ci4": [P, P, P, ct.c_longlong],
        "epic_set_gains_device": [P, P],
        "epic_image_backward": [P, P, ct.c_longlong, P, P],
        "epic_autotune": [P, P, ct.c_longlong, P, ct.POINTER(TuneResult)],
        "epic_graph_capture": [P, P, ct.c_longlong, P, P],
        "epic_graph_launch": [P],
        "epic_measure_fma_peak": [ct.c_int, ct.c_int, ct.c_longlong, P, P, c_dp],
        "epical_configure_pixels": [P, ct.c_int, c_dp],
        "epical_get_direction_gains": [P, c_dp],
        "epic_visibilities": [P, P, ct.c_longlong, P, ct.c_int],
        "epic_visibility_solve": [P, P, P, ct.c_int, ct.c_double, ct.c_double, c_ip],
        "epical_fit_bandpass": [P, ct.c_int, ct.c_int, ct.c_int, ct.c_int],
        "epic_set_phase_centre": [P, ct.c_double, ct.c_double],
        "epic_plan_set_wait_limit": [P, ct.c_int],
        "epic_plan_set_adjoint_precision": [P, ct.c_int],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ct.c_int
    lib.epic_last_error.argtypes = []
    lib.epic_last_error.restype = ct.c_char_p
    _lib = lib
    return lib


def check(status: int) -> int:
    """Raise EpicError for a non-OK status."""
    if status != EPIC_OK:
        msg = _lib.epic_last_error().decode() if _lib is not None else ""
        raise EpicError(status, msg)
    return status
