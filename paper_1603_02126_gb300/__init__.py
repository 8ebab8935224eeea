"""GB300-native EPIC direct imaging and EPICal feedback calibration.

The hot path (4-bit unpack, gain correction, gridding, 2D FFT,
square-accumulate, antenna-pixel correlation, damped gain update) runs in
hand-written sm_103a CUDA kernels inside libepic.so behind the C ABI of
include/epic.h.  This package holds that library's sources (csrc/), its
build script and a ctypes binding.
"""
from .api import (EpicError, Plan, epic_image, epic_image_host, epic_plan_create,  # noqa: F401
                  epic_plan_destroy, epic_plan_sync, epical_configure, epical_update)
