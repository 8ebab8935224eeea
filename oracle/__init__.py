"""FP64 CPU oracle for EPIC imaging and EPICal calibration.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline arm may import this package.  The CUDA library never
calls it and shares no code with it.

Everything here is plain NumPy in float64/complex128, written from the paper
(Beardsley et al., "An Efficient Feedback Calibration Algorithm for Direct
Imaging Radio Telescopes"): direct loops for gridding, the naive separable
DFT for the image, explicit time averages.  Each function cites the section
and equation it follows.  See `epic_oracle` for the functions.
"""
from .epic_oracle import *  # noqa: F401,F403
