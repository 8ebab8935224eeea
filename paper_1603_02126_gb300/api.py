"""Python binding of the EPIC/EPICal C ABI.

Thin wrappers with the C names (epic_plan_create, epic_image, epical_update,
...) plus a `Plan` object that owns the handle.  torch tensors provide device
memory and the CUDA stream; all computation is in libepic.so.  If the
library is missing the calls raise: there is no CPU path.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import _binding as B
from ._binding import EpicError  # noqa: F401

_KERNELS = {"gaussian": B.EPIC_KERNEL_GAUSSIAN, "tophat": B.EPIC_KERNEL_TOPHAT}
_INPUTS = {"ci4": B.EPIC_IN_CI4, "c64": B.EPIC_IN_COMPLEX64}
_PATHS = {"auto": B.EPIC_PATH_AUTO, "fused": B.EPIC_PATH_FUSED, "unfused": B.EPIC_PATH_UNFUSED,
          "cluster": B.EPIC_PATH_CLUSTER, "piped": B.EPIC_PATH_PIPED}


def _torch():
    import torch  # deferred so that non-GPU users of the module need not import it
    return torch


def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return ct.c_void_p(t.data_ptr())


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _c128_as_f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.complex128).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} complex values, got {a.size}")
    return a.view(np.float64)


class Plan:
    """One EPIC/EPICal plan: array, grid, kernel and channels (Sec. 2.1)."""

    def __init__(self, ant_xy_m, freq_hz, grid_n, cell=0.5, kernel="gaussian", support=3,
                 param=0.5, input="ci4", voltage_scale=None, flags=None, stream=None,
                 path="auto", workspace_bytes=0, precision="fp32", batch_persistent=False):
        lib = B.load()
        self._lib = lib
        self.ant = _f64(ant_xy_m).reshape(-1, 2)
        self.freqs = _f64(freq_hz).reshape(-1)
        self.n_ant, self.n_chan, self.grid_n = self.ant.shape[0], self.freqs.size, int(grid_n)
        self.input = input
        self._vs = None if voltage_scale is None else np.ascontiguousarray(voltage_scale, np.float32)
        self._fl = None if flags is None else np.ascontiguousarray(np.asarray(flags) != 0, np.uint8)
        if stream is None:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        d = B.PlanDesc()
        d.n_ant = self.n_ant
        d.ant_xy_m = self.ant.ctypes.data_as(B.c_dp)
        d.n_chan = self.n_chan
        d.freq_hz = self.freqs.ctypes.data_as(B.c_dp)
        d.grid_n = self.grid_n
        d.cell_wavelengths = float(cell)
        d.kernel = _KERNELS[kernel]
        d.kernel_support = int(support)
        kp = np.asarray(param, np.float64)
        if kp.ndim == 0:
            d.kernel_param = float(kp)
            self._kp = None
        else:                                   # one kernel parameter per antenna
            self._kp = np.ascontiguousarray(kp.reshape(-1))
            d.kernel_param = float(self._kp[0]) if self._kp.size else 0.0
            d.kernel_param_ant = self._kp.ctypes.data_as(B.c_dp)
        d.input = _INPUTS[input]
        d.voltage_scale = None if self._vs is None else self._vs.ctypes.data_as(B.c_fp)
        d.flags = None if self._fl is None else self._fl.ctypes.data_as(B.c_u8p)
        d.precision = {"fp32": B.EPIC_PREC_FP32, "fp16": B.EPIC_PREC_FP16,
                       "bf16": B.EPIC_PREC_BF16}[precision]
        d.cuda_stream = ct.c_void_p(int(stream))
        d.path = _PATHS[path]
        d.workspace_bytes = int(workspace_bytes)
        d.batch_persistent = int(bool(batch_persistent))
        h = ct.c_void_p()
        B.check(lib.epic_plan_create(ct.byref(h), ct.byref(d)))
        self.handle = h

    # ---- lifetime ----
    def close(self):
        if getattr(self, "handle", None):
            self._lib.epic_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- wrappers ----
    def set_stream(self, stream):
        B.check(self._lib.epic_plan_set_stream(self.handle, ct.c_void_p(int(stream))))

    def info(self) -> dict:
        i = B.PlanInfo()
        B.check(self._lib.epic_plan_get_info(self.handle, ct.byref(i)))
        return {k: getattr(i, k) for k, _ in B.PlanInfo._fields_}

    def set_gains(self, gains):
        g = _c128_as_f64(gains, self.n_chan * self.n_ant)
        B.check(self._lib.epic_set_gains(self.handle, g.ctypes.data_as(B.c_dp)))

    def image(self, volt, image=None, accumulate=False):
        """Image a device voltage batch [T][C][Na] (uint8 ci4 or complex64)
        into image [C][N][N] float64 (allocated if None)."""
        torch = _torch()
        want = torch.uint8 if self.input == "ci4" else torch.complex64
        if volt.dim() != 3 or volt.shape[1] != self.n_chan or volt.shape[2] != self.n_ant:
            raise ValueError("volt must be [T][C][Na]")
        if image is None:
            image = torch.empty((self.n_chan, self.grid_n, self.grid_n), dtype=torch.float64,
                                device=volt.device)
        B.check(self._lib.epic_image(self.handle, _dptr(volt, want, "volt"), int(volt.shape[0]),
                                     _dptr(image, torch.float64, "image"), int(bool(accumulate))))
        return image

    def _host_buffers(self, volt, image, name):
        """Validated host pointers of a [T][C][Na] voltage array and a
        [C][N][N] float64 image (allocated if None): the C side copies
        exactly those sizes, so a mismatched array is refused here."""
        torch = _torch()
        want = np.uint8 if self.input == "ci4" else np.complex64
        if isinstance(volt, torch.Tensor):
            if volt.is_cuda:
                raise TypeError(f"{name} takes host memory")
            tdt = torch.uint8 if self.input == "ci4" else torch.complex64
            if volt.dtype != tdt:
                raise TypeError(f"volt must be {tdt}, got {volt.dtype}")
            vt = volt.contiguous()
            vptr, vshape = ct.c_void_p(vt.data_ptr()), tuple(vt.shape)
        else:
            if np.asarray(volt).dtype != want:
                raise TypeError(f"volt must be {np.dtype(want)}, got {np.asarray(volt).dtype}")
            vt = np.ascontiguousarray(volt)
            vptr, vshape = ct.c_void_p(vt.ctypes.data), vt.shape
        if len(vshape) != 3 or vshape[1:] != (self.n_chan, self.n_ant) or vshape[0] < 1:
            raise ValueError(f"volt must be [T][{self.n_chan}][{self.n_ant}], got {list(vshape)}")
        shape = (self.n_chan, self.grid_n, self.grid_n)
        if image is None:
            image = np.zeros(shape, np.float64)
        if isinstance(image, torch.Tensor):
            if image.is_cuda or image.dtype != torch.float64 or tuple(image.shape) != shape \
                    or not image.is_contiguous():
                raise ValueError(f"image must be a contiguous host float64 {list(shape)} array")
            iptr = ct.c_void_p(image.data_ptr())
        else:
            if not isinstance(image, np.ndarray) or image.dtype != np.float64 or image.shape != shape \
                    or not image.flags.c_contiguous:
                raise ValueError(f"image must be a C-contiguous float64 {list(shape)} array")
            iptr = ct.c_void_p(image.ctypes.data)
        return vt, vptr, int(vshape[0]), image, iptr

    def image_host(self, volt, image=None, accumulate=False):
        """Host-buffer form (copies inside the call).  volt: numpy array or
        CPU tensor [T][C][Na] (uint8 ci4 or complex64); returns the float64
        [C][N][N] image (a new numpy array if image is None)."""
        vt, vptr, T, image, iptr = self._host_buffers(volt, image, "image_host")
        B.check(self._lib.epic_image_host(self.handle, vptr, T, iptr, int(bool(accumulate))))
        return image

    def image_host_static(self, volt, image=None, accumulate=False):
        """image_host without any device allocation: stages through the
        library's fixed 32 MiB device array (for callers that may not call
        cudaMalloc).  Same arguments and result as image_host; the plan must
        be on the fused FP32 path."""
        vt, vptr, T, image, iptr = self._host_buffers(volt, image, "image_host_static")
        B.check(self._lib.epic_image_host_static(self.handle, vptr, T, iptr, int(bool(accumulate))))
        return image

    def set_gains_device(self, gains):
        """Set g from a device complex128 [C][Na] tensor (asynchronous)."""
        torch = _torch()
        B.check(self._lib.epic_set_gains_device(self.handle, _dptr(gains, torch.complex128, "gains")))

    def image_backward(self, volt, dl_di, grad=None):
        """2 dL/dconj(g) for dl_di = dL/dI (float64 [C][N][N], device)."""
        torch = _torch()
        if grad is None:
            grad = torch.empty((self.n_chan, self.n_ant), dtype=torch.complex128, device=volt.device)
        want = torch.uint8 if self.input == "ci4" else torch.complex64
        B.check(self._lib.epic_image_backward(self.handle, _dptr(volt, want, "volt"),
                                              int(volt.shape[0]),
                                              _dptr(dl_di, torch.float64, "dl_di"),
                                              _dptr(grad, torch.complex128, "grad")))
        return grad

    def set_adjoint_precision(self, precision):
        """Arithmetic of image_backward's transforms: "fp32" or "bf16"
        (two frames at a time as BF16 pairs)."""
        code = {"fp32": B.EPIC_PREC_FP32, "bf16": B.EPIC_PREC_BF16}.get(precision)
        if code is None:
            raise ValueError(f"adjoint precision must be 'fp32' or 'bf16', not {precision!r}")
        B.check(self._lib.epic_plan_set_adjoint_precision(self.handle, code))

    def autotune(self, volt, image=None) -> dict:
        """Time launch-shape candidates on this batch and keep the fastest."""
        torch = _torch()
        if image is None:
            image = torch.empty((self.n_chan, self.grid_n, self.grid_n), dtype=torch.float64,
                                device=volt.device)
        r = B.TuneResult()
        B.check(self._lib.epic_autotune(self.handle, _dptr(volt, None, "volt"), int(volt.shape[0]),
                                        _dptr(image, torch.float64, "image"), ct.byref(r)))
        return {k: getattr(r, k) for k, _ in B.TuneResult._fields_}

    def graph_capture(self, volt, image, gains_out=None):
        """Capture one interval (image + update) into a CUDA graph."""
        torch = _torch()
        B.check(self._lib.epic_graph_capture(self.handle, _dptr(volt, None, "volt"), int(volt.shape[0]),
                                             _dptr(image, torch.float64, "image"),
                                             _dptr(gains_out, torch.complex128, "gains_out")))

    def graph_launch(self):
        B.check(self._lib.epic_graph_launch(self.handle))

    def configure(self, cal_lm, model_lmS, gamma, g0=None):
        src = _f64(model_lmS).reshape(-1, 3)
        g = None if g0 is None else _c128_as_f64(g0, self.n_chan * self.n_ant)
        B.check(self._lib.epical_configure(
            self.handle, float(cal_lm[0]), float(cal_lm[1]), src.shape[0],
            src.ctypes.data_as(B.c_dp), float(gamma),
            None if g is None else g.ctypes.data_as(B.c_dp)))

    def configure_pixels(self, pix_lm):
        """Multiple-pixel / direction-dependent EPICal (Sec. 6): calibration
        pixels at the directions pix_lm [P][2] (l, m); after epical_configure."""
        pl = _f64(pix_lm).reshape(-1, 2)
        self.n_pix = pl.shape[0]
        B.check(self._lib.epical_configure_pixels(self.handle, self.n_pix, pl.ctypes.data_as(B.c_dp)))

    def direction_gains(self) -> np.ndarray:
        """Per-direction solutions [C][Na][P] complex128 (host)."""
        out = np.empty((self.n_chan, self.n_ant, self.n_pix), np.complex128)
        B.check(self._lib.epical_get_direction_gains(self.handle, out.view(np.float64).ctypes.data_as(B.c_dp)))
        return out

    def visibilities(self, volt, vis=None, accumulate=False):
        """X-engine (Sec. 4 comparison): V [C][Na][Na] complex128 on the
        device from a device voltage batch [T][C][Na]."""
        torch = _torch()
        want = torch.uint8 if self.input == "ci4" else torch.complex64
        if vis is None:
            vis = torch.empty((self.n_chan, self.n_ant, self.n_ant), dtype=torch.complex128,
                              device=volt.device)
        B.check(self._lib.epic_visibilities(self.handle, _dptr(volt, want, "volt"), int(volt.shape[0]),
                                            _dptr(vis, torch.complex128, "vis"), int(bool(accumulate))))
        return vis

    def visibility_solve(self, vis, gains, max_iter=5000, tol=1e-12, min_baseline=0.0):
        """Eq. 21 by StEFCal on the device, in place on gains [C][Na]
        complex128 (start -> solution).  Returns the iterations per channel."""
        torch = _torch()
        it = np.zeros(self.n_chan, np.int32)
        B.check(self._lib.epic_visibility_solve(self.handle, _dptr(vis, torch.complex128, "vis"),
                                                _dptr(gains, torch.complex128, "gains"), int(max_iter),
                                                float(tol), float(min_baseline), it.ctypes.data_as(B.c_ip)))
        return it

    def fit_bandpass(self, c_lo, c_hi, deg_amp, deg_phase):
        """Polynomial gain model in amplitude and phase across channels
        c_lo..c_hi-1 (Sec. 6); after update."""
        B.check(self._lib.epical_fit_bandpass(self.handle, int(c_lo), int(c_hi), int(deg_amp), int(deg_phase)))

    def set_phase_centre(self, l0, m0):
        """Phase the array to (l0, m0) (Sec. 2.1 footnote); resets EPICal."""
        B.check(self._lib.epic_set_phase_centre(self.handle, float(l0), float(m0)))

    def set_wait_limit(self, polls):
        """Polls per bounded wait of the warp-specialised kernel and of the
        persistent unfused kernel's grid barrier (0 = default)."""
        B.check(self._lib.epic_plan_set_wait_limit(self.handle, int(polls)))

    def update(self, gains_out=None, status=None):
        torch = _torch()
        B.check(self._lib.epical_update(self.handle, _dptr(gains_out, torch.complex128, "gains_out"),
                                        _dptr(status, torch.int32, "status")))

    def average_channels(self, c_lo, c_hi):
        """Take the gains as constant across channels c_lo .. c_hi - 1: each
        antenna's gains there become their complex mean (asynchronous; call
        after `update`)."""
        B.check(self._lib.epical_average_channels(self.handle, int(c_lo), int(c_hi)))

    def sync(self) -> int:
        """Wait for the stream; return the number of gains held since the
        last sync (EPIC_ERR_NUMERIC is reported through the count)."""
        n = ct.c_int(0)
        st = self._lib.epic_plan_sync(self.handle, ct.byref(n))
        if st not in (B.EPIC_OK, 5):
            B.check(st)
        return n.value

    def gains(self) -> np.ndarray:
        out = np.zeros((self.n_chan, self.n_ant), np.complex128)
        B.check(self._lib.epical_get_gains(self.handle, out.view(np.float64).ctypes.data_as(B.c_dp)))
        return out

    def get_state(self) -> bytes:
        n = ct.c_size_t(0)
        B.check(self._lib.epical_get_state(self.handle, None, ct.byref(n)))
        buf = ct.create_string_buffer(n.value)
        B.check(self._lib.epical_get_state(self.handle, buf, ct.byref(n)))
        return buf.raw

    def set_state(self, state: bytes):
        buf = ct.create_string_buffer(state, len(state))
        B.check(self._lib.epical_set_state(self.handle, buf, len(state)))

    def grid_table(self):
        K = None
        base = np.zeros((self.n_chan, self.n_ant, 2), np.int32)
        B.check(self._lib.epic_plan_get_grid_table(self.handle, base.ctypes.data_as(B.c_ip), None))
        info = self.info()
        K = info["kernel_support"]
        w = np.zeros((self.n_chan, self.n_ant, K, K), np.float64)
        B.check(self._lib.epic_plan_get_grid_table(self.handle, None, w.ctypes.data_as(B.c_dp)))
        return base, w

    def unpack_ci4(self, d_in, d_out=None):
        torch = _torch()
        if d_out is None:
            d_out = torch.empty((d_in.numel(), 2), dtype=torch.float32, device=d_in.device)
        B.check(self._lib.epic_unpack_ci4(self.handle, _dptr(d_in, torch.uint8, "d_in"),
                                          _dptr(d_out, torch.float32, "d_out"), int(d_in.numel())))
        return d_out


# C-ABI-named module functions (thin aliases of the Plan methods)
def measure_fma_peak(fp64=False, stream=None, reps=5):
    """Measured FMA rate of the device in TFLOP/s (FP32, or FP64): the
    median over reps of one epic_measure_fma_peak launch timed with CUDA
    events on `stream` (default: a new stream on the current device).  The
    roofline denominator of the FP32-arithmetic-bound imaging kernels."""
    torch = _torch()
    lib = B.load()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8                       # 8 x 256 threads per SM: 64 warps
    iters = 64 if fp64 else 4096
    st = stream if stream is not None else torch.cuda.Stream()
    sink = torch.zeros(blocks, dtype=torch.float64, device="cuda")
    flops = ct.c_double()
    times = []
    for i in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        B.check(lib.epic_measure_fma_peak(int(bool(fp64)), blocks, iters, ct.c_void_p(sink.data_ptr()),
                                          ct.c_void_p(st.cuda_stream), ct.byref(flops)))
        e1.record(st)
        e1.synchronize()
        if i:
            times.append(e0.elapsed_time(e1))
    return flops.value / (float(np.median(times)) / 1e3) / 1e12


def epic_plan_create(*args, **kw) -> Plan:
    return Plan(*args, **kw)


def epic_plan_destroy(plan: Plan):
    plan.close()


def epic_image(plan: Plan, volt, image=None, accumulate=False):
    return plan.image(volt, image, accumulate)


def epic_image_host(plan: Plan, volt, image=None, accumulate=False):
    return plan.image_host(volt, image, accumulate)


def epical_configure(plan: Plan, cal_lm, model_lmS, gamma, g0=None):
    return plan.configure(cal_lm, model_lmS, gamma, g0)


def epical_update(plan: Plan, gains_out=None, status=None):
    return plan.update(gains_out, status)


def epic_plan_sync(plan: Plan) -> int:
    return plan.sync()
