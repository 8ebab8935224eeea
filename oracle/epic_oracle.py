"""FP64 oracle for the EPIC imaging chain and the EPICal gain update.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline of the benchmark, never by the CUDA library.

Notation follows the paper.  Na antennas a, b; grid cells j = (jx, jy);
image pixels k = (kx, ky); N x N grid of cell size du (wavelengths);
frames are (t, channel) pairs.  u_a = r_a f / c is the antenna position in
wavelengths.  Readings of points the paper leaves open are listed with each
function (gain direction, grid geometry, kernel, FFT sign and centring,
calibrator pixel, Na vs Na-1 in the single-source limit, flags).

Parity pins for every function live in tests/test_oracle_pins.py.  Pinned:
unpack (exhaustive), grid table (properties and special positions), the
image (visibility route, numpy.fft route, direct O(N^4) sum, phase-ramp
closed form, source position), the EPICal correlation and update (visibility
route, zenith single-source limit, noise-free fixed point, damping closed
form, effective integration time), the visibility solve (noise-free
truth) and the chi^2 model image and gradient (noise-free identity, central
finite differences), and the sampled-output checkers image_pixels and
correlate_sampled (visibility route at every pixel, the full transform).
Nothing in this module is parity-unpinned.
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299792458.0  # speed of light, m/s

__all__ = [
    "C_LIGHT", "GridTooSmall", "unpack_ci4", "antenna_uv", "grid_table",
    "apply_gains", "grid_frames", "efield_image", "efield_image_direct",
    "calibrator_pixel", "pixel_row", "model_visibilities",
    "cal_denominator", "correlate", "epical_update", "image_interval",
    "epical_interval", "visibilities", "visibility_solve", "gain_error",
    "align_phase", "Plan", "image_pixels", "correlate_sampled", "pixel_matrix",
    "model_image", "chi2_loss", "chi2_gradient", "average_channels",
    "MultiPixelPlan", "pixel_taps", "correlate_multi", "multipixel_update",
    "direction_update", "multipixel_interval", "baseline_mask", "bandpass_x", "fit_bandpass",
    "phase_factors",
]


class GridTooSmall(ValueError):
    """A gridding stencil falls outside [0, N)."""


# --------------------------------------------------------------------------
# input format
# --------------------------------------------------------------------------
def unpack_ci4(b: np.ndarray) -> np.ndarray:
    """4-bit complex byte -> complex128 integers (high nibble real, low
    nibble imaginary, two's complement in [-8, 7]).

    Input to the calibration step of Eq. 8: the F-engine output of Sec. 2.1
    in the 4-bit format of the LWA-like workload.
    """
    b = np.asarray(b).astype(np.int64)
    hi = b >> 4
    lo = b & 15
    re = np.where(hi > 7, hi - 16, hi)
    im = np.where(lo > 7, lo - 16, lo)
    return re.astype(np.float64) + 1j * im.astype(np.float64)


# --------------------------------------------------------------------------
# geometry and gridding kernel (Sec. 2.1, Eq. 9)
# --------------------------------------------------------------------------
def antenna_uv(ant_xy_m: np.ndarray, freq_hz: float) -> np.ndarray:
    """u_a = r_a f / c in wavelengths (exponent of Eq. 3), computed as
    (r * f) / c in float64."""
    return (np.asarray(ant_xy_m, np.float64) * float(freq_hz)) / C_LIGHT


def grid_table(ant_xy_m, freq_hz, grid_n: int, cell: float,
               kernel: str = "gaussian", support: int = 3, param: float = 0.5,
               flags=None):
    """Gridding stencil of Eq. 9 for every (channel, antenna).

    Reading: the grid is in wavelengths with cell `cell`; the continuous grid
    coordinate is p = u / cell + N/2 (grid centre at index N/2, x = East ->
    column, y = North -> row); the stencil centre is the nearest cell,
    floor(p + 0.5); taps are base + d with d in [-(K-1)/2, (K-1)/2] per axis.
    Gaussian: W = exp(-|j - p|^2 / (2 sigma^2)), sigma = param cells.
    Tophat: W = 1 for taps inside a square of side `param` metres centred on
    the antenna, else 0.  `param` may also be an array [Na], one value per
    antenna (heterogeneous illumination patterns).  Weights are normalised to sum to 1 so that the far
    field pattern is 1 at its centre (Sec. 2.1, normalisation of W_a).
    Flagged antennas get zero weights (excluded from the image).

    Returns base [C][Na][2] int64 (x, y) of the stencil centre and
    weights [C][Na][K][K] float64 indexed [dy][dx].
    Raises GridTooSmall if any tap of an unflagged antenna is outside [0, N).
    """
    ant = np.asarray(ant_xy_m, np.float64)
    freqs = np.atleast_1d(np.asarray(freq_hz, np.float64))
    C, Na = len(freqs), ant.shape[0]
    K = int(support)
    if K < 1 or K % 2 == 0:
        raise ValueError("kernel support must be odd")
    h = (K - 1) // 2
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    pa = np.broadcast_to(np.asarray(param, np.float64), (Na,))
    base = np.zeros((C, Na, 2), np.int64)
    W = np.zeros((C, Na, K, K), np.float64)
    for c in range(C):
        uv = antenna_uv(ant, freqs[c])
        for a in range(Na):
            p = uv[a] / cell + grid_n / 2
            b = np.floor(p + 0.5).astype(np.int64)
            base[c, a] = b
            if flags[a]:
                continue
            if b.min() - h < 0 or b.max() + h >= grid_n:
                raise GridTooSmall(f"antenna {a} channel {c} stencil outside grid")
            for dy in range(K):
                for dx in range(K):
                    jx = b[0] + dx - h
                    jy = b[1] + dy - h
                    if kernel == "gaussian":
                        d2 = (jx - p[0]) ** 2 + (jy - p[1]) ** 2
                        W[c, a, dy, dx] = np.exp(-d2 / (2.0 * pa[a] * pa[a]))
                    elif kernel == "tophat":
                        half = (pa[a] * freqs[c] / C_LIGHT) / cell / 2.0
                        inside = abs(jx - p[0]) <= half and abs(jy - p[1]) <= half
                        W[c, a, dy, dx] = 1.0 if inside else 0.0
                    else:
                        raise ValueError(kernel)
            s = W[c, a].sum()
            if not s > 0:
                raise ValueError(f"antenna {a} channel {c}: kernel has no support")
            W[c, a] /= s
    return base, W


# --------------------------------------------------------------------------
# imaging chain for one channel (Eqs. 8-10, Sec. 2.1 square-and-average)
# --------------------------------------------------------------------------
def apply_gains(E: np.ndarray, g: np.ndarray) -> np.ndarray:
    """E'_a = E_a / g'_a (Eq. 8).  E: [..., Na], g: [Na]."""
    return E / g


def grid_frames(Ecal: np.ndarray, base: np.ndarray, W: np.ndarray,
                grid_n: int, flags=None) -> np.ndarray:
    """E'_j = sum_a W_a(r_j - r_a) E'_a (Eq. 9) by direct loops over antennas
    and taps, vectorised over frames.  Ecal: [F][Na]; base [Na][2];
    W [Na][K][K].  Returns G [F][N(y)][N(x)] complex128."""
    F, Na = Ecal.shape
    K = W.shape[-1]
    h = (K - 1) // 2
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    G = np.zeros((F, grid_n, grid_n), np.complex128)
    for a in range(Na):
        if flags[a]:
            continue
        for dy in range(K):
            for dx in range(K):
                jx = base[a, 0] + dx - h
                jy = base[a, 1] + dy - h
                G[:, jy, jx] += W[a, dy, dx] * Ecal[:, a]
    return G


def _phase_matrix(n: int) -> np.ndarray:
    """F[k, j] = exp(+2 pi i (j - N/2)(k - N/2) / N), exponent reduced mod N
    as an exact integer (Eq. 10 kernel, centred grid and image)."""
    j = np.arange(n) - n // 2
    m = np.mod(np.outer(j, j), n)          # symmetric in (k, j)
    return np.exp(2j * np.pi * m / n)


def efield_image(G: np.ndarray, n_ant: int) -> np.ndarray:
    """E-field image of Eq. 10 as a naive separable DFT:
    E[ky, kx] = (1/Na) sum_{jy,jx} G[jy,jx] exp(+2 pi i ((jx-N/2)(kx-N/2)
                + (jy-N/2)(ky-N/2)) / N).
    Reading: '+' sign and 1/Na as printed in Eq. 10; pixel (N/2, N/2) is the
    phase centre, l = (kx - N/2) / (N du).  G: [..., N, N]."""
    n = G.shape[-1]
    F = _phase_matrix(n)
    return (F @ G @ F.T) / n_ant


def efield_image_direct(G: np.ndarray, n_ant: int) -> np.ndarray:
    """Eq. 10 as the direct double sum over cells for every pixel (O(N^4));
    for tiny grids only.  G: [N, N]."""
    n = G.shape[-1]
    out = np.zeros((n, n), np.complex128)
    c = n // 2
    for ky in range(n):
        for kx in range(n):
            acc = 0j
            for jy in range(n):
                for jx in range(n):
                    m = ((jx - c) * (kx - c) + (jy - c) * (ky - c)) % n
                    acc += G[jy, jx] * np.exp(2j * np.pi * m / n)
            out[ky, kx] = acc / n_ant
    return out


# --------------------------------------------------------------------------
# EPICal (Sec. 2.2, Eqs. 12-17)
# --------------------------------------------------------------------------
def calibrator_pixel(l: float, m: float, grid_n: int, cell: float):
    """Pixel centre nearest the calibrator direction (Sec. 2.2): pixel k has
    l = (k - N/2)/(N du), so k = floor(l N du + N/2 + 0.5) per axis."""
    kx = int(np.floor(l * grid_n * cell + grid_n / 2 + 0.5))
    ky = int(np.floor(m * grid_n * cell + grid_n / 2 + 0.5))
    if not (0 <= kx < grid_n and 0 <= ky < grid_n):
        raise ValueError("calibrator outside the image")
    return kx, ky


def pixel_row(base: np.ndarray, W: np.ndarray, grid_n: int, k0, n_ant: int) -> np.ndarray:
    """A_{0,a}: response of image pixel k0 to antenna a, the exact discrete
    form of Eq. 11's (1/Na) W_a(s0) exp(2 pi i f s0 . r_a / c):
    A_{0,a} = (1/Na) sum_taps W_a(j) exp(+2 pi i ((jx-N/2)(k0x-N/2)
              + (jy-N/2)(k0y-N/2)) / N).
    Reading: the exact form is used instead of the approximation so that
    the noise-free fixed point is exact.  base [Na][2], W [Na][K][K]."""
    Na, K = W.shape[0], W.shape[-1]
    h = (K - 1) // 2
    c = grid_n // 2
    A = np.zeros(Na, np.complex128)
    for a in range(Na):
        for dy in range(K):
            for dx in range(K):
                jx = base[a, 0] + dx - h
                jy = base[a, 1] + dy - h
                mm = ((jx - c) * (k0[0] - c) + (jy - c) * (k0[1] - c)) % grid_n
                A[a] += W[a, dy, dx] * np.exp(2j * np.pi * mm / grid_n)
    return A / n_ant


def model_visibilities(ant_xy_m, freq_hz: float, sky_lmS: np.ndarray) -> np.ndarray:
    """V^M_ab = sum_s S_s exp(-2 pi i (u_a - u_b) . s_s): point sources with
    apparent fluxes and isotropic antenna response (Sec. 3 'perfect model
    visibilities'; sign from Eq. 3)."""
    uv = antenna_uv(ant_xy_m, freq_hz)
    Na = uv.shape[0]
    V = np.zeros((Na, Na), np.complex128)
    for l, m, S in np.asarray(sky_lmS, np.float64):
        e = np.exp(-2j * np.pi * (uv[:, 0] * l + uv[:, 1] * m))
        V += S * np.outer(e, np.conj(e))
    return V


def cal_denominator(A0: np.ndarray, VM: np.ndarray, flags=None) -> np.ndarray:
    """D_a = sum_{b != a} conj(A_{0,b}) V^M_ab.  With conj(A_{0,b}) Na =
    W*_b(s0) exp(-2 pi i f s0 . r_b / c), D_a is the denominator of Eq. 16
    divided by Na, so that g^{(n+1)}_a = C_a / D_a.  Flagged b are left out
    of the sum."""
    Na = A0.shape[0]
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    D = np.zeros(Na, np.complex128)
    for a in range(Na):
        for b in range(Na):
            if b != a and not flags[b]:
                D[a] += np.conj(A0[b]) * VM[a, b]
    return D


def correlate(E: np.ndarray, pix: np.ndarray):
    """Antenna-pixel correlation of Eq. 12 and the autocorrelation of Eq. 15
    over one calibration interval, using the uncalibrated voltages:
    K_a = < E_a(t) conj(E'(s0, t)) >_t,  P_a = < |E_a(t)|^2 >_t.
    E: [T][Na], pix: [T]."""
    T = E.shape[0]
    Kc = (E * np.conj(pix)[:, None]).sum(axis=0) / T
    P = (np.abs(E) ** 2).sum(axis=0) / T
    return Kc, P


def epical_update(Kc, P, A0, D, g, gamma: float, flags=None, d_min: float = 0.0):
    """Damped EPICal gain update (Eqs. 15, 16, 17):
    C_a = K_a - conj(A_{0,a}) P_a / conj(g_a)          (Eq. 15)
    g_a <- (1 - gamma) C_a / D_a + gamma g_a           (Eqs. 16, 17)
    Flagged antennas, |D_a| <= d_min and non-finite results hold g_a.
    Returns (g_new, held mask)."""
    if not (0.0 <= gamma < 1.0):
        raise ValueError("gamma must be in [0, 1)")
    Na = g.shape[0]
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    Cc = Kc - np.conj(A0) * P / np.conj(g)
    with np.errstate(divide="ignore", invalid="ignore"):
        gn = (1.0 - gamma) * Cc / D + gamma * g
    held = flags | ~(np.abs(D) > d_min) | ~np.isfinite(gn)
    return np.where(held, g, gn), held


def average_channels(g, c_lo: int, c_hi: int, flags=None):
    """Gains assumed constant across a band of channels (Sec. 5, LWA data):
    after an interval's update, every channel c_lo <= c < c_hi takes the
    plain mean of the complex solutions of those channels, antenna by
    antenna.  Channels outside the band, flagged antennas and antennas whose
    mean is zero or not finite are returned unchanged.  g: [C][Na] complex."""
    g = np.array(g, np.complex128, copy=True)
    C, Na = g.shape
    if not (0 <= c_lo < c_hi <= C):
        raise ValueError("need 0 <= c_lo < c_hi <= C")
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    mean = g[c_lo:c_hi].mean(axis=0)
    use = ~flags & np.isfinite(mean) & (np.abs(mean) > 0)
    g[c_lo:c_hi, use] = mean[use]
    return g


def bandpass_x(freqs, c_lo: int, c_hi: int) -> np.ndarray:
    """Fit abscissa of channels c_lo..c_hi-1: frequency mapped linearly onto
    [-1, 1] over the band (0 for a one-channel band)."""
    f = np.asarray(freqs, np.float64)[c_lo:c_hi]
    lo, hi = f.min(), f.max()
    if hi == lo:
        return np.zeros_like(f)
    return (f - 0.5 * (lo + hi)) / (0.5 * (hi - lo))


def fit_bandpass(g, freqs, c_lo: int, c_hi: int, deg_amp: int, deg_phase: int, flags=None):
    """Gain model fitted across frequency (Sec. 6, "Fitting gain models": a
    low-order polynomial in amplitude and in phase over a band of channels).
    Per unflagged antenna: the amplitudes |g| and the phases arg g, unwrapped
    along the band from its first channel (each step taken within pi), are
    fitted by least squares with polynomials of degrees deg_amp and deg_phase
    in the band abscissa x (bandpass_x); the gains of the band are replaced
    by A(x) e^{i Phi(x)}.  Channels outside the band, flagged antennas and
    antennas with a zero or non-finite gain in the band are returned
    unchanged.  g: [C][Na] complex.  Needs c_hi - c_lo > max(deg_amp, deg_phase)."""
    g = np.array(g, np.complex128, copy=True)
    C, Na = g.shape
    if not (0 <= c_lo < c_hi <= C):
        raise ValueError("need 0 <= c_lo < c_hi <= C")
    if min(deg_amp, deg_phase) < 0 or c_hi - c_lo <= max(deg_amp, deg_phase):
        raise ValueError("need 0 <= degree < channels in the band")
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    x = bandpass_x(freqs, c_lo, c_hi)
    for a in range(Na):
        ga = g[c_lo:c_hi, a]
        if flags[a] or not np.all(np.isfinite(ga)) or np.any(ga == 0):
            continue
        amp = np.abs(ga)
        ph = np.unwrap(np.angle(ga))
        pa = np.polynomial.polynomial.polyfit(x, amp, deg_amp)
        pp = np.polynomial.polynomial.polyfit(x, ph, deg_phase)
        g[c_lo:c_hi, a] = (np.polynomial.polynomial.polyval(x, pa)
                           * np.exp(1j * np.polynomial.polynomial.polyval(x, pp)))
    return g


def phase_factors(ant_xy_m, freq_hz: float, phase_lm) -> np.ndarray:
    """Phasing to a phase centre s0 = (l0, m0) away from zenith (Sec. 2.1
    footnote: a phase applied to the electric fields as one phases
    visibilities): p_a = exp(+2 pi i u_a . s0) for the planar array, so that
    p_a E_a of a source at s equals the unphased field of a source at s - s0
    and the image is centred on s0 (pixel l = l0 + (kx - N/2)/(N du))."""
    uv = antenna_uv(ant_xy_m, freq_hz)
    return np.exp(2j * np.pi * (uv[:, 0] * phase_lm[0] + uv[:, 1] * phase_lm[1]))


# --------------------------------------------------------------------------
# one calibration interval for all channels
# --------------------------------------------------------------------------
class Plan:
    """Static per-array quantities of one observation: grid tables, the
    calibrator pixel, A_{0,a} and D_a per channel."""

    def __init__(self, ant_xy_m, freq_hz, grid_n, cell, kernel="gaussian",
                 support=3, param=0.5, flags=None, cal_lm=(0.0, 0.0),
                 model_lmS=None, n_ant_norm=None, phase_lm=None):
        self.ant = np.asarray(ant_xy_m, np.float64)
        self.freqs = np.atleast_1d(np.asarray(freq_hz, np.float64))
        self.N = int(grid_n)
        self.cell = float(cell)
        self.Na = self.ant.shape[0]
        self.norm = self.Na if n_ant_norm is None else n_ant_norm
        self.flags = np.zeros(self.Na, bool) if flags is None else np.asarray(flags, bool)
        self.base, self.W = grid_table(self.ant, self.freqs, self.N, self.cell,
                                       kernel, support, param, self.flags)
        # phase centre (Sec. 2.1 footnote): E_a phased by p_a, image
        # coordinates relative to it
        self.phase_lm = (0.0, 0.0) if phase_lm is None else (float(phase_lm[0]), float(phase_lm[1]))
        self.phase = np.stack([phase_factors(self.ant, f, self.phase_lm) for f in self.freqs])
        self.k0 = calibrator_pixel(cal_lm[0] - self.phase_lm[0], cal_lm[1] - self.phase_lm[1],
                                   self.N, self.cell)
        self.A0 = np.stack([pixel_row(self.base[c], self.W[c], self.N, self.k0, self.norm)
                            for c in range(len(self.freqs))]) * self.phase
        if model_lmS is not None:
            self.D = np.stack([cal_denominator(self.A0[c],
                                               model_visibilities(self.ant, f, model_lmS),
                                               self.flags)
                               for c, f in enumerate(self.freqs)])
        else:
            self.D = None


def image_interval(plan: Plan, E: np.ndarray, g: np.ndarray, block: int = 256):
    """Dirty image of one interval for every channel plus the calibrator
    pixel series, following Eq. 8 -> Eq. 9 -> Eq. 10 -> square-and-average.
    E: [T][C][Na] raw voltages, g: [C][Na] current gains.
    Returns (image [C][N][N] float64, pixel [T][C] complex128)."""
    T, C, Na = E.shape
    N = plan.N
    img = np.zeros((C, N, N))
    pix = np.zeros((T, C), np.complex128)
    for c in range(C):
        for t0 in range(0, T, block):
            Ec = apply_gains(E[t0:t0 + block, c, :], g[c]) * plan.phase[c]
            G = grid_frames(Ec, plan.base[c], plan.W[c], N, plan.flags)
            Ei = efield_image(G, plan.norm)
            img[c] += (np.abs(Ei) ** 2).sum(axis=0)
            pix[t0:t0 + block, c] = Ei[:, plan.k0[1], plan.k0[0]]
    return img / T, pix


def epical_interval(plan: Plan, E: np.ndarray, g: np.ndarray, gamma: float,
                    with_image: bool = True, d_min: float = 0.0):
    """One EPICal loop (Sec. 2.2, Fig. 3): image the interval with g^{(n)},
    correlate each raw antenna signal with the calibrator pixel and apply
    the damped update.  Returns (g^{(n+1)}, K, P, image or None, held)."""
    T, C, Na = E.shape
    g = np.asarray(g, np.complex128)       # gains are complex (Eqs. 15-17)
    if with_image:
        img, pix = image_interval(plan, E, g)
    else:
        img = None
        pix = np.zeros((T, C), np.complex128)
        for c in range(C):
            G = grid_frames(apply_gains(E[:, c, :], g[c]) * plan.phase[c], plan.base[c], plan.W[c],
                            plan.N, plan.flags)
            # the single pixel k0 of the Eq. 10 DFT
            n = plan.N
            j = np.arange(n) - n // 2
            fx = np.exp(2j * np.pi * np.mod(j * (plan.k0[0] - n // 2), n) / n)
            fy = np.exp(2j * np.pi * np.mod(j * (plan.k0[1] - n // 2), n) / n)
            pix[:, c] = np.einsum("tyx,y,x->t", G, fy, fx) / plan.norm
    gn = np.empty_like(g)
    Ks = np.empty_like(g)
    Ps = np.empty(g.shape)
    held = np.zeros(g.shape, bool)
    for c in range(C):
        Ks[c], Ps[c] = correlate(E[:, c, :], pix[:, c])
        gn[c], held[c] = epical_update(Ks[c], Ps[c], plan.A0[c], plan.D[c], g[c],
                                       gamma, plan.flags, d_min)
    return gn, Ks, Ps, img, held


def image_pixels(plan: Plan, E: np.ndarray, g: np.ndarray, c: int, pixels,
                 block: int = 512) -> np.ndarray:
    """Selected pixels of the channel-c dirty image, each from the Eq. 10
    sum evaluated at that pixel only (grid, then the single-pixel DFT).
    For checking full-size runs at sampled outputs.  pixels: [(kx, ky)]."""
    T = E.shape[0]
    n = plan.N
    j = np.arange(n) - n // 2
    out = np.zeros(len(pixels))
    for t0 in range(0, T, block):
        G = grid_frames(apply_gains(E[t0:t0 + block, c, :], g[c]) * plan.phase[c], plan.base[c],
                        plan.W[c], n, plan.flags)
        for i, (kx, ky) in enumerate(pixels):
            fx = np.exp(2j * np.pi * np.mod(j * (kx - n // 2), n) / n)
            fy = np.exp(2j * np.pi * np.mod(j * (ky - n // 2), n) / n)
            v = np.einsum("tyx,y,x->t", G, fy, fx) / plan.norm
            out[i] += (np.abs(v) ** 2).sum()
    return out / T


def correlate_sampled(plan: Plan, E: np.ndarray, g: np.ndarray, c: int, ants,
                      block: int = 512):
    """K_a and P_a (Eqs. 12, 15) for selected antennas of channel c, with the
    calibrator pixel taken from the single-pixel Eq. 10 sum."""
    T = E.shape[0]
    n = plan.N
    j = np.arange(n) - n // 2
    fx = np.exp(2j * np.pi * np.mod(j * (plan.k0[0] - n // 2), n) / n)
    fy = np.exp(2j * np.pi * np.mod(j * (plan.k0[1] - n // 2), n) / n)
    pix = np.zeros(T, np.complex128)
    for t0 in range(0, T, block):
        G = grid_frames(apply_gains(E[t0:t0 + block, c, :], g[c]) * plan.phase[c], plan.base[c],
                        plan.W[c], n, plan.flags)
        pix[t0:t0 + block] = np.einsum("tyx,y,x->t", G, fy, fx) / plan.norm
    Kc, P = correlate(E[:, c, list(ants)], pix)
    return Kc, P


# --------------------------------------------------------------------------
# multiple-pixel and direction-dependent EPICal (Sec. 6, "Multiple pixel
# correlations")
# --------------------------------------------------------------------------
class MultiPixelPlan(Plan):
    """EPICal with several calibration pixels (Sec. 6): every raw antenna
    signal is correlated with the E-field at P image pixels, O(Na P) per
    sample.  Per channel and pixel p: A_{p,a}, the exact response of pixel
    k_p to antenna a (as pixel_row), and D_{p,a} = sum_{b != a}
    conj(A_{p,b}) V^M_ab (as cal_denominator).  pix_lm: [P][2] directions
    (l, m); each maps to its nearest pixel centre as the calibrator does."""

    def __init__(self, ant_xy_m, freq_hz, grid_n, cell, pix_lm, model_lmS, **kw):
        super().__init__(ant_xy_m, freq_hz, grid_n, cell, model_lmS=model_lmS, **kw)
        self.pix = [calibrator_pixel(l - self.phase_lm[0], m - self.phase_lm[1], self.N, self.cell)
                    for l, m in np.asarray(pix_lm, np.float64).reshape(-1, 2)]
        C = len(self.freqs)
        self.Ap = np.stack([np.stack([pixel_row(self.base[c], self.W[c], self.N, k, self.norm)
                                      * self.phase[c] for k in self.pix]) for c in range(C)])  # [C][P][Na]
        self.Dp = np.stack([np.stack([cal_denominator(self.Ap[c, i],
                                                      model_visibilities(self.ant, f, model_lmS),
                                                      self.flags)
                                      for i in range(len(self.pix))])
                            for c, f in enumerate(self.freqs)])                   # [C][P][Na]


def pixel_taps(plan: Plan, Ecal: np.ndarray, c: int, pixels) -> np.ndarray:
    """E'(s_k, t) of Eq. 10 at the listed pixels only, for the gain-corrected
    voltages Ecal [T][Na] of channel c: grid (Eq. 9), then the single-pixel
    DFT at each k.  Returns [T][P]."""
    n = plan.N
    j = np.arange(n) - n // 2
    G = grid_frames(Ecal, plan.base[c], plan.W[c], n, plan.flags)
    out = np.zeros((Ecal.shape[0], len(pixels)), np.complex128)
    for i, (kx, ky) in enumerate(pixels):
        fx = np.exp(2j * np.pi * np.mod(j * (kx - n // 2), n) / n)
        fy = np.exp(2j * np.pi * np.mod(j * (ky - n // 2), n) / n)
        out[:, i] = np.einsum("tyx,y,x->t", G, fy, fx) / plan.norm
    return out


def correlate_multi(E: np.ndarray, taps: np.ndarray):
    """Eq. 12 for every calibration pixel: K_{a,p} = < E_a(t) conj(E'(s_p, t)) >_t
    with the uncalibrated voltages, and P_a = < |E_a|^2 >_t (Eq. 15).
    E: [T][Na], taps: [T][P].  Returns K [Na][P], P [Na]."""
    T = E.shape[0]
    Kc = (E.T @ np.conj(taps)) / T
    P = (np.abs(E) ** 2).sum(axis=0) / T
    return Kc, P


def multipixel_update(Kc, P, Ap, Dp, g, gamma: float, flags=None, d_min: float = 0.0):
    """Gain update from P pixel correlations.  Eq. 15 per pixel,
    C_{a,p} = K_{a,p} - conj(A_{p,a}) P_a / conj(g_a); the noise-free fixed
    point C_{a,p} = g_a D_{p,a} holds for every pixel at once (Eqs. 13-16),
    and the reading here combines them by least squares over the pixels,
    g_a <- (1 - gamma) sum_p conj(D_{p,a}) C_{a,p} / sum_p |D_{p,a}|^2
           + gamma g_a                                    (Eq. 17 damping),
    which is Eq. 16 exactly when P = 1.  Flagged antennas, a denominator
    sum_p |D_{p,a}|^2 <= d_min^2 and non-finite results hold g_a.
    Kc [Na][P], P [Na], Ap / Dp [P][Na], g [Na].  Returns (g_new, held, C)."""
    if not (0.0 <= gamma < 1.0):
        raise ValueError("gamma must be in [0, 1)")
    Na = g.shape[0]
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    Cc = Kc - (np.conj(Ap) * (P / np.conj(g))[None, :]).T          # [Na][P]
    num = np.sum(np.conj(Dp).T * Cc, axis=1)
    den = np.sum(np.abs(Dp) ** 2, axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        gn = (1.0 - gamma) * num / den + gamma * g
    held = flags | ~(den > d_min * d_min) | ~np.isfinite(gn)
    return np.where(held, g, gn), held, Cc


def direction_update(Cc, Dp, gdir, gamma: float, flags=None, d_min: float = 0.0):
    """Direction-dependent solutions (Sec. 6): each pixel correlation solves
    for the gains in its own direction independently, g_{a,p} <- (1 - gamma)
    C_{a,p} / D_{p,a} + gamma g_{a,p} (Eqs. 16, 17 per pixel).  Cc [Na][P]
    from multipixel_update, Dp [P][Na], gdir [Na][P].  Flagged antennas,
    |D_{p,a}| <= d_min and non-finite results hold.  Returns (gdir_new, held)."""
    Na = gdir.shape[0]
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    D = Dp.T
    with np.errstate(divide="ignore", invalid="ignore"):
        gn = (1.0 - gamma) * Cc / D + gamma * gdir
    held = flags[:, None] | ~(np.abs(D) > d_min) | ~np.isfinite(gn)
    return np.where(held, gdir, gn), held


def multipixel_interval(plan: MultiPixelPlan, E: np.ndarray, g: np.ndarray, gdir: np.ndarray,
                        gamma: float, d_min: float = 0.0):
    """One multiple-pixel EPICal loop: image the interval's calibration
    pixels with g^{(n)} (Eqs. 8-10), correlate (Eq. 12 per pixel), then the
    joint update of the imaging gains and the per-direction updates.
    E [T][C][Na], g [C][Na], gdir [C][Na][P].
    Returns (g_new, gdir_new, K [C][Na][P], P [C][Na], held [C][Na])."""
    T, C, Na = E.shape
    g = np.asarray(g, np.complex128)
    gdir = np.asarray(gdir, np.complex128)
    gn = np.empty_like(g)
    gdn = np.empty_like(gdir)
    Ks = np.empty(gdir.shape, np.complex128)
    Ps = np.empty(g.shape)
    held = np.zeros(g.shape, bool)
    for c in range(C):
        taps = pixel_taps(plan, apply_gains(E[:, c, :], g[c]) * plan.phase[c], c, plan.pix)
        Ks[c], Ps[c] = correlate_multi(E[:, c, :], taps)
        gn[c], held[c], Cc = multipixel_update(Ks[c], Ps[c], plan.Ap[c], plan.Dp[c], g[c],
                                               gamma, plan.flags, d_min)
        gdn[c], _ = direction_update(Cc, plan.Dp[c], gdir[c], gamma, plan.flags, d_min)
    return gn, gdn, Ks, Ps, held


# --------------------------------------------------------------------------
# visibility-based comparison solve (Sec. 3, Eq. 21) and metrics (Eq. 22)
# --------------------------------------------------------------------------
def visibilities(E: np.ndarray) -> np.ndarray:
    """V_ab = < E_a(t) conj(E_b(t)) >_t.  E: [T][Na]."""
    return (E.T @ np.conj(E)) / E.shape[0]


def baseline_mask(uv: np.ndarray, min_baseline: float) -> np.ndarray:
    """Pairs (a, b) used by the visibility solve: a != b and |u_a - u_b| >=
    min_baseline wavelengths (Sec. 5 leaves out baselines shorter than 10
    wavelengths, where the diffuse sky is not modelled).  uv: [Na][2]."""
    d = np.hypot(uv[:, None, 0] - uv[None, :, 0], uv[:, None, 1] - uv[None, :, 1])
    m = d >= min_baseline
    np.fill_diagonal(m, False)
    return m


def visibility_solve(V, VM, g0, tol: float = 1e-12, max_iter: int = 5000, flags=None,
                     pair_mask=None, return_iters: bool = False):
    """Minimise chi^2 = sum_a sum_{b != a} |V_ab - g_a conj(g_b) V^M_ab|^2
    (Eq. 21).  Reading: the paper does not name its solver; this uses the
    alternating least-squares step with every other iterate averaged
    (StEFCal, Salvini & Wijnholds 2014):
      g_a <- sum_{b!=a} V_ab g_b conj(V^M_ab) / sum_{b!=a} |g_b V^M_ab|^2,
    every antenna from the previous iterate, stopping when
    max_a |g_new - g| <= tol max_a |g_new|.  pair_mask [Na][Na] (optional)
    restricts the sums to the listed pairs (baseline_mask); flagged antennas
    and antennas left without a usable pair keep g0."""
    Na = V.shape[0]
    flags = np.zeros(Na, bool) if flags is None else np.asarray(flags, bool)
    use = ~flags
    pm = ~np.eye(Na, dtype=bool) if pair_mask is None else np.asarray(pair_mask, bool)
    g = np.array(g0, np.complex128)
    for it in range(max_iter):
        gn = g.copy()
        for a in range(Na):
            if flags[a]:
                continue
            m = use & pm[a]
            m[a] = False
            z = g[m] * np.conj(VM[a, m])
            den = np.sum(np.abs(z) ** 2)
            if den > 0:                    # an antenna with no usable pair keeps its gain
                gn[a] = np.sum(V[a, m] * z) / den
        if it % 2 == 1:
            gn = 0.5 * (gn + g)
        if np.max(np.abs(gn - g)) <= tol * np.max(np.abs(gn)):
            return (gn, it + 1) if return_iters else gn
        g = gn
    return (g, max_iter) if return_iters else g


def align_phase(g_est: np.ndarray, g_true: np.ndarray) -> np.ndarray:
    """Remove the unobservable global phase: multiply g_est by
    exp(-i phi) with phi = arg sum_a g_est conj(g_true) (least squares)."""
    phi = np.angle(np.sum(g_est * np.conj(g_true)))
    return g_est * np.exp(-1j * phi)


def gain_error(g_est: np.ndarray, g_true: np.ndarray) -> float:
    """sigma_g of Eq. 22: RMS fractional gain error over antennas and
    channels.  Arrays [C][Na] (or [Na])."""
    g_est = np.atleast_2d(g_est)
    g_true = np.atleast_2d(g_true)
    return float(np.sqrt(np.mean(np.abs(g_est - g_true) ** 2 / np.abs(g_true) ** 2)))


# --------------------------------------------------------------------------
# differentiation form: chi^2 between the dirty image and a sky-model image
# --------------------------------------------------------------------------
def pixel_matrix(plan: Plan, c: int) -> np.ndarray:
    """A_{k,a} for every pixel k of channel c ([N*N][Na], k = ky*N + kx):
    the response of pixel k to antenna a through gridding (Eq. 9) and the
    Eq. 10 transform, E'(s_k) = sum_a A_{k,a} E'_a (with the phasing factor
    p_a of the plan's phase centre).  Explicit sums over taps."""
    N = plan.N
    K = plan.W.shape[-1]
    h = (K - 1) // 2
    A = np.zeros((N * N, plan.Na), np.complex128)
    ky, kx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ky = ky.ravel() - N // 2
    kx = kx.ravel() - N // 2
    for a in range(plan.Na):
        if plan.flags[a]:
            continue
        for dy in range(K):
            for dx in range(K):
                jx = plan.base[c, a, 0] + dx - h - N // 2
                jy = plan.base[c, a, 1] + dy - h - N // 2
                m = np.mod(jx * kx + jy * ky, N)
                A[:, a] += plan.W[c, a, dy, dx] * np.exp(2j * np.pi * m / N)
    return A / plan.norm * plan.phase[c][None, :]


def model_image(plan: Plan, sky_lmS: np.ndarray) -> np.ndarray:
    """Sky-model dirty image [C][N][N]: the Eq. 8-10 imaging operator applied
    to the model visibilities, M_k = sum_ab A_{k,a} conj(A_{k,b}) V^M_ab with
    V^M_ab = sum_s S_s e_a conj(e_b), e_a = exp(-2 pi i u_a . s), i.e.
    M_k = sum_s S_s |sum_a A_{k,a} e_a|^2 (perfectly calibrated, noise free)."""
    C = len(plan.freqs)
    out = np.zeros((C, plan.N, plan.N))
    for c in range(C):
        A = pixel_matrix(plan, c)
        uv = antenna_uv(plan.ant, plan.freqs[c])
        for l, m, S in np.asarray(sky_lmS, np.float64):
            e = np.exp(-2j * np.pi * (uv[:, 0] * l + uv[:, 1] * m))
            out[c] += S * (np.abs(A @ e) ** 2).reshape(plan.N, plan.N)
    return out


def chi2_loss(plan: Plan, E: np.ndarray, g: np.ndarray, M: np.ndarray) -> float:
    """L = sum_c sum_k (I_k(g) - M_k)^2 with I the dirty image of Eqs. 8-10
    and the square-and-average step.  E: [T][C][Na], g: [C][Na]."""
    img, _ = image_interval(plan, E, g)
    return float(np.sum((img - M) ** 2))


def chi2_gradient(plan: Plan, E: np.ndarray, g: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Gradient of chi2_loss with respect to the complex gains, returned in
    the convention grad = 2 dL/dconj(g) (so that dL = Re(conj(grad) dg)).
    With w = 1/g, E'(s_k, t) = sum_a A_{k,a} w_a E_a(t) and R_k = dL/dI_k =
    2 (I_k - M_k):  dL/dconj(w_a) = (1/T) sum_t conj(E_a(t)) sum_k
    conj(A_{k,a}) R_k E'(s_k, t),  dL/dconj(g_a) = dL/dconj(w_a) (-1/conj(g_a)^2).
    Evaluated with explicit A_{k,a} (tiny arrays only)."""
    T, C, Na = E.shape
    img, _ = image_interval(plan, E, g)
    out = np.zeros((C, Na), np.complex128)
    for c in range(C):
        A = pixel_matrix(plan, c)
        R = 2.0 * (img[c] - M[c]).ravel()
        w = 1.0 / g[c]
        Eimg = (E[:, c, :] * w) @ A.T                 # [T][N*N]
        Y = (R[None, :] * Eimg) @ np.conj(A)          # [T][Na]
        dw = np.sum(np.conj(E[:, c, :]) * Y, axis=0) / T
        out[c] = 2.0 * dw * (-1.0 / np.conj(g[c]) ** 2)
    out[:, plan.flags] = 0.0
    return out
