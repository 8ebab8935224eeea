"""Seeded synthetic inputs for the EPIC/EPICal tests and benchmark.

This module draws array layouts, sky models, antenna gains and channelised
antenna voltages.  It holds none of the imaging or calibration arithmetic
(no gain correction, gridding, Fourier imaging, correlation or gain update):
both the FP64 oracle and the CUDA library consume what it writes, and it
imports neither of them.

Data model (the paper's measurement equation, used only to make test data):
  E_a(f,t) = g_a(f) * sum_s sqrt(S_s) z_s(t) exp(-2 pi i u_a . s_s) + n_a(t)
with u_a = r_a f / c in wavelengths (Sec. 2.1, Eq. 3 propagation and Eq. 7
gain/noise corruption).  Source signals z_s are complex Gaussian with unit
variance (Sec. 3: the source amplitudes vary randomly in time) or, for the
noise-free convergence pins, unit-modulus phasors.

4-bit complex input format: one byte per (t, c, a); the high nibble holds the
real part and the low nibble the imaginary part, each a two's-complement
integer in [-8, 7].
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299792458.0  # m/s


# --------------------------------------------------------------------------
# array layouts (metres, East = x, North = y)
# --------------------------------------------------------------------------
def layout_disc(n_ant: int, diameter_m: float, rng: np.random.Generator,
                min_sep_m: float = 0.0) -> np.ndarray:
    """Uniform-random positions inside a disc, optional minimum separation."""
    return layout_ellipse(n_ant, diameter_m / 2, diameter_m / 2, rng, min_sep_m)


def layout_ellipse(n_ant: int, semi_x_m: float, semi_y_m: float,
                   rng: np.random.Generator, min_sep_m: float = 0.0) -> np.ndarray:
    """Uniform-random positions inside an ellipse (rejection sampling)."""
    out = np.empty((n_ant, 2))
    k = 0
    tries = 0
    while k < n_ant:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place antennas with that separation")
        x, y = rng.uniform(-1.0, 1.0, size=2)
        if x * x + y * y > 1.0:
            continue
        p = np.array([x * semi_x_m, y * semi_y_m])
        if min_sep_m > 0 and k > 0:
            if np.min(np.hypot(*(out[:k] - p).T)) < min_sep_m:
                continue
        out[k] = p
        k += 1
    return out


def layout_hex(n_ant: int, pitch_m: float, jitter_m: float,
               rng: np.random.Generator) -> np.ndarray:
    """Hexagonal lattice (closest points to the centre) plus uniform jitter."""
    r = int(np.ceil(np.sqrt(n_ant))) + 2
    pts = []
    for i in range(-r, r + 1):
        for j in range(-r, r + 1):
            pts.append((pitch_m * (i + 0.5 * j), pitch_m * (np.sqrt(3) / 2) * j))
    pts = np.array(pts)
    pts = pts[np.argsort(np.hypot(pts[:, 0], pts[:, 1]), kind="stable")[:n_ant]]
    return pts + rng.uniform(-jitter_m, jitter_m, size=pts.shape)


def channels(n_chan: int, f_lo_hz: float, f_hi_hz: float) -> np.ndarray:
    """Channel centre frequencies, evenly spaced across [f_lo, f_hi]."""
    if n_chan == 1:
        return np.array([f_lo_hz])
    return np.linspace(f_lo_hz, f_hi_hz, n_chan)


# --------------------------------------------------------------------------
# gains and skies
# --------------------------------------------------------------------------
def true_gains(n_chan: int, n_ant: int, rng: np.random.Generator,
               amp_sigma: float = 0.1) -> np.ndarray:
    """|g| ~ N(1, amp_sigma) redrawn while <= 0, arg g ~ U[-pi, pi)."""
    amp = rng.normal(1.0, amp_sigma, size=(n_chan, n_ant))
    bad = amp <= 0
    while bad.any():
        amp[bad] = rng.normal(1.0, amp_sigma, size=bad.sum())
        bad = amp <= 0
    ph = rng.uniform(-np.pi, np.pi, size=(n_chan, n_ant))
    return amp * np.exp(1j * ph)


def random_directions(n: int, rng: np.random.Generator, r2_max: float = 1.0) -> np.ndarray:
    """(l, m) uniform inside l^2 + m^2 < r2_max."""
    out = np.empty((n, 2))
    k = 0
    while k < n:
        l, m = rng.uniform(-1.0, 1.0, size=2) * np.sqrt(r2_max)
        if l * l + m * m < r2_max:
            out[k] = (l, m)
            k += 1
    return out


def sky_tiny(rng: np.random.Generator) -> np.ndarray:
    """10 Jy calibrator at the phase centre + 3 sources, S ~ U[0.5, 2],
    l^2 + m^2 < 0.5.  Rows are (l, m, S)."""
    lm = random_directions(3, rng, 0.5)
    s = rng.uniform(0.5, 2.0, size=3)
    return np.vstack([[0.0, 0.0, 10.0], np.column_stack([lm, s])])


def sky_powerlaw(n_src: int, s_min: float, s_max: float,
                 rng: np.random.Generator) -> np.ndarray:
    """Point sources with dN/dS ~ S^-2 on [s_min, s_max]; the brightest is
    moved to the phase centre as the calibrator.  Rows are (l, m, S)."""
    u = rng.uniform(size=n_src)
    s = 1.0 / (1.0 / s_min - u * (1.0 / s_min - 1.0 / s_max))
    lm = random_directions(n_src, rng, 0.5)
    i = int(np.argmax(s))
    lm[i] = (0.0, 0.0)
    order = np.r_[i, np.delete(np.arange(n_src), i)]
    return np.column_stack([lm, s])[order]


def sky_diffuse(n_src: int, total_flux: float, rng: np.random.Generator) -> np.ndarray:
    """Faint sources at random directions in l^2+m^2<1 with exponential
    fluxes scaled to `total_flux` (stand-in for a diffuse sky)."""
    lm = random_directions(n_src, rng, 1.0)
    s = rng.exponential(1.0, size=n_src)
    s *= total_flux / s.sum()
    return np.column_stack([lm, s])


# --------------------------------------------------------------------------
# voltages
# --------------------------------------------------------------------------
def voltages(ant_xy_m: np.ndarray, freq_hz: np.ndarray, gains: np.ndarray,
             sky_lmS: np.ndarray, n_time: int, noise_power: float,
             rng: np.random.Generator, unit_modulus: bool = False,
             tones: bool = False) -> np.ndarray:
    """Channelised antenna voltages, complex128 [T][C][Na].

    gains: [C][Na] complex, or [C][Na][Ns] for gains that differ by source
    direction.  sky_lmS: [Ns][3] rows (l, m, S).  noise_power: <|n_a|^2> per
    sample (0 = noise free).  unit_modulus: source signals are exp(i theta_t)
    with theta uniform (so <|z|^2> = 1 exactly per sample).  tones: source s
    is the unit-modulus tone exp(2 pi i (k_s t / T + phi_s)) with distinct
    integers k_s, so that different sources are exactly uncorrelated over
    the T samples (noise-free sample visibilities equal the model).
    """
    ant = np.asarray(ant_xy_m, float)
    T, C, Na, Ns = n_time, len(freq_hz), ant.shape[0], sky_lmS.shape[0]
    out = np.empty((T, C, Na), np.complex128)
    amp = np.sqrt(sky_lmS[:, 2])
    gains = np.asarray(gains)
    for c, f in enumerate(freq_hz):
        u = ant * f / C_LIGHT                                   # [Na][2]
        ph = np.exp(-2j * np.pi * (u @ sky_lmS[:, :2].T))      # [Na][Ns]
        if tones:
            if Ns >= T:
                raise ValueError("tones need fewer sources than samples")
            k = rng.choice(np.arange(1, T), size=Ns, replace=False)
            phi = rng.uniform(0.0, 1.0, size=Ns)
            z = np.exp(2j * np.pi * (np.outer(np.arange(T), k) / T + phi[None, :]))
        elif unit_modulus:
            z = np.exp(1j * rng.uniform(-np.pi, np.pi, size=(T, Ns)))
        else:
            z = (rng.normal(size=(T, Ns)) + 1j * rng.normal(size=(T, Ns))) / np.sqrt(2)
        if gains.ndim == 3:                                     # direction-dependent
            e = (z * amp) @ (ph * gains[c]).T
        else:
            e = (z * amp) @ ph.T                                # [T][Na]
            e = e * gains[c][None, :]
        if noise_power > 0:
            e = e + np.sqrt(noise_power / 2) * (rng.normal(size=(T, Na))
                                                + 1j * rng.normal(size=(T, Na)))
        out[:, c, :] = e
    return out


def quantise_ci4(e: np.ndarray, lsb: np.ndarray | float) -> np.ndarray:
    """Round e / lsb to integers, clip each part to [-7, 7] and pack into one
    byte per sample (high nibble = real, low nibble = imaginary).
    lsb broadcasts against the channel axis of e ([T][C][Na] -> lsb [C])."""
    lsb = np.asarray(lsb, float)
    if lsb.ndim == 1:
        lsb = lsb[None, :, None]
    re = np.clip(np.rint(e.real / lsb), -7, 7).astype(np.int64)
    im = np.clip(np.rint(e.imag / lsb), -7, 7).astype(np.int64)
    return (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)


def pack_ci4(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack integer parts in [-8, 7] into the 4-bit complex byte format."""
    re = np.asarray(re, np.int64)
    im = np.asarray(im, np.int64)
    return (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def workload(name: str, seed: int | None = None, n_time: int | None = None,
             n_chan: int | None = None, n_ant: int | None = None):
    """Return a dict describing one synthetic workload (small sizes can be
    overridden for tests).  Keys: ant_xy, freqs, grid_n, cell, kernel_support,
    kernel_sigma, gains, sky, model, n_time, noise_power, input ('ci4' or
    'c64'), gamma, lsb (per-channel ci4 step, or None)."""
    if name == "tiny":             # Na=32, 20 m disc, 1 ch @ 50 MHz, 32^2 grid
        rng = np.random.default_rng(0 if seed is None else seed)
        na = n_ant or 32
        ant = layout_disc(na, 20.0, rng, min_sep_m=1.0)
        freqs = channels(n_chan or 1, 50e6, 50e6)
        gains = true_gains(len(freqs), na, rng)
        sky = sky_tiny(rng)
        return dict(ant_xy=ant, freqs=freqs, grid_n=32, cell=0.5, kernel_support=3,
                    kernel_sigma=0.5, gains=gains, sky=sky, model=sky,
                    n_time=n_time or 2000, noise_power=sky[:, 2].sum() / 5.0,
                    input="c64", gamma=0.5, lsb=None, rng=rng)
    if name in ("lwa", "lwa_diff"):  # Na=256, 100 m x 90 m ellipse, 40-80 MHz, 128^2
        rng = np.random.default_rng((1 if name == "lwa" else 4) if seed is None else seed)
        na = n_ant or 256
        ant = layout_ellipse(na, 50.0, 45.0, rng, min_sep_m=2.0)
        nc = n_chan or (64 if name == "lwa" else 16)
        freqs = channels(nc, 40e6, 80e6)
        gains = true_gains(nc, na, rng)
        pts = sky_powerlaw(50, 0.5, 50.0, rng)
        diffuse = sky_diffuse(1000, pts[:, 2].sum(), rng)
        sky = np.vstack([pts, diffuse])
        noise = sky[:, 2].sum() / 5.0
        # ci4 step: per-component RMS of the data ~ 2 LSB
        rms = np.sqrt((sky[:, 2].sum() * np.mean(np.abs(gains) ** 2) + noise) / 2)
        lsb = np.full(nc, rms / 2.0)
        return dict(ant_xy=ant, freqs=freqs, grid_n=128, cell=0.5, kernel_support=3,
                    kernel_sigma=0.5, gains=gains, sky=sky, model=pts,
                    n_time=n_time or (10000 if name == "lwa" else 4096),
                    noise_power=noise, input="ci4", gamma=0.5, lsb=lsb, rng=rng)
    if name == "noise":            # Sec. 4 sky on the LWA-like array: 5 Jy + 49 x U[0.2, 0.5] Jy
        rng = np.random.default_rng(5 if seed is None else seed)
        na = n_ant or 256
        ant = layout_ellipse(na, 50.0, 45.0, rng, min_sep_m=2.0)
        nc = n_chan or 64
        freqs = channels(nc, 40e6, 80e6)
        faint = np.column_stack([random_directions(49, rng, 0.5), rng.uniform(0.2, 0.5, 49)])
        sky = np.vstack([[0.0, 0.0, 5.0], faint])
        return dict(ant_xy=ant, freqs=freqs, grid_n=128, cell=0.5, kernel_support=3,
                    kernel_sigma=0.5, gains=np.ones((nc, na), complex), sky=sky, model=sky,
                    model_single=sky[:1], n_time=n_time or 1024, noise_power=10.0,
                    input="ci4", gamma=0.35, lsb=None, rng=rng)
    if name == "compact1024":      # Na=1024 in a 200 m disc, 32 ch 40-80 MHz, 256^2, 4-bit
        rng = np.random.default_rng(2 if seed is None else seed)
        na = n_ant or 1024
        ant = layout_disc(na, 200.0, rng, min_sep_m=2.0)
        nc = n_chan or 32
        freqs = channels(nc, 40e6, 80e6)
        gains = true_gains(nc, na, rng)
        pts = sky_powerlaw(50, 0.5, 50.0, rng)
        sky = np.vstack([pts, sky_diffuse(1000, pts[:, 2].sum(), rng)])
        noise = sky[:, 2].sum() / 5.0
        rms = np.sqrt((sky[:, 2].sum() * np.mean(np.abs(gains) ** 2) + noise) / 2)
        return dict(ant_xy=ant, freqs=freqs, grid_n=256, cell=0.5, kernel_support=3,
                    kernel_sigma=0.5, gains=gains, sky=sky, model=pts,
                    n_time=n_time or 4096, noise_power=noise, input="ci4", gamma=0.5,
                    lsb=np.full(nc, rms / 2.0), rng=rng)
    if name == "hex2048":          # Na=2048 hexagonal 8 m pitch +-0.5 m, 256 ch 50-100 MHz, 512^2
        rng = np.random.default_rng(3 if seed is None else seed)
        na = n_ant or 2048
        ant = layout_hex(na, 8.0, 0.5, rng)
        nc = n_chan or 256
        freqs = channels(nc, 50e6, 100e6)
        gains = true_gains(nc, na, rng)
        pts = sky_powerlaw(50, 0.5, 50.0, rng)
        sky = np.vstack([pts, sky_diffuse(200, pts[:, 2].sum(), rng)])
        noise = sky[:, 2].sum() / 5.0
        return dict(ant_xy=ant, freqs=freqs, grid_n=512, cell=0.5, kernel_support=3,
                    kernel_sigma=0.5, gains=gains, sky=sky, model=pts,
                    n_time=n_time or 4096, noise_power=noise, input="c64", gamma=0.5,
                    lsb=None, rng=rng)
    raise ValueError(name)


def voltages_ci4_torch(ant_xy_m, freq_hz, gains, sky_lmS, n_time, noise_power, lsb,
                       seed: int, device="cuda", chunk: int = 4096):
    """Large-workload generator on a torch device: the same data model as
    `voltages`, drawn with a seeded torch.Generator, quantised straight to
    the 4-bit byte format.  Returns a uint8 tensor [T][C][Na] on `device`."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    ant = torch.as_tensor(np.asarray(ant_xy_m, np.float64), device=device)
    sky = torch.as_tensor(np.asarray(sky_lmS, np.float64), device=device)
    T, C, Na, Ns = int(n_time), len(freq_hz), ant.shape[0], sky.shape[0]
    out = torch.empty((T, C, Na), dtype=torch.uint8, device=device)
    amp = torch.sqrt(sky[:, 2]).to(torch.float32)
    g = torch.as_tensor(np.asarray(gains), device=device).to(torch.complex64)
    for c, f in enumerate(freq_hz):
        u = ant * float(f) / C_LIGHT
        ph = torch.exp(-2j * np.pi * (u @ sky[:, :2].T)).to(torch.complex64)   # [Na][Ns]
        q = float(np.asarray(lsb).reshape(-1)[c]) if np.ndim(lsb) else float(lsb)
        for t0 in range(0, T, chunk):
            n = min(chunk, T - t0)
            zr = torch.randn((n, Ns), generator=gen, device=device)
            zi = torch.randn((n, Ns), generator=gen, device=device)
            z = torch.complex(zr, zi) * (amp / np.sqrt(2.0))
            e = (z @ ph.T) * g[c][None, :]
            if noise_power > 0:
                nr = torch.randn((n, Na), generator=gen, device=device)
                ni = torch.randn((n, Na), generator=gen, device=device)
                e = e + torch.complex(nr, ni) * float(np.sqrt(noise_power / 2))
            re = torch.clamp(torch.round(e.real / q), -7, 7).to(torch.int32)
            im = torch.clamp(torch.round(e.imag / q), -7, 7).to(torch.int32)
            out[t0:t0 + n, c, :] = (((re & 15) << 4) | (im & 15)).to(torch.uint8)
    return out


def voltages_c64_torch(ant_xy_m, freq_hz, gains, sky_lmS, n_time, noise_power, seed: int,
                       device="cuda", chunk: int = 2048):
    """Large-workload generator: complex64 voltages [T][C][Na] on `device`,
    same data model as `voltages`, seeded torch.Generator."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    ant = torch.as_tensor(np.asarray(ant_xy_m, np.float64), device=device)
    sky = torch.as_tensor(np.asarray(sky_lmS, np.float64), device=device)
    T, C, Na, Ns = int(n_time), len(freq_hz), ant.shape[0], sky.shape[0]
    out = torch.empty((T, C, Na), dtype=torch.complex64, device=device)
    amp = torch.sqrt(sky[:, 2]).to(torch.float32)
    g = torch.as_tensor(np.asarray(gains), device=device).to(torch.complex64)
    for c, f in enumerate(freq_hz):
        u = ant * float(f) / C_LIGHT
        ph = torch.exp(-2j * np.pi * (u @ sky[:, :2].T)).to(torch.complex64)
        for t0 in range(0, T, chunk):
            n = min(chunk, T - t0)
            z = torch.complex(torch.randn((n, Ns), generator=gen, device=device),
                              torch.randn((n, Ns), generator=gen, device=device)) * (amp / np.sqrt(2.0))
            e = (z @ ph.T) * g[c][None, :]
            if noise_power > 0:
                e = e + torch.complex(torch.randn((n, Na), generator=gen, device=device),
                                      torch.randn((n, Na), generator=gen, device=device)) * float(
                                          np.sqrt(noise_power / 2))
            out[t0:t0 + n, c, :] = e
    return out


def model_frames_c64(ant_xy_m, freq_hz, sky_lmS) -> np.ndarray:
    """One noise-free frame per model source, sqrt(S_s) exp(-2 pi i u_a . s_s),
    complex64 [Ns][C][Na]: imaged with unit gains and multiplied by Ns they
    give the sky-model image sum_s S_s |sum_a A_{k,a} e_a|^2."""
    ant = np.asarray(ant_xy_m, float)
    out = np.empty((len(sky_lmS), len(freq_hz), ant.shape[0]), np.complex64)
    for c, f in enumerate(freq_hz):
        u = ant * f / C_LIGHT
        for i, (l, m, S) in enumerate(np.asarray(sky_lmS, float)):
            out[i, c] = np.sqrt(S) * np.exp(-2j * np.pi * (u[:, 0] * l + u[:, 1] * m))
    return out
