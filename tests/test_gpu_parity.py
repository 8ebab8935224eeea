"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle
on the same seeded inputs.

Bars: bit-exact unpack and grid indices; image relative L2 <= 1e-5 (FP32
against FP64); gains within 1e-4 in amplitude and 1e-4 rad in phase.
"""
import numpy as np
import pytest

import epic_synth as synth
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
GAIN_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _plan(w, **kw):
    from paper_1603_02126_gb300 import Plan
    return Plan(w["ant_xy"], w["freqs"], w["grid_n"], w["cell"], support=w["kernel_support"],
                param=w["kernel_sigma"], input=w["input"], voltage_scale=w.get("lsb"), **kw)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gain_err(g, ref):
    amp = np.max(np.abs(np.abs(g) - np.abs(ref)) / np.abs(ref))
    ph = np.max(np.abs(np.angle(g * np.conj(ref))))
    return amp, ph


def _lwa_small(n_chan, n_time, n_ant=256, seed=1, flags=None):
    w = synth.workload("lwa", seed=seed, n_time=n_time, n_chan=n_chan, n_ant=n_ant)
    rng = w["rng"]
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:80], n_time,
                       w["noise_power"], rng)
    b = synth.quantise_ci4(E, w["lsb"])
    Eint = O.unpack_ci4(b) * w["lsb"][None, :, None]
    return w, b, Eint


# --------------------------------------------------------------------------
def test_unpack_exhaustive_bit_exact():
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("tiny", n_time=4)
    p = Plan(w["ant_xy"], w["freqs"], 32, 0.5, input="ci4")
    b = np.tile(np.arange(256, dtype=np.uint8), 37)
    d = p.unpack_ci4(torch.from_numpy(b).cuda()).cpu().numpy()
    ref = O.unpack_ci4(b)
    assert np.array_equal(d[:, 0], ref.real.astype(np.float32))
    assert np.array_equal(d[:, 1], ref.imag.astype(np.float32))


@pytest.mark.parametrize("name,n_chan", [("tiny", 1), ("lwa", 64)])
def test_grid_table_bit_exact(name, n_chan):
    w = synth.workload(name, n_chan=n_chan, n_time=4)
    p = _plan(w)
    base, W = p.grid_table()
    ob, oW = O.grid_table(w["ant_xy"], w["freqs"], w["grid_n"], w["cell"], "gaussian",
                          w["kernel_support"], w["kernel_sigma"])
    assert np.array_equal(base, ob)
    assert np.max(np.abs(W - oW)) < 1e-14


def test_grid_table_flags_and_tophat():
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(21)
    ant = synth.layout_disc(45, 30.0, rng, 1.0)
    freqs = [41e6, 57e6, 73e6]
    flags = np.zeros(45, bool)
    flags[[3, 17, 44]] = True
    p = Plan(ant, freqs, 64, 0.5, kernel="tophat", support=5, param=4.4, flags=flags)
    base, W = p.grid_table()
    ob, oW = O.grid_table(ant, freqs, 64, 0.5, "tophat", 5, 4.4, flags)
    assert np.array_equal(base, ob)
    assert np.max(np.abs(W - oW)) < 1e-14


# --------------------------------------------------------------------------
def test_image_tiny_c64():
    w = synth.workload("tiny", n_time=64)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"], 64, w["noise_power"], w["rng"])
    g = synth.true_gains(1, 32, np.random.default_rng(5))
    p = _plan(w)
    p.set_gains(g)
    img = p.image(torch.from_numpy(E.astype(np.complex64)).cuda()).cpu().numpy()
    oplan = O.Plan(w["ant_xy"], w["freqs"], 32, 0.5)
    ref, _ = O.image_interval(oplan, E.astype(np.complex64).astype(np.complex128), g)
    assert _rel(img, ref) <= IMG_TOL


def test_image_lwa_ci4_three_channels_ragged():
    """N = 128, Na = 256, ci4, T not a multiple of the time segmentation."""
    w, b, Eint = _lwa_small(3, 41)
    g = w["gains"]
    p = _plan(w)
    p.set_gains(g)
    img = p.image(torch.from_numpy(b).cuda()).cpu().numpy()
    oplan = O.Plan(w["ant_xy"], w["freqs"], 128, 0.5)
    ref, _ = O.image_interval(oplan, Eint, g)
    for c in range(3):
        assert _rel(img[c], ref[c]) <= IMG_TOL, c


@pytest.mark.parametrize("n,na,k", [(16, 7, 1), (32, 37, 3), (64, 70, 5), (128, 600, 3)])
def test_image_sizes_flags_supports(n, na, k):
    """Grid sizes 16..128, odd antenna counts (incl. more than one per
    thread), flags, kernel supports 1/3/5, two channels."""
    rng = np.random.default_rng(n + na)
    diam = {16: 6.0, 32: 14.0, 64: 30.0, 128: 70.0}[n]
    ant = synth.layout_disc(na, diam, rng, 0.3)
    freqs = [45e6, 62e6]
    flags = np.zeros(na, bool)
    flags[rng.choice(na, max(1, na // 10), replace=False)] = True
    gains = synth.true_gains(2, na, rng)
    sky = np.array([[0.1, -0.2, 3.0], [-0.3, 0.3, 1.0]])
    E = synth.voltages(ant, freqs, gains, sky, 23, 1.0, rng).astype(np.complex64)
    from paper_1603_02126_gb300 import Plan
    p = Plan(ant, freqs, n, 0.5, support=k, param=0.6, input="c64", flags=flags)
    gcur = synth.true_gains(2, na, rng)
    p.set_gains(gcur)
    img = p.image(torch.from_numpy(E).cuda()).cpu().numpy()
    oplan = O.Plan(ant, freqs, n, 0.5, support=k, param=0.6, flags=flags)
    ref, _ = O.image_interval(oplan, E.astype(np.complex128), gcur)
    assert _rel(img, ref) <= IMG_TOL


@pytest.mark.parametrize("path", ["fused", "unfused"])
@pytest.mark.parametrize("n,na,diam", [(32, 40, 57.0), (64, 60, 117.0), (128, 120, 217.0)])
def test_full_window_matches_oracle(n, na, diam, path):
    """An array whose occupied grid window spans more than N/2 cells in both
    channels, so that the fused kernel and the plain path's row and column
    kernels take their unpruned-FFT variants (every lane holds N2 non-zero
    inputs).  Image and one EPICal interval with an off-centre calibrator
    against the oracle; T odd (a one-frame last step)."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(500 + n)
    ant = synth.layout_disc(na, diam, rng, 0.5)
    freqs = [50e6, 60e6]
    base, _ = O.grid_table(ant, freqs, n, 0.5, "gaussian", 3, 0.5)
    for c in range(2):
        span = max(np.ptp(base[c, :, 0]), np.ptp(base[c, :, 1])) + 3
        assert n // 2 < span <= n, (c, span)
    sky = np.array([[0.0625, -0.125, 4.0], [-0.2, 0.25, 1.0]])
    g_true = synth.true_gains(2, na, rng)
    T = 47
    E = synth.voltages(ant, freqs, g_true, sky, T, 1.0, rng).astype(np.complex64)
    p = Plan(ant, freqs, n, 0.5, input="c64", path=path)
    assert p.info()["path"] == {"fused": 1, "unfused": 2}[path]
    cal = (sky[0, 0], sky[0, 1])
    g0 = synth.true_gains(2, na, rng)
    p.configure(cal, sky, 0.5, g0=g0)
    img = p.image(torch.from_numpy(E).cuda()).cpu().numpy()
    out = torch.zeros((2, na), dtype=torch.complex128, device="cuda")
    p.update(out)
    assert p.sync() == 0
    oplan = O.Plan(ant, freqs, n, 0.5, cal_lm=cal, model_lmS=sky)
    Eref = E.astype(np.complex128)
    ref, _ = O.image_interval(oplan, Eref, g0)
    assert _rel(img, ref) <= IMG_TOL
    g_ref, *_ = O.epical_interval(oplan, Eref, g0, 0.5, with_image=False)
    amp, ph = _gain_err(out.cpu().numpy(), g_ref)
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)


@pytest.mark.parametrize("path", ["fused", "unfused"])
def test_heterogeneous_kernels_match_oracle(path):
    """One Gaussian width per antenna (heterogeneous illumination patterns):
    the plan's FP64 taps equal the oracle's, and the image and the EPICal
    interval (A_0 through the per-antenna stencils) match the oracle."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(77)
    na, C, n = 50, 2, 64
    ant = synth.layout_disc(na, 30.0, rng, 0.5)
    freqs = [48e6, 61e6]
    sig = rng.uniform(0.35, 1.0, na)
    sky = np.array([[0.0, 0.0, 4.0], [0.15, -0.2, 1.0]])
    E = synth.voltages(ant, freqs, synth.true_gains(C, na, rng), sky, 40, 1.0, rng).astype(np.complex64)
    p = Plan(ant, freqs, n, 0.5, support=5, param=sig, input="c64", path=path)
    base, W = p.grid_table()
    ob, oW = O.grid_table(ant, freqs, n, 0.5, "gaussian", 5, sig)
    assert np.array_equal(base, ob)
    assert np.max(np.abs(W - oW)) < 1e-14
    p.configure((0.0, 0.0), sky, 0.5)
    img = p.image(torch.from_numpy(E).cuda()).cpu().numpy()
    out = torch.zeros((C, na), dtype=torch.complex128, device="cuda")
    p.update(out)
    assert p.sync() == 0
    oplan = O.Plan(ant, freqs, n, 0.5, support=5, param=sig, model_lmS=sky)
    Eref = E.astype(np.complex128)
    ref, _ = O.image_interval(oplan, Eref, np.ones((C, na), complex))
    assert _rel(img, ref) <= IMG_TOL
    g_ref, *_ = O.epical_interval(oplan, Eref, np.ones((C, na), complex), 0.5, with_image=False)
    amp, ph = _gain_err(out.cpu().numpy(), g_ref)
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)

def test_image_accumulate_and_single_frame():
    w = synth.workload("tiny", n_time=3)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"], 3, w["noise_power"], w["rng"])
    E = E.astype(np.complex64)
    p = _plan(w)
    one = torch.from_numpy(E[:1]).cuda()
    img = p.image(one)
    img2 = p.image(one, img.clone(), accumulate=True)
    # FP64 atomics across time segments add in a run-dependent order
    assert _rel(img2.cpu().numpy(), 2 * img.cpu().numpy()) <= 1e-6
    oplan = O.Plan(w["ant_xy"], w["freqs"], 32, 0.5)
    ref, _ = O.image_interval(oplan, E[:1].astype(np.complex128), np.ones((1, 32)))
    assert _rel(img.cpu().numpy(), ref) <= IMG_TOL


def test_image_host_matches_device():
    w, b, Eint = _lwa_small(2, 16)
    p = _plan(w)
    d = p.image(torch.from_numpy(b).cuda()).cpu().numpy()
    h = p.image_host(b)
    assert np.array_equal(d.shape, h.shape)
    assert _rel(h, d) < 1e-6     # same kernel; FP64 atomic order across segments differs


def test_image_host_long_interval_matches_device_and_epical():
    """The host-buffer call over a 2,100-sample interval: image and one
    EPICal interval against the device call."""
    w, b, Eint = _lwa_small(2, 2100)
    pd, ph = _plan(w), _plan(w)
    for p in (pd, ph):
        p.configure((0.0, 0.0), w["model"], w["gamma"])
    d = pd.image(torch.from_numpy(b).cuda()).cpu().numpy()
    h = ph.image_host(b)
    assert _rel(h, d) < 1e-6
    gd = torch.zeros((2, 256), dtype=torch.complex128, device="cuda")
    gh = torch.zeros((2, 256), dtype=torch.complex128, device="cuda")
    pd.update(gd)
    ph.update(gh)
    assert pd.sync() == 0 and ph.sync() == 0
    amp, phs = _gain_err(gh.cpu().numpy(), gd.cpu().numpy())
    assert amp <= 1e-5 and phs <= 1e-5, (amp, phs)


# --------------------------------------------------------------------------
def test_epical_one_interval_matches_oracle():
    w, b, Eint = _lwa_small(2, 96)
    p = _plan(w)
    p.configure((0.0, 0.0), w["model"], w["gamma"])
    p.image(torch.from_numpy(b).cuda())
    out = torch.zeros((2, 256), dtype=torch.complex128, device="cuda")
    p.update(out)
    assert p.sync() == 0
    oplan = O.Plan(w["ant_xy"], w["freqs"], 128, 0.5, model_lmS=w["model"])
    g_ref, *_ = O.epical_interval(oplan, Eint, np.ones((2, 256), complex), w["gamma"],
                                  with_image=False)
    amp, ph = _gain_err(out.cpu().numpy(), g_ref)
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)


def test_epical_feedback_loop_tiny_matches_oracle():
    """Config-0 geometry and data, 12 loops of T = 2000 complex64 samples,
    gamma = 0.5, calibrator at the phase centre, full sky model."""
    w = synth.workload("tiny")
    T, loops = 2000, 12
    p = _plan(w)
    p.configure((0.0, 0.0), w["model"], w["gamma"])
    oplan = O.Plan(w["ant_xy"], w["freqs"], 32, 0.5, model_lmS=w["model"])
    g_ref = np.ones((1, 32), complex)
    for n in range(loops):
        E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"], T, w["noise_power"],
                           w["rng"]).astype(np.complex64)
        p.image(torch.from_numpy(E).cuda())
        p.update()
        g_ref, *_ = O.epical_interval(oplan, E.astype(np.complex128), g_ref, w["gamma"],
                                      with_image=False)
    g = p.gains()
    amp, ph = _gain_err(g, g_ref)
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)
    # and the solution is near the truth up to a global phase
    assert O.gain_error(O.align_phase(g[0], w["gains"][0]), w["gains"][0]) < 0.2


@pytest.mark.slow
def test_epical_feedback_loop_tiny_full_400_loops():
    """The whole tiny workload: 400 feedback loops of T = 2000 complex64
    samples (8 x 10^5 frames), gamma = 0.5, full sky model, against the
    oracle's loop on the same bytes; gains compared every 50 loops and at
    the end."""
    w = synth.workload("tiny")
    T, loops = 2000, 400
    p = _plan(w)
    p.configure((0.0, 0.0), w["model"], w["gamma"])
    oplan = O.Plan(w["ant_xy"], w["freqs"], 32, 0.5, model_lmS=w["model"])
    g_ref = np.ones((1, 32), complex)
    worst = (0.0, 0.0)
    for n in range(loops):
        E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"], T, w["noise_power"],
                           w["rng"]).astype(np.complex64)
        p.image(torch.from_numpy(E).cuda())
        p.update()
        g_ref, *_ = O.epical_interval(oplan, E.astype(np.complex128), g_ref, w["gamma"],
                                      with_image=False)
        if (n + 1) % 50 == 0:
            amp, ph = _gain_err(p.gains(), g_ref)
            worst = (max(worst[0], amp), max(worst[1], ph))
    assert p.sync() == 0
    assert worst[0] <= GAIN_TOL and worst[1] <= GAIN_TOL, worst
    g = p.gains()[0]
    assert O.gain_error(O.align_phase(g, w["gains"][0]), w["gains"][0]) < 0.05


def test_epical_noise_free_converges_on_gpu():
    rng = np.random.default_rng(31)
    na = 24
    ant = synth.layout_disc(na, 14.0, rng, 1.0)
    sky = np.array([[0.125, -0.0625, 3.0]])
    g_true = synth.true_gains(1, na, rng)
    E = synth.voltages(ant, [50e6], g_true, sky, 64, 0.0, rng, unit_modulus=True)
    from paper_1603_02126_gb300 import Plan
    p = Plan(ant, [50e6], 32, 0.5, input="c64")
    p.configure((0.125, -0.0625), sky, 0.35)
    d = torch.from_numpy(E.astype(np.complex64)).cuda()
    for _ in range(60):
        p.image(d)
        p.update()
    g = p.gains()[0]
    ga = O.align_phase(g, g_true[0])
    assert np.max(np.abs(ga - g_true[0]) / np.abs(g_true[0])) < 1e-4


def test_epical_channel_average_loop_matches_oracle():
    """Gains taken as constant across channels 1..4 of six (Sec. 5): six
    feedback loops, each followed by the channel average, match the oracle's
    loop step for step; the averaged channels end with one gain per antenna
    and the others keep their own."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(41)
    Na, C = 24, 6
    ant = synth.layout_disc(Na, 20.0, rng, 1.0)
    f = np.linspace(49e6, 52e6, C)
    g = np.repeat(synth.true_gains(1, Na, rng), C, axis=0)
    sky = np.array([[0.0, 0.0, 4.0], [0.2, -0.1, 1.0]])
    flags = np.zeros(Na, bool)
    flags[5] = True
    p = Plan(ant, f, 32, 0.5, input="c64", flags=flags)
    p.configure((0.0, 0.0), sky, 0.5)
    oplan = O.Plan(ant, f, 32, 0.5, model_lmS=sky, flags=flags)
    gref = np.ones((C, Na), complex)
    rr = np.random.default_rng(5)
    for _ in range(6):
        E = synth.voltages(ant, f, g, sky, 300, 1.0, rr).astype(np.complex64)
        p.image(torch.from_numpy(E).cuda())
        p.update()
        p.average_channels(1, 5)
        gref, *_ = O.epical_interval(oplan, E.astype(np.complex128), gref, 0.5, with_image=False)
        gref = O.average_channels(gref, 1, 5, flags)
    gg = p.gains()
    live = ~flags
    amp, ph = _gain_err(gg[:, live], gref[:, live])
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)
    assert np.array_equal(gg[1:5], np.repeat(gg[1:2], 4, axis=0))
    assert not np.allclose(gg[0, live], gg[1, live])

def test_epical_held_antennas_and_state_roundtrip():
    w, b, Eint = _lwa_small(1, 32, n_ant=64)
    flags = np.zeros(64, bool)
    flags[5] = True
    p = _plan(w, flags=flags)
    p.configure((0.0, 0.0), w["model"], w["gamma"])
    d = torch.from_numpy(b).cuda()
    p.image(d)
    st = torch.zeros((1, 64), dtype=torch.int32, device="cuda")
    p.update(None, st)
    assert p.sync() == 0
    assert st.cpu().numpy()[0, 5] == 1 and st.cpu().numpy().sum() == 1
    g1 = p.gains()
    assert g1[0, 5] == 1.0
    p.image(d)
    state = p.get_state()
    p.update()
    g2 = p.gains()
    p.set_state(state)
    p.update()
    assert np.array_equal(p.gains(), g2)
    from paper_1603_02126_gb300 import EpicError
    with pytest.raises(EpicError):
        p.update()          # no frames since the last update


# --------------------------------------------------------------------------
def test_full_size_lwa_sampled():
    """The full LWA-like interval (Na=256, C=64, N=128, T=10^4, ci4) in the
    benchmark's launch configuration, checked at sampled pixels and
    antennas against the oracle's single-pixel sums."""
    w = synth.workload("lwa")
    d = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"], w["n_time"],
                                 w["noise_power"], w["lsb"], seed=1)
    p = _plan(w)
    p.configure((0.0, 0.0), w["model"], w["gamma"])
    img = p.image(d).cpu().numpy()
    kacc_out = torch.zeros((64, 256), dtype=torch.complex128, device="cuda")
    p.update(kacc_out)
    p.sync()
    g_gpu = kacc_out.cpu().numpy()
    rng = np.random.default_rng(0)
    for c in (0, 37, 63):
        Eint = O.unpack_ci4(d[:, c:c + 1, :].cpu().numpy()) * w["lsb"][c]
        pix = [(64, 64), (int(rng.integers(128)), int(rng.integers(128))), (0, 127)]
        sub = O.Plan(w["ant_xy"], [w["freqs"][c]], 128, 0.5, model_lmS=w["model"])
        ref = O.image_pixels(sub, Eint, np.ones((1, 256)), 0, pix)
        for i, (kx, ky) in enumerate(pix):
            assert abs(img[c, ky, kx] - ref[i]) <= 1e-5 * abs(ref[i]) + 1e-6 * img[c].max()
        ants = [0, 101, 255]
        Kc, P = O.correlate_sampled(sub, Eint, np.ones((1, 256)), 0, ants)
        gs, _ = O.epical_update(Kc, P, sub.A0[0, ants], sub.D[0, ants], np.ones(3, complex),
                                w["gamma"])
        amp, ph = _gain_err(g_gpu[c, ants], gs)
        assert amp <= GAIN_TOL and ph <= GAIN_TOL, (c, amp, ph)


@pytest.mark.parametrize("armed", [False, True])
def test_image_many_units_per_cta(armed):
    """More time segments than CTAs, so CTAs carry several work units; full
    LWA-like sky; with and without the EPICal correlation armed."""
    w = synth.workload("lwa", n_chan=1, n_time=4000)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"], 4000, w["noise_power"],
                       w["rng"])
    b = synth.quantise_ci4(E, w["lsb"])
    Eint = O.unpack_ci4(b) * w["lsb"][None, :, None]
    p = _plan(w)
    if armed:
        p.configure((0.0, 0.0), w["model"], w["gamma"])
    img = p.image(torch.from_numpy(b).cuda()).cpu().numpy()
    oplan = O.Plan(w["ant_xy"], w["freqs"], 128, 0.5)
    ref, _ = O.image_interval(oplan, Eint, np.ones((1, 256)))
    assert _rel(img, ref) <= IMG_TOL


@pytest.mark.parametrize("path", ["fused", "unfused"])
def test_gather_limit_255_taps_per_cell(path):
    """The gather lists hold at most 255 taps per grid cell: 255 co-located
    antennas still image exactly (every tap of the 3x3 stencil lands 255
    times on the same cell), 256 are refused with UNSUPPORTED."""
    from paper_1603_02126_gb300 import Plan
    from paper_1603_02126_gb300._binding import EpicError
    rng = np.random.default_rng(255)
    freqs = [50e6]
    ant = np.tile([[3.0, -2.0]], (255, 1))
    E = (rng.standard_normal((5, 1, 255)) + 1j * rng.standard_normal((5, 1, 255))).astype(np.complex64)
    p = Plan(ant, freqs, 32, 0.5, input="c64", path=path)
    img = p.image(torch.from_numpy(E).cuda()).cpu().numpy()
    ref, _ = O.image_interval(O.Plan(ant, freqs, 32, 0.5), E.astype(np.complex128), np.ones((1, 255)))
    assert _rel(img, ref) <= IMG_TOL
    with pytest.raises(EpicError) as ei:
        Plan(np.tile([[3.0, -2.0]], (256, 1)), freqs, 32, 0.5, input="c64", path=path)
    assert ei.value.status == 7
