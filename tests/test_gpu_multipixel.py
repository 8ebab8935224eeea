"""Multiple-pixel and direction-dependent EPICal (Sec. 6) on the GPU: the
fused kernel's pixel taps, the [Na x T] x [T x P] correlation and the joint
and per-direction updates against the FP64 oracle on the same bytes."""
import numpy as np
import pytest

import epic_synth as synth
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAIN_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _gain_err(g, ref):
    amp = np.max(np.abs(np.abs(g) - np.abs(ref)) / np.abs(ref))
    ph = np.max(np.abs(np.angle(g * np.conj(ref))))
    return amp, ph


def _pixels_lm(n, cell, pix):
    """Directions (l, m) at the centres of pixels (kx, ky)."""
    return np.array([[(kx - n / 2) / (n * cell), (ky - n / 2) / (n * cell)] for kx, ky in pix])


@pytest.mark.parametrize("n,na,diam,fmt", [(16, 9, 5.0, "c64"), (32, 30, 14.0, "c64"),
                                           (64, 60, 30.0, "ci4"), (128, 200, 70.0, "ci4")])
def test_multipixel_loops_match_oracle(n, na, diam, fmt):
    """Three feedback loops with pixels spread over the image (edges, the
    calibrator, several thread owners and register slots): joint gains and
    per-direction gains after every loop."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(900 + n)
    ant = synth.layout_disc(na, diam, rng, 0.3)
    freqs = [47e6, 61e6]
    flags = np.zeros(na, bool)
    flags[rng.choice(na, max(1, na // 12), replace=False)] = True
    sky = np.array([[0.0, 0.0, 4.0], [0.2, -0.15, 2.0], [-0.3, 0.1, 1.5]])
    pix = [(n // 2, n // 2), (0, 0), (n - 1, n // 2 + 1), (n // 4 + 1, n - 1), (3, n // 2 - 2),
           (n // 2 + 5, 7)]
    pix_lm = _pixels_lm(n, 0.5, pix)
    g_true = synth.true_gains(2, na, rng)
    T = 37
    p = Plan(ant, freqs, n, 0.5, input=fmt, flags=flags,
             voltage_scale=np.array([0.5, 0.7], np.float32) if fmt == "ci4" else None)
    g0 = synth.true_gains(2, na, rng)
    p.configure((0.0, 0.0), sky, 0.4, g0=g0)
    p.configure_pixels(pix_lm)
    oplan = O.MultiPixelPlan(ant, freqs, n, 0.5, pix_lm, sky, flags=flags)
    assert oplan.pix == pix
    g_ref = g0.astype(complex)
    gd_ref = np.repeat(g_ref[:, :, None], len(pix), axis=2)
    for loop in range(3):
        E = synth.voltages(ant, freqs, g_true, sky, T, 1.0, rng)
        if fmt == "ci4":
            lsb = np.array([0.5, 0.7])
            b = synth.quantise_ci4(E, lsb)
            d = torch.from_numpy(b).cuda()
            Eref = O.unpack_ci4(b) * lsb[None, :, None]
        else:
            E = E.astype(np.complex64)
            d = torch.from_numpy(E).cuda()
            Eref = E.astype(np.complex128)
        p.image(d)
        out = torch.zeros((2, na), dtype=torch.complex128, device="cuda")
        p.update(out)
        assert p.sync() == 0
        g_ref, gd_ref, *_ = O.multipixel_interval(oplan, Eref, g_ref, gd_ref, 0.4)
        amp, ph = _gain_err(out.cpu().numpy()[:, ~flags], g_ref[:, ~flags])
        assert amp <= GAIN_TOL and ph <= GAIN_TOL, (loop, amp, ph)
        gd = p.direction_gains()
        amp, ph = _gain_err(gd[:, ~flags], gd_ref[:, ~flags])
        assert amp <= GAIN_TOL and ph <= GAIN_TOL, (loop, "direction", amp, ph)
        assert np.array_equal(out.cpu().numpy()[:, flags], g0[:, flags])


def test_multipixel_one_pixel_equals_single_pixel_path():
    """One calibration pixel at the calibrator: the multiple-pixel form
    gives the single-pixel EPICal update (same interval, two plans)."""
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_time=64, n_chan=3)
    rng = np.random.default_rng(7)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:60], 64, w["noise_power"], rng)
    b = torch.from_numpy(synth.quantise_ci4(E, w["lsb"])).cuda()
    outs = []
    for multi in (False, True):
        p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, input="ci4", voltage_scale=w["lsb"])
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        if multi:
            p.configure_pixels([[0.0, 0.0]])
        for _ in range(2):
            p.image(b)
            p.update()
        outs.append(p.gains())
    amp, ph = _gain_err(outs[1], outs[0])
    assert amp <= 1e-6 and ph <= 1e-6, (amp, ph)


def test_multipixel_noise_free_converges_on_gpu():
    """Three sources with orthogonal tone signals, no noise: the joint and
    per-direction solutions converge to the true gains (global phase)."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(62)
    na = 40
    ant = synth.layout_disc(na, 20.0, rng, 1.0)
    freqs = [50e6]
    sky = np.array([[0.0, 0.0, 4.0], [0.3125, -0.1875, 2.0], [-0.25, 0.375, 1.5]])
    g = synth.true_gains(1, na, rng)
    E = synth.voltages(ant, freqs, g, sky, 64, 0.0, rng, tones=True).astype(np.complex64)
    p = Plan(ant, freqs, 64, 0.5, input="c64")
    p.configure((0.0, 0.0), sky, 0.35)
    p.configure_pixels(sky[:, :2])
    d = torch.from_numpy(E).cuda()
    for _ in range(80):
        p.image(d)
        p.update()
    ga = O.align_phase(p.gains()[0], g[0])
    assert np.max(np.abs(ga - g[0]) / np.abs(g[0])) < 1e-4
    gd = p.direction_gains()[0]
    for q in range(3):
        gq = O.align_phase(gd[:, q], g[0])
        assert np.max(np.abs(gq - g[0]) / np.abs(g[0])) < 1e-4


def test_multipixel_refusals():
    from paper_1603_02126_gb300 import EpicError, Plan
    rng = np.random.default_rng(3)
    ant = synth.layout_disc(20, 12.0, rng, 1.0)
    p = Plan(ant, [50e6], 32, 0.5, input="c64")
    with pytest.raises(EpicError):                      # not configured
        p.configure_pixels([[0.0, 0.0]])
    p.configure((0.0, 0.0), np.array([[0.0, 0.0, 1.0]]), 0.5)
    with pytest.raises(EpicError):                      # same pixel twice
        p.configure_pixels([[0.0, 0.0], [0.001, 0.0]])
    with pytest.raises(EpicError):                      # outside the image
        p.configure_pixels([[1.5, 0.0]])
    pu = Plan(ant, [50e6], 32, 0.5, input="c64", path="unfused")
    pu.configure((0.0, 0.0), np.array([[0.0, 0.0, 1.0]]), 0.5)
    with pytest.raises(EpicError) as ei:
        pu.configure_pixels([[0.0, 0.0]])
    assert ei.value.status == 7
