"""Phasing to a phase centre off zenith (Sec. 2.1 footnote) and the
polynomial bandpass model across channels (Sec. 6) on the GPU, against the
FP64 oracle."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gain_err(g, ref):
    amp = np.max(np.abs(np.abs(g) - np.abs(ref)) / np.abs(ref))
    ph = np.max(np.abs(np.angle(g * np.conj(ref))))
    return amp, ph


@pytest.mark.parametrize("path,n", [("fused", 64), ("unfused", 64), ("fused", 128)])
def test_phased_image_and_epical_match_oracle(path, n):
    """Array phased to s0 = (0.4, -0.3), calibrator there: image and one
    EPICal interval (feedback gains g0) against the oracle."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(300 + n)
    na = 60 if n == 64 else 150
    ant = synth.layout_disc(na, 30.0 if n == 64 else 60.0, rng, 0.5)
    freqs = [48e6, 63e6]
    s0 = (0.4, -0.3)
    sky = np.array([[s0[0], s0[1], 4.0], [0.2, 0.1, 1.0], [0.55, -0.45, 1.5]])
    flags = np.zeros(na, bool)
    flags[[2, 9]] = True
    E = synth.voltages(ant, freqs, synth.true_gains(2, na, rng), sky, 41, 1.0, rng).astype(np.complex64)
    g0 = synth.true_gains(2, na, rng)
    p = Plan(ant, freqs, n, 0.5, input="c64", path=path, flags=flags)
    p.set_phase_centre(*s0)
    p.configure(s0, sky, 0.5, g0=g0)
    assert (p.info()["cal_kx"], p.info()["cal_ky"]) == (n // 2, n // 2)
    img = p.image(torch.from_numpy(E).cuda()).cpu().numpy()
    out = torch.zeros((2, na), dtype=torch.complex128, device="cuda")
    p.update(out)
    assert p.sync() == 0
    oplan = O.Plan(ant, freqs, n, 0.5, cal_lm=s0, model_lmS=sky, phase_lm=s0, flags=flags)
    Eref = E.astype(np.complex128)
    ref, _ = O.image_interval(oplan, Eref, g0)
    assert _rel(img, ref) <= IMG_TOL
    g_ref, *_ = O.epical_interval(oplan, Eref, g0, 0.5, with_image=False)
    amp, ph = _gain_err(out.cpu().numpy()[:, ~flags], g_ref[:, ~flags])
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)


def test_phased_image_is_shifted_sky_on_gpu():
    """Noise-free: the phased GPU image of a sky equals the zenith GPU image
    of that sky moved by -s0 (same source signals)."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(81)
    na = 40
    ant = synth.layout_disc(na, 20.0, rng, 0.5)
    s0 = (-0.25, 0.3125)
    sky = np.array([[0.1, 0.2, 3.0], [-0.3, 0.45, 1.0]])
    g = synth.true_gains(1, na, rng)
    E = synth.voltages(ant, [55e6], g, sky, 30, 0.0, np.random.default_rng(9)).astype(np.complex64)
    Es = synth.voltages(ant, [55e6], g, sky - np.array([s0[0], s0[1], 0.0]), 30, 0.0,
                        np.random.default_rng(9)).astype(np.complex64)
    p = Plan(ant, [55e6], 64, 0.5, input="c64")
    zen = p.image(torch.from_numpy(Es).cuda()).cpu().numpy()
    p.set_phase_centre(*s0)
    ph = p.image(torch.from_numpy(E).cuda()).cpu().numpy()
    assert _rel(ph, zen) <= 2 * IMG_TOL


def test_phased_gradient_matches_oracle():
    from paper_1603_02126_gb300 import Plan
    from paper_1603_02126_gb300.autograd import EpicImageFn, chi2
    rng = np.random.default_rng(12)
    na, n = 16, 32
    ant = synth.layout_disc(na, 12.0, rng, 0.8)
    freqs = [46e6, 60e6]
    s0 = (0.3, 0.2)
    sky = np.array([[0.3, 0.2, 4.0], [0.45, 0.1, 1.5]])
    g_true = synth.true_gains(2, na, rng)
    E = synth.voltages(ant, freqs, g_true, sky, 40, 0.3, rng).astype(np.complex64)
    g = g_true * (1 + 0.15 * (rng.normal(size=g_true.shape) + 1j * rng.normal(size=g_true.shape)))
    oplan = O.Plan(ant, freqs, n, 0.5, phase_lm=s0)
    M = O.model_image(oplan, sky)
    ref = O.chi2_gradient(oplan, E.astype(np.complex128), g, M)
    p = Plan(ant, freqs, n, 0.5, input="c64")
    p.set_phase_centre(*s0)
    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    chi2(EpicImageFn.apply(gt, torch.from_numpy(E).cuda(), p), torch.from_numpy(M).cuda()).backward()
    grad = gt.grad.cpu().numpy()
    assert np.linalg.norm(grad - ref) / np.linalg.norm(ref) <= 1e-4


def test_fit_bandpass_matches_oracle():
    """Noisy per-channel gains around smooth bandpasses with phase slopes
    that wrap: the GPU fit (degrees 2 and 3, band 5..59 of 64 channels, one
    flagged antenna) equals the oracle's; other channels untouched."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(73)
    C, Na = 64, 48
    ant = synth.layout_disc(Na, 30.0, rng, 0.5)
    freqs = np.linspace(40e6, 80e6, C)
    x = O.bandpass_x(freqs, 0, C)
    true = np.empty((C, Na), complex)
    for a in range(Na):
        c0, c1 = rng.normal(size=2)
        true[:, a] = (1.0 + 0.1 * c0 * x) * np.exp(1j * (rng.uniform(-np.pi, np.pi) + 8.0 * c1 * x))
    noisy = true * (1 + 0.05 * (rng.normal(size=(C, Na)) + 1j * rng.normal(size=(C, Na))))
    flags = np.zeros(Na, bool)
    flags[7] = True
    p = Plan(ant, freqs, 64, 0.5, input="c64", flags=flags)
    p.set_gains(noisy)
    p.fit_bandpass(5, 59, 2, 3)
    got = p.gains()
    ref = O.fit_bandpass(noisy, freqs, 5, 59, 2, 3, flags)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-9
    assert np.array_equal(got[:5], noisy[:5]) and np.array_equal(got[59:], noisy[59:])
    assert np.array_equal(got[:, 7], noisy[:, 7])
