"""Reduced-precision form on the GPU: the row and column DFTs on tcgen05
tensor cores in FP16 and BF16 (FP32 accumulation, per-frame power-of-two
scaling), FP32 gridding, FP64 image accumulation.  Each case states its image
error against the FP64 oracle; the bar is relative L2 <= 3e-3."""
import numpy as np
import pytest

import epic_synth as synth
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LP_TOL = 3e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _lp_case(n, na, diam, C, T, seed):
    rng = np.random.default_rng(seed)
    ant = synth.layout_disc(na, diam, rng, 0.5)
    freqs = np.linspace(42e6, 78e6, C)
    gains = synth.true_gains(C, na, rng)
    sky = np.vstack([[0.0, 0.0, 20.0], synth.sky_powerlaw(20, 0.5, 5.0, rng)[1:],
                     synth.sky_diffuse(200, 20.0, rng)])
    E = synth.voltages(ant, freqs, gains, sky, T, sky[:, 2].sum() / 5, rng)
    rms = np.sqrt(np.mean(np.abs(E) ** 2) / 2)
    lsb = np.full(C, rms / 2)
    b = synth.quantise_ci4(E, lsb)
    Eint = O.unpack_ci4(b) * lsb[None, :, None]
    return ant, freqs, gains, lsb, b, Eint


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n,na,diam,C,T", [(128, 256, 80.0, 2, 150), (256, 600, 170.0, 1, 70)])
def test_tensor_core_image_error(prec, n, na, diam, C, T):
    from paper_1603_02126_gb300 import Plan
    ant, freqs, gains, lsb, b, Eint = _lp_case(n, na, diam, C, T, seed=n + C)
    p = Plan(ant, freqs, n, 0.5, input="ci4", voltage_scale=lsb, precision=prec)
    gcur = synth.true_gains(C, na, np.random.default_rng(1))
    p.set_gains(gcur)
    img = p.image(torch.from_numpy(b).cuda()).cpu().numpy()
    assert p.sync() == 0
    ref, _ = O.image_interval(O.Plan(ant, freqs, n, 0.5), Eint, gcur)
    err = _rel(img, ref)
    print(f"{prec} N={n} image rel-L2 vs FP64 oracle: {err:.3e}")
    assert err <= LP_TOL


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tensor_core_wide_window(prec):
    """An array elongated in x (about 228 x 120 occupied cells at N = 256):
    the row DFT's K extent is 2 x 256 window columns (eight 64-element
    chunks per tile) against 2 x 128 in the square cases."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(91)
    ant = synth.layout_ellipse(300, 290.0, 150.0, rng, 1.0)
    freqs = np.array([60e6])
    sky = np.vstack([[0.0, 0.0, 20.0], synth.sky_powerlaw(10, 0.5, 5.0, rng)[1:]])
    gains = synth.true_gains(1, 300, rng)
    E = synth.voltages(ant, freqs, gains, sky, 40, sky[:, 2].sum() / 5, rng)
    lsb = np.full(1, np.sqrt(np.mean(np.abs(E) ** 2) / 2) / 2)
    b = synth.quantise_ci4(E, lsb)
    Eint = O.unpack_ci4(b) * lsb[None, :, None]
    oplan = O.Plan(ant, freqs, 256, 0.5)
    bx, by = oplan.base[0][:, 0], oplan.base[0][:, 1]
    cols, rows = bx.max() - bx.min() + 3, by.max() - by.min() + 3
    assert 2 * cols > 256 and 2 * rows <= 256, (rows, cols)
    p = Plan(ant, freqs, 256, 0.5, input="ci4", voltage_scale=lsb, precision=prec)
    img = p.image(torch.from_numpy(b).cuda()).cpu().numpy()
    assert p.sync() == 0
    ref, _ = O.image_interval(oplan, Eint, np.ones((1, 300), complex))
    err = _rel(img, ref)
    print(f"{prec} wide window ({rows} x {cols} cells) image rel-L2 vs FP64 oracle: {err:.3e}")
    assert err <= LP_TOL


def test_tensor_core_many_batches_and_epical():
    """Small scratch budget (several batches, a ragged last one); EPICal's
    pixel stays FP32, so the gains meet the FP32 gain bar."""
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_chan=2, n_time=300)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:80], 300,
                       w["noise_power"], w["rng"])
    b = synth.quantise_ci4(E, w["lsb"])
    Eint = O.unpack_ci4(b) * w["lsb"][None, :, None]
    p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, input="ci4", voltage_scale=w["lsb"],
             precision="fp16", workspace_bytes=40 << 20)
    p.configure((0.0, 0.0), w["model"], w["gamma"])
    img = p.image(torch.from_numpy(b).cuda()).cpu().numpy()
    out = torch.zeros((2, 256), dtype=torch.complex128, device="cuda")
    p.update(out)
    assert p.sync() == 0
    oplan = O.Plan(w["ant_xy"], w["freqs"], 128, 0.5, model_lmS=w["model"])
    g_ref, _, _, ref, _ = O.epical_interval(oplan, Eint, np.ones((2, 256), complex), w["gamma"])
    assert _rel(img, ref) <= LP_TOL
    g = out.cpu().numpy()
    amp = np.max(np.abs(np.abs(g) - np.abs(g_ref)) / np.abs(g_ref))
    ph = np.max(np.abs(np.angle(g * np.conj(g_ref))))
    assert amp <= 1e-4 and ph <= 1e-4, (amp, ph)
