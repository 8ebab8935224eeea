"""GPU parity of the plain unfused FP32 path (grid and row spectra through
device memory) against the FP64 oracle, N = 32..512."""
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


@pytest.mark.parametrize("n,na,T,C,diam", [(32, 30, 21, 2, 14.0), (64, 90, 13, 2, 30.0),
                                           (128, 256, 9, 3, 70.0), (256, 400, 4, 1, 150.0),
                                           (512, 700, 2, 1, 300.0)])
def test_unfused_image_matches_oracle(n, na, T, C, diam):
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(n)
    ant = synth.layout_disc(na, diam, rng, 0.5)
    freqs = np.linspace(45e6, 62e6, C)
    flags = np.zeros(na, bool)
    flags[rng.choice(na, 3, replace=False)] = True
    gains = synth.true_gains(C, na, rng)
    sky = np.array([[0.1, -0.2, 3.0], [-0.3, 0.3, 1.0], [0.0, 0.0, 5.0]])
    E = synth.voltages(ant, freqs, gains, sky, T, 1.0, rng)
    lsb = np.full(C, 0.6)
    b = synth.quantise_ci4(E, lsb)
    Eint = O.unpack_ci4(b) * lsb[None, :, None]
    p = Plan(ant, freqs, n, 0.5, support=3, param=0.5, input="ci4", voltage_scale=lsb,
             flags=flags, path="unfused")
    assert p.info()["path"] == 2
    gcur = synth.true_gains(C, na, rng)
    p.set_gains(gcur)
    img = p.image(torch.from_numpy(b).cuda()).cpu().numpy()
    oplan = O.Plan(ant, freqs, n, 0.5, flags=flags)
    ref, _ = O.image_interval(oplan, Eint, gcur, block=4)
    assert _rel(img, ref) <= IMG_TOL


def test_unfused_equals_fused_many_batches():
    """Small scratch budget: the interval runs as many batches; the plain
    path and the fused kernel agree to FP32 rounding."""
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_chan=8, n_time=200)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:80], 200,
                       w["noise_power"], w["rng"])
    b = torch.from_numpy(synth.quantise_ci4(E, w["lsb"])).cuda()
    kw = dict(support=3, param=0.5, input="ci4", voltage_scale=w["lsb"])
    pf = Plan(w["ant_xy"], w["freqs"], 128, 0.5, path="fused", **kw)
    pu = Plan(w["ant_xy"], w["freqs"], 128, 0.5, path="unfused", workspace_bytes=64 << 20, **kw)
    a = pf.image(b).cpu().numpy()
    u = pu.image(b).cpu().numpy()
    assert 1 < pu.info()["batch_time"] < 200
    assert _rel(u, a) <= 1e-6


def test_unfused_epical_interval_matches_oracle():
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_chan=2, n_time=96)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:80], 96,
                       w["noise_power"], w["rng"])
    b = synth.quantise_ci4(E, w["lsb"])
    Eint = O.unpack_ci4(b) * w["lsb"][None, :, None]
    p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
             voltage_scale=w["lsb"], path="unfused", workspace_bytes=16 << 20)
    p.configure((0.0, 0.0), w["model"], w["gamma"])
    p.image(torch.from_numpy(b).cuda())
    out = torch.zeros((2, 256), dtype=torch.complex128, device="cuda")
    p.update(out)
    assert p.sync() == 0
    oplan = O.Plan(w["ant_xy"], w["freqs"], 128, 0.5, model_lmS=w["model"])
    g_ref, *_ = O.epical_interval(oplan, Eint, np.ones((2, 256), complex), w["gamma"],
                                  with_image=False)
    g = out.cpu().numpy()
    amp = np.max(np.abs(np.abs(g) - np.abs(g_ref)) / np.abs(g_ref))
    ph = np.max(np.abs(np.angle(g * np.conj(g_ref))))
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)
