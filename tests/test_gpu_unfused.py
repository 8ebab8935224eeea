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


@pytest.mark.parametrize("n,na,diam,C,T", [(256, 300, 150.0, 2, 9), (512, 600, 300.0, 2, 7)])
def test_persistent_launch_matches_oracle_and_batched(n, na, diam, C, T):
    """One persistent cooperative launch per call (row phase, grid barrier,
    column phase, grid barrier, correlation, for every batch): image and an
    EPICal interval against the oracle and against the batched launches,
    with a scratch small enough for several batches per call; then the same
    interval captured in a CUDA graph and replayed."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(700 + n)
    ant = synth.layout_disc(na, diam, rng, 0.5)
    freqs = np.linspace(45e6, 62e6, C)
    flags = np.zeros(na, bool)
    flags[[5, 77]] = True
    sky = np.array([[0.0, 0.0, 5.0], [0.1, -0.2, 3.0], [-0.3, 0.3, 1.0]])
    E = synth.voltages(ant, freqs, synth.true_gains(C, na, rng), sky, T, 1.0, rng)
    lsb = np.full(C, 0.6)
    b = synth.quantise_ci4(E, lsb)
    Eint = O.unpack_ci4(b) * lsb[None, :, None]
    d = torch.from_numpy(b).cuda()
    ws = 3 * C * n * (n // 2 + 8) * 8                    # about 3 samples per batch
    kw = dict(support=3, param=0.5, input="ci4", voltage_scale=lsb, flags=flags, path="unfused",
              workspace_bytes=ws)
    outs = []
    for pers in (True, False):
        p = Plan(ant, freqs, n, 0.5, batch_persistent=pers, **kw)
        p.configure((0.0, 0.0), sky, 0.5)
        img = p.image(d).cpu().numpy()
        g = torch.zeros((C, na), dtype=torch.complex128, device="cuda")
        p.update(g)
        assert p.sync() == 0
        assert p.info()["batch_time"] < T                 # several batches per call
        outs.append((img, g.cpu().numpy(), p))
    oplan = O.Plan(ant, freqs, n, 0.5, flags=flags, model_lmS=sky)
    ref, _ = O.image_interval(oplan, Eint, np.ones((C, na), complex), block=4)
    assert _rel(outs[0][0], ref) <= IMG_TOL
    assert _rel(outs[0][0], outs[1][0]) <= 1e-6
    g_ref, *_ = O.epical_interval(oplan, Eint, np.ones((C, na), complex), 0.5, with_image=False)
    ok = ~flags
    amp = np.max(np.abs(np.abs(outs[0][1][:, ok]) - np.abs(g_ref[:, ok])) / np.abs(g_ref[:, ok]))
    ph = np.max(np.abs(np.angle(outs[0][1][:, ok] * np.conj(g_ref[:, ok]))))
    assert amp <= 1e-4 and ph <= 1e-4, (amp, ph)
    # the persistent interval inside a CUDA graph
    p = outs[0][2]
    stream = torch.cuda.Stream()
    p.set_stream(stream.cuda_stream)
    img_g = torch.empty((C, n, n), dtype=torch.float64, device="cuda")
    p.graph_capture(d, img_g)
    p.graph_launch()
    torch.cuda.synchronize()
    # the replay images with the gains of the first update
    ref1, _ = O.image_interval(oplan, Eint, outs[0][1], block=4)
    assert _rel(img_g.cpu().numpy(), ref1) <= IMG_TOL


def test_persistent_grid_barrier_timeout_is_reported_and_recoverable():
    """Failure detection without a fault: with one poll per grid-barrier
    wait the persistent kernel's early arrivers give up before the last CTA
    arrives, raise the abort word and the plan's error flag, and every CTA
    returns at its next barrier; epic_plan_sync reports EPIC_ERR_TIMEOUT.
    With the default limit restored the same plan images correctly again."""
    from paper_1603_02126_gb300 import EpicError, Plan
    n, na, C, T = 256, 300, 2, 9
    rng = np.random.default_rng(811)
    ant = synth.layout_disc(na, 150.0, rng, 0.5)
    freqs = np.linspace(45e6, 62e6, C)
    sky = np.array([[0.0, 0.0, 5.0], [0.1, -0.2, 3.0]])
    E = synth.voltages(ant, freqs, synth.true_gains(C, na, rng), sky, T, 1.0, rng)
    lsb = np.full(C, 0.6)
    b = synth.quantise_ci4(E, lsb)
    d = torch.from_numpy(b).cuda()
    kw = dict(support=3, param=0.5, input="ci4", voltage_scale=lsb, path="unfused",
              workspace_bytes=3 * C * n * (n // 2 + 8) * 8)
    p = Plan(ant, freqs, n, 0.5, batch_persistent=True, **kw)
    p.set_wait_limit(1)
    p.image(d)
    with pytest.raises(EpicError) as ei:
        p.sync()
    assert ei.value.status == 6                       # EPIC_ERR_TIMEOUT
    p.set_wait_limit(0)
    img = p.image(d).cpu().numpy()
    assert p.sync() == 0
    ref = Plan(ant, freqs, n, 0.5, **kw).image(d).cpu().numpy()
    assert _rel(img, ref) <= 1e-6
