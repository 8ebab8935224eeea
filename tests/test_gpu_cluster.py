"""GPU parity of the thread-block-cluster path (N = 256 with 8 CTAs per
cluster, N = 512 with 16; row spectra exchanged through distributed shared
memory) against the FP64 oracle and the plain unfused path."""
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


@pytest.mark.parametrize("n,na,T,C,diam", [(256, 300, 7, 2, 150.0), (512, 700, 3, 1, 300.0)])
def test_cluster_image_matches_oracle(n, na, T, C, diam):
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(n + 7)
    ant = synth.layout_disc(na, diam, rng, 0.5)
    freqs = np.linspace(45e6, 62e6, C)
    flags = np.zeros(na, bool)
    flags[rng.choice(na, 4, replace=False)] = True
    gains = synth.true_gains(C, na, rng)
    sky = np.array([[0.1, -0.2, 3.0], [-0.3, 0.3, 1.0], [0.0, 0.0, 5.0]])
    E = synth.voltages(ant, freqs, gains, sky, T, 1.0, rng)
    lsb = np.full(C, 0.6)
    b = synth.quantise_ci4(E, lsb)
    Eint = O.unpack_ci4(b) * lsb[None, :, None]
    p = Plan(ant, freqs, n, 0.5, input="ci4", voltage_scale=lsb, flags=flags, path="cluster")
    assert p.info()["path"] == 3
    gcur = synth.true_gains(C, na, rng)
    p.set_gains(gcur)
    img = p.image(torch.from_numpy(b).cuda()).cpu().numpy()
    ref, _ = O.image_interval(O.Plan(ant, freqs, n, 0.5, flags=flags), Eint, gcur, block=4)
    assert _rel(img, ref) <= IMG_TOL


@pytest.mark.parametrize("name,n_chan,T", [("compact1024", 4, 40), ("hex2048", 3, 20)])
def test_cluster_equals_unfused(name, n_chan, T):
    """The config-2 and config-3 arrays: cluster and plain paths agree to
    FP32 rounding, with many work units per cluster."""
    from paper_1603_02126_gb300 import Plan
    w = synth.workload(name, n_chan=n_chan, n_time=T)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:60], T, w["noise_power"],
                       w["rng"])
    if w["input"] == "ci4":
        d = torch.from_numpy(synth.quantise_ci4(E, w["lsb"])).cuda()
        kw = dict(input="ci4", voltage_scale=w["lsb"])
    else:
        d = torch.from_numpy(E.astype(np.complex64)).cuda()
        kw = dict(input="c64")
    n = w["grid_n"]
    pc = Plan(w["ant_xy"], w["freqs"], n, 0.5, path="cluster", **kw)
    pu = Plan(w["ant_xy"], w["freqs"], n, 0.5, path="unfused", workspace_bytes=1 << 30, **kw)
    a = pc.image(d).cpu().numpy()
    u = pu.image(d).cpu().numpy()
    assert _rel(a, u) <= 1e-6


def test_cluster_epical_interval_matches_oracle():
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("compact1024", n_chan=2, n_time=48, n_ant=400)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:60], 48, w["noise_power"],
                       w["rng"])
    b = synth.quantise_ci4(E, w["lsb"])
    Eint = O.unpack_ci4(b) * w["lsb"][None, :, None]
    p = Plan(w["ant_xy"], w["freqs"], 256, 0.5, input="ci4", voltage_scale=w["lsb"], path="cluster")
    p.configure((0.0, 0.0), w["model"], w["gamma"])
    p.image(torch.from_numpy(b).cuda())
    out = torch.zeros((2, 400), dtype=torch.complex128, device="cuda")
    p.update(out)
    assert p.sync() == 0
    oplan = O.Plan(w["ant_xy"], w["freqs"], 256, 0.5, model_lmS=w["model"])
    g_ref, *_ = O.epical_interval(oplan, Eint, np.ones((2, 400), complex), w["gamma"],
                                  with_image=False)
    g = out.cpu().numpy()
    amp = np.max(np.abs(np.abs(g) - np.abs(g_ref)) / np.abs(g_ref))
    ph = np.max(np.abs(np.angle(g * np.conj(g_ref))))
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)


def test_cluster_graph_replay():
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(5)
    ant = synth.layout_disc(200, 120.0, rng, 0.8)
    freqs = [50e6, 58e6]
    sky = np.array([[0.0, 0.0, 5.0], [0.3, 0.1, 1.0]])
    E = synth.voltages(ant, freqs, synth.true_gains(2, 200, rng), sky, 30, 0.5, rng)
    d = torch.from_numpy(E.astype(np.complex64)).cuda()
    stream = torch.cuda.Stream()
    res = []
    for use_graph in (False, True):
        p = Plan(ant, freqs, 256, 0.5, input="c64", path="cluster", stream=stream.cuda_stream)
        p.configure((0.0, 0.0), sky, 0.5)
        img = torch.empty((2, 256, 256), dtype=torch.float64, device="cuda")
        gout = torch.empty((2, 200), dtype=torch.complex128, device="cuda")
        with torch.cuda.stream(stream):
            if use_graph:
                p.graph_capture(d, img, gout)
                for _ in range(5):
                    p.graph_launch()
            else:
                for _ in range(5):
                    p.image(d, img)
                    p.update(gout)
        stream.synchronize()
        res.append((img.cpu().numpy(), gout.cpu().numpy()))
    assert _rel(res[1][0], res[0][0]) <= 1e-6
    assert np.max(np.abs(res[1][1] - res[0][1]) / np.abs(res[0][1])) <= 1e-5
