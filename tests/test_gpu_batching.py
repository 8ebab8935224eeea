"""Batching form on the GPU: the autotuner keeps results unchanged and the
captured CUDA graph of a calibration interval replays the same EPICal
loop as individual calls."""
import numpy as np
import pytest

import epic_synth as synth
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("path", ["fused", "unfused"])
def test_autotune_keeps_parity(path):
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_chan=4, n_time=150)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:80], 150,
                       w["noise_power"], w["rng"])
    b = synth.quantise_ci4(E, w["lsb"])
    Eint = O.unpack_ci4(b) * w["lsb"][None, :, None]
    p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
             voltage_scale=w["lsb"], path=path, workspace_bytes=64 << 20)
    d = torch.from_numpy(b).cuda()
    r = p.autotune(d)
    assert r["candidates"] >= 6 and r["ms_best"] <= r["ms_default"] * 1.0001
    img = p.image(d).cpu().numpy()
    ref, _ = O.image_interval(O.Plan(w["ant_xy"], w["freqs"], 128, 0.5), Eint, np.ones((4, 256)))
    assert _rel(img, ref) <= 1e-5


@pytest.mark.parametrize("n,path", [(32, "fused"), (256, "unfused")])
def test_graph_replay_matches_calls(n, path):
    """Eight EPICal loops on the same interval data, once through
    individual calls and once as replays of the captured interval."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(n)
    na = 24 if n == 32 else 200
    ant = synth.layout_disc(na, 14.0 if n == 32 else 120.0, rng, 0.8)
    freqs = [50e6, 58e6]
    g_true = synth.true_gains(2, na, rng)
    sky = np.array([[0.0, 0.0, 5.0], [0.3, 0.1, 1.0]])
    E = synth.voltages(ant, freqs, g_true, sky, 40, 0.5, rng).astype(np.complex64)
    d = torch.from_numpy(E).cuda()
    stream = torch.cuda.Stream()
    res = []
    for use_graph in (False, True):
        p = Plan(ant, freqs, n, 0.5, input="c64", path=path, stream=stream.cuda_stream)
        p.configure((0.0, 0.0), sky, 0.5)
        img = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
        gout = torch.empty((2, na), dtype=torch.complex128, device="cuda")
        with torch.cuda.stream(stream):
            if use_graph:
                p.graph_capture(d, img, gout)
                for _ in range(8):
                    p.graph_launch()
            else:
                for _ in range(8):
                    p.image(d, img)
                    p.update(gout)
        stream.synchronize()
        res.append((img.cpu().numpy(), gout.cpu().numpy(), p.info()["iteration"]))
    (i0, g0, it0), (i1, g1, it1) = res
    assert it0 == it1 == 8
    assert _rel(i1, i0) <= 1e-6
    assert np.max(np.abs(g1 - g0) / np.abs(g0)) <= 1e-5
