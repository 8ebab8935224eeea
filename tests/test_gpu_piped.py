"""GPU parity of the warp-specialised fused form (producer warps grid and
row-transform frame t + 1 while consumer warps column-transform frame t)
against the FP64 oracle and the two-barrier fused form."""
import numpy as np
import pytest

import epic_synth as synth
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
GAIN_TOL = 1e-4
PIPED, FUSED = 4, 1


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


def _case(n, na, k, n_chan, T, fmt, seed):
    rng = np.random.default_rng(seed)
    diam = {64: 30.0, 128: 70.0}[n]
    ant = synth.layout_disc(na, diam, rng, 0.3)
    freqs = np.linspace(45e6, 62e6, n_chan)
    flags = np.zeros(na, bool)
    flags[rng.choice(na, max(1, na // 12), replace=False)] = True
    gains = synth.true_gains(n_chan, na, rng)
    sky = np.array([[0.1, -0.2, 3.0], [-0.3, 0.3, 1.0], [0.0, 0.0, 4.0]])
    E = synth.voltages(ant, freqs, gains, sky, T, 1.0, rng)
    if fmt == "ci4":
        lsb = np.full(n_chan, 0.6)
        b = synth.quantise_ci4(E, lsb)
        return ant, freqs, flags, rng, torch.from_numpy(b).cuda(), O.unpack_ci4(b) * lsb[None, :, None], \
            dict(input="ci4", voltage_scale=lsb)
    E = E.astype(np.complex64)
    return ant, freqs, flags, rng, torch.from_numpy(E).cuda(), E.astype(np.complex128), dict(input="c64")


def test_path_selection():
    """AUTO keeps the two-barrier form (measured faster); PIPED on request."""
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_chan=2, n_time=8)
    kw = dict(input="ci4", voltage_scale=w["lsb"])
    assert Plan(w["ant_xy"], w["freqs"], 128, 0.5, **kw).info()["path"] == FUSED
    assert Plan(w["ant_xy"], w["freqs"], 128, 0.5, path="fused", **kw).info()["path"] == FUSED
    assert Plan(w["ant_xy"], w["freqs"], 128, 0.5, path="piped", **kw).info()["path"] == PIPED


@pytest.mark.parametrize("n,na,k,n_chan,T,fmt", [
    (128, 256, 3, 3, 37, "ci4"),      # one voltage slot per producer thread pair
    (128, 500, 3, 2, 13, "c64"),      # four slots per producer, two per consumer
    (64, 100, 5, 2, 29, "c64"),       # N = 64, support 5
    (64, 33, 1, 1, 1, "ci4"),         # one frame, nearest-cell gridding
])
def test_piped_image_and_epical_match_oracle(n, na, k, n_chan, T, fmt):
    from paper_1603_02126_gb300 import Plan
    ant, freqs, flags, rng, d, Eref, kw = _case(n, na, k, n_chan, T, fmt, seed=n + na + T)
    model = np.array([[0.0, 0.0, 4.0], [0.1, -0.2, 3.0]])
    p = Plan(ant, freqs, n, 0.5, support=k, param=0.6, flags=flags, path="piped", **kw)
    gcur = synth.true_gains(n_chan, na, rng)
    p.configure((0.0, 0.0), model, 0.5, g0=gcur)
    img = p.image(d).cpu().numpy()
    out = torch.zeros((n_chan, na), dtype=torch.complex128, device="cuda")
    p.update(out)
    assert p.sync() == 0
    oplan = O.Plan(ant, freqs, n, 0.5, support=k, param=0.6, flags=flags, model_lmS=model)
    ref, _ = O.image_interval(oplan, Eref, gcur)
    assert _rel(img, ref) <= IMG_TOL
    g_ref, *_ = O.epical_interval(oplan, Eref, gcur, 0.5, with_image=False)
    g = out.cpu().numpy()
    live = ~flags
    amp, ph = _gain_err(g[:, live], g_ref[:, live])
    assert amp <= GAIN_TOL and ph <= GAIN_TOL, (amp, ph)


def test_piped_equals_two_barrier_form_many_units():
    """LWA-like array, 4 channels, 700 samples: many work units per CTA and
    both forms agree to FP32 rounding (image and EPICal gains)."""
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_chan=4, n_time=700)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:60], 700, w["noise_power"],
                       w["rng"])
    d = torch.from_numpy(synth.quantise_ci4(E, w["lsb"])).cuda()
    res = []
    for path in ("piped", "fused"):
        p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, input="ci4", voltage_scale=w["lsb"], path=path)
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        img = p.image(d)
        out = torch.zeros((4, 256), dtype=torch.complex128, device="cuda")
        p.update(out)
        assert p.sync() == 0
        res.append((img.cpu().numpy(), out.cpu().numpy()))
    assert _rel(res[0][0], res[1][0]) <= 1e-6
    assert np.max(np.abs(res[0][1] - res[1][1]) / np.abs(res[1][1])) <= 1e-5


def test_piped_graph_replay_matches_direct_calls():
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_chan=2, n_time=64)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:40], 64, w["noise_power"],
                       w["rng"])
    d = torch.from_numpy(synth.quantise_ci4(E, w["lsb"])).cuda()
    stream = torch.cuda.Stream()
    res = []
    for use_graph in (False, True):
        p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, input="ci4", voltage_scale=w["lsb"],
                 path="piped", stream=stream.cuda_stream)
        assert p.info()["path"] == PIPED
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        img = torch.empty((2, 128, 128), dtype=torch.float64, device="cuda")
        gout = torch.empty((2, 256), dtype=torch.complex128, device="cuda")
        with torch.cuda.stream(stream):
            if use_graph:
                p.graph_capture(d, img, gout)
                for _ in range(4):
                    p.graph_launch()
            else:
                for _ in range(4):
                    p.image(d, img)
                    p.update(gout)
        stream.synchronize()
        assert p.sync() == 0
        res.append((img.cpu().numpy(), gout.cpu().numpy()))
    assert _rel(res[1][0], res[0][0]) <= 1e-6
    assert np.max(np.abs(res[1][1] - res[0][1]) / np.abs(res[0][1])) <= 1e-5


def test_piped_bounded_wait_timeout_is_reported_and_recoverable():
    """Failure detection without a fault: with one poll per bounded wait the
    consumer warps give up waiting for the producers' first frame, the kernel
    raises the plan's error flag, stops waiting and runs to its end, and
    epic_plan_sync reports EPIC_ERR_TIMEOUT.  The context stays usable: with
    the default limit restored the same plan images correctly again."""
    from paper_1603_02126_gb300 import EpicError, Plan
    w = synth.workload("lwa", n_time=64, n_chan=2)
    rng = np.random.default_rng(12)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:40], 64, w["noise_power"], rng)
    b = torch.from_numpy(synth.quantise_ci4(E, w["lsb"])).cuda()
    kw = dict(support=3, param=0.5, input="ci4", voltage_scale=w["lsb"])
    p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, path="piped", **kw)
    assert p.info()["path"] == PIPED
    p.set_wait_limit(1)
    p.image(b)
    with pytest.raises(EpicError) as ei:
        p.sync()
    assert ei.value.status == 6                       # EPIC_ERR_TIMEOUT
    p.set_wait_limit(0)
    img = p.image(b).cpu().numpy()
    assert p.sync() == 0
    ref = Plan(w["ant_xy"], w["freqs"], 128, 0.5, path="fused", **kw).image(b).cpu().numpy()
    assert _rel(img, ref) <= IMG_TOL
