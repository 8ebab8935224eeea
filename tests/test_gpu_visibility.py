"""Visibility-based comparison path (Sec. 4 noise trends, Eq. 21) on the
GPU: the X-engine against the oracle's visibilities (integer-exact for 4-bit
input) and the StEFCal solve against the oracle's solve of the oracle's own
visibilities of the same bytes."""
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


@pytest.mark.parametrize("na,T", [(5, 7), (70, 100), (256, 40000)])
def test_xengine_ci4_integer_exact(na, T):
    """4-bit voltages: V T / s^2 are integers and equal the oracle's sums
    exactly (one and two FP32 segments; tiles with ragged edges)."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(na)
    ant = synth.layout_disc(na, 30.0, rng, 0.2)
    freqs = [45e6, 70e6]
    b = rng.integers(0, 256, size=(T, 2, na), dtype=np.uint8)
    lsb = np.array([0.5, 0.25], np.float32)
    p = Plan(ant, freqs, 64, 0.5, input="ci4", voltage_scale=lsb)
    V = p.visibilities(torch.from_numpy(b).cuda()).cpu().numpy()
    for c in range(2):
        E = O.unpack_ci4(b[:, c, :])
        ref = E.T @ np.conj(E)                    # integer sums
        got = V[c] * T / float(lsb[c]) ** 2
        assert np.array_equal(np.rint(got.real), ref.real) and np.array_equal(np.rint(got.imag), ref.imag)
        assert np.max(np.abs(got - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)))


def test_xengine_c64_and_accumulate():
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(11)
    na, T = 45, 333
    ant = synth.layout_disc(na, 20.0, rng, 0.5)
    E = (rng.normal(size=(T, 1, na)) + 1j * rng.normal(size=(T, 1, na))).astype(np.complex64)
    p = Plan(ant, [50e6], 32, 0.5, input="c64")
    d = torch.from_numpy(E).cuda()
    V = p.visibilities(d)
    ref = O.visibilities(E[:, 0, :].astype(np.complex128))
    rel = np.linalg.norm(V.cpu().numpy()[0] - ref) / np.linalg.norm(ref)
    assert rel < 1e-6
    V2 = p.visibilities(d, V.clone(), accumulate=True).cpu().numpy()
    assert np.allclose(V2[0], 2 * V.cpu().numpy()[0], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("cut", [0.0, 0.7])
def test_stefcal_matches_oracle(cut):
    """Noisy data, 50-source sky, full model: the GPU solve of the GPU
    visibilities equals the oracle's solve of its own visibilities of the
    same bytes (start g = 1, same iteration), flagged antenna held."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(17)
    na, T = 24, 800
    ant = synth.layout_disc(na, 12.0, rng, 1.0)
    freqs = [48e6, 62e6]
    flags = np.zeros(na, bool)
    flags[5] = True
    faint = np.column_stack([synth.random_directions(10, rng, 0.5), rng.uniform(0.2, 0.5, 10)])
    sky = np.vstack([[0.0, 0.0, 5.0], faint])
    g = synth.true_gains(2, na, rng)
    E = synth.voltages(ant, freqs, g, sky, T, 10.0, rng).astype(np.complex64)
    p = Plan(ant, freqs, 32, 0.5, input="c64", flags=flags)
    p.configure((0.0, 0.0), sky, 0.35)
    Vo = np.stack([O.visibilities(E[:, c, :].astype(np.complex128)) for c in range(2)])
    # the whole GPU chain (FP32 X-engine sums of complex64 input, FP64 solve)
    V = p.visibilities(torch.from_numpy(E).cuda())
    gd = torch.ones((2, na), dtype=torch.complex128, device="cuda")
    p.visibility_solve(V, gd, max_iter=3000, tol=1e-12, min_baseline=cut)
    gd = gd.cpu().numpy()
    # the GPU solver alone, on the oracle's visibilities
    gs = torch.ones((2, na), dtype=torch.complex128, device="cuda")
    iters = p.visibility_solve(torch.from_numpy(Vo).cuda(), gs, max_iter=3000, tol=1e-12, min_baseline=cut)
    gs = gs.cpu().numpy()
    for c, f in enumerate(freqs):
        VM = O.model_visibilities(ant, f, sky)
        mask = O.baseline_mask(O.antenna_uv(ant, f), cut)
        go, it = O.visibility_solve(Vo[c], VM, np.ones(na, complex), flags=flags, pair_mask=mask,
                                    return_iters=True)
        # FP32 pair products: the GPU stops at a relative change of 1e-6
        assert 1 <= int(iters[c]) <= it, (iters[c], it)
        assert np.max(np.abs(gs[c] - go) / np.abs(go)) < 1e-5
        assert np.max(np.abs(gd[c] - go) / np.abs(go)) < 1e-5
        assert gd[c, 5] == 1.0 and gs[c, 5] == 1.0


def test_stefcal_noise_free_truth_on_gpu():
    """Orthogonal tone signals, no noise: the solve returns the injected gains
    up to one global phase."""
    from paper_1603_02126_gb300 import Plan
    rng = np.random.default_rng(23)
    na = 40
    ant = synth.layout_disc(na, 20.0, rng, 1.0)
    sky = np.array([[0.0, 0.0, 4.0], [0.3, -0.2, 1.0], [-0.1, 0.35, 2.0]])
    g = synth.true_gains(1, na, rng)
    E = synth.voltages(ant, [55e6], g, sky, 128, 0.0, rng, tones=True).astype(np.complex64)
    p = Plan(ant, [55e6], 64, 0.5, input="c64")
    p.configure((0.0, 0.0), sky, 0.35)
    V = p.visibilities(torch.from_numpy(E).cuda())
    gd = torch.ones((1, na), dtype=torch.complex128, device="cuda")
    p.visibility_solve(V, gd)
    ga = O.align_phase(gd.cpu().numpy()[0], g[0])
    assert np.max(np.abs(ga - g[0]) / np.abs(g[0])) < 1e-5
