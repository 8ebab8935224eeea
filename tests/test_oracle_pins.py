"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: a
closed form, an identity the paper derives, an exhaustive enumeration, a
library routine in a special case or a brute-force sum.  No GPU needed.
"""
import json
import os

import numpy as np
import pytest

import epic_synth as synth
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# unpack (4-bit complex input format)
# --------------------------------------------------------------------------
def test_unpack_exhaustive_roundtrip():
    """All 256 bytes: unpack is the inverse of the generator's packing, a
    bijection onto [-8, 7]^2."""
    re, im = np.meshgrid(np.arange(-8, 8), np.arange(-8, 8), indexing="ij")
    b = synth.pack_ci4(re.ravel(), im.ravel())
    assert sorted(b.tolist()) == list(range(256))
    z = O.unpack_ci4(b)
    assert np.array_equal(z.real, re.ravel()) and np.array_equal(z.imag, im.ravel())


def test_unpack_golden_bytes():
    """Hand-decoded bytes (two's complement nibbles)."""
    with open(os.path.join(GOLDEN, "ci4_bytes.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        z = O.unpack_ci4(np.array([c["byte"]], np.uint8))[0]
        assert (z.real, z.imag) == (c["re"], c["im"]), c


# --------------------------------------------------------------------------
# grid table (Eq. 9 stencil and kernel)
# --------------------------------------------------------------------------
def test_grid_table_cell_centre_special_case():
    """An antenna exactly on a cell centre: base = that cell, and the 3x3
    Gaussian weights are the normalised products of 1 and e^{-1/(2 s^2)}."""
    f = 50e6
    lam = O.C_LIGHT / f
    N, du = 16, 0.5
    # x = 3 cells east, y = 2 cells south of the centre
    ant = np.array([[3 * du * lam, -2 * du * lam]])
    base, W = O.grid_table(ant, [f], N, du, "gaussian", 3, 0.5)
    assert tuple(base[0, 0]) == (N // 2 + 3, N // 2 - 2)
    e = np.exp(-1.0 / (2 * 0.25))
    w1 = np.array([e, 1.0, e])
    expect = np.outer(w1, w1) / np.outer(w1, w1).sum()
    assert np.allclose(W[0, 0], expect, rtol=0, atol=1e-12)


def test_grid_table_properties_random():
    rng = np.random.default_rng(3)
    ant = rng.uniform(-10, 10, size=(40, 2))
    freqs = [40e6, 63e6, 80e6]
    N, du = 64, 0.5
    base, W = O.grid_table(ant, freqs, N, du, "gaussian", 5, 0.7)
    for c, f in enumerate(freqs):
        p = ant * f / O.C_LIGHT / du + N / 2
        # nearest cell
        assert np.all(np.abs(base[c] - p) <= 0.5)
        # normalised: far-field pattern is 1 at the centre
        assert np.allclose(W[c].sum(axis=(1, 2)), 1.0, atol=1e-14)
        # largest tap is the centre tap (nearest cell)
        assert np.all(W[c].reshape(len(ant), -1).argmax(axis=1) == 12)
    # mirroring the array in x mirrors the weights in dx
    base2, W2 = O.grid_table(ant * np.array([-1, 1]), freqs, N, du, "gaussian", 5, 0.7)
    for c, f in enumerate(freqs):
        # away from exact half-cell ties, where the nearest cell flips side
        ok = np.abs((ant[:, 0] * f / O.C_LIGHT / du) % 1 - 0.5) > 1e-9
        assert np.allclose(W2[c, ok], W[c, ok][..., ::-1], atol=1e-13)


def test_grid_table_tophat_counts():
    """Tophat of side s metres covers the cells whose centres lie within
    s/2 of the antenna on both axes; weights are 1/count."""
    f = 60e6
    lam = O.C_LIGHT / f
    du = 0.5
    ant = np.array([[0.0, 0.0], [0.3 * du * lam, 0.05 * du * lam]])
    # side 2.2 cells: half 1.1 cells -> 3 x 3 cells around a centred antenna
    base, W = O.grid_table(ant, [f], 32, du, "tophat", 5, 2.2 * du * lam)
    assert np.count_nonzero(W[0, 0]) == 9 and np.allclose(W[0, 0][W[0, 0] > 0], 1 / 9)
    # offset antenna: x in [-0.8, 1.4] cells -> cells 0, 1; y in [-1.05, 1.15] -> -1, 0, 1
    assert np.count_nonzero(W[0, 1]) == 6 and np.allclose(W[0, 1][W[0, 1] > 0], 1 / 6)


def test_grid_table_overflow():
    f = 80e6
    lam = O.C_LIGHT / f
    ant = np.array([[7.6 * 0.5 * lam, 0.0]])  # cell 16+8 = 23.6 -> 24 -> taps 23..25
    with pytest.raises(O.GridTooSmall):
        O.grid_table(ant, [f], 16, 0.5)
    # flagged antennas are not checked
    O.grid_table(ant, [f], 16, 0.5, flags=[1])


# --------------------------------------------------------------------------
# E-field image (Eq. 10)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 8, 16])
def test_dft_separable_equals_direct(n):
    rng = np.random.default_rng(n)
    G = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    a = O.efield_image(G, 7)
    b = O.efield_image_direct(G, 7)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("n", [8, 32, 128])
def test_dft_equals_numpy_ifft(n):
    """Library special case: with sign flips (-1)^(jx+jy) on the grid and
    (-1)^(kx+ky) on the image, Eq. 10 is N^2 ifft2 / Na."""
    rng = np.random.default_rng(n + 1)
    G = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    s = (-1.0) ** np.add.outer(np.arange(n), np.arange(n))
    ref = s * np.fft.ifft2(s * G) * n * n / 5.0
    got = O.efield_image(G, 5)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_dft_single_cell_phase_ramp():
    """One non-zero cell gives a pure phase ramp of unit modulus / Na."""
    n = 16
    G = np.zeros((n, n), complex)
    jx, jy = 11, 3
    G[jy, jx] = 1.0
    img = O.efield_image(G, 4)
    assert np.allclose(np.abs(img), 0.25, atol=1e-14)
    # phase at (kx, ky) = (N/2 + 1, N/2): 2 pi (jx - N/2) / N
    assert np.isclose(np.angle(img[n // 2, n // 2 + 1]),
                      np.angle(np.exp(2j * np.pi * (jx - n // 2) / n)), atol=1e-12)
    assert np.isclose(img[n // 2, n // 2], 0.25, atol=1e-15)


def test_point_source_images_at_its_direction():
    """Sign convention: a noise-free point source at pixel (kx, ky) gives the
    brightest dirty-image pixel there (Eq. 3 propagation, Eq. 10 imaging)."""
    rng = np.random.default_rng(5)
    N, du, f = 32, 0.5, 50e6
    ant = synth.layout_disc(24, 20.0, rng, 1.0)
    kx, ky = 21, 12
    l, m = (kx - N / 2) / (N * du), (ky - N / 2) / (N * du)
    sky = np.array([[l, m, 1.0]])
    E = synth.voltages(ant, [f], np.ones((1, 24)), sky, 64, 0.0, rng)
    plan = O.Plan(ant, [f], N, du)
    img, _ = O.image_interval(plan, E, np.ones((1, 24)))
    assert np.unravel_index(np.argmax(img[0]), img[0].shape) == (ky, kx)
    assert O.calibrator_pixel(l, m, N, du) == (kx, ky)


def _explicit_A(plan, c):
    """A_{k,a} for every pixel k by explicit sums over taps (test-local)."""
    N = plan.N
    Na = plan.Na
    K = plan.W.shape[-1]
    h = (K - 1) // 2
    A = np.zeros((N, N, Na), complex)
    ky, kx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    for a in range(Na):
        if plan.flags[a]:
            continue
        for dy in range(K):
            for dx in range(K):
                jx = plan.base[c, a, 0] + dx - h
                jy = plan.base[c, a, 1] + dy - h
                ph = 2 * np.pi * ((jx - N // 2) * (kx - N // 2) + (jy - N // 2) * (ky - N // 2)) / N
                A[:, :, a] += plan.W[c, a, dy, dx] * np.exp(1j * ph)
    return A / plan.norm


def test_image_equals_gridded_visibilities_with_autos():
    """Sec. 2.1: the squared, averaged E-field image equals the image made
    from all antenna-pair visibilities, autos included:
    I_k = sum_{a,b} A_{k,a} conj(A_{k,b}) V'_ab, V'_ab = <E'_a conj(E'_b)>."""
    rng = np.random.default_rng(11)
    Na, N, T = 6, 16, 48
    ant = synth.layout_disc(Na, 8.0, rng, 1.0)
    f = [45e6, 70e6]
    g = synth.true_gains(2, Na, rng)
    sky = np.array([[0.0, 0.0, 3.0], [0.3, -0.2, 1.0]])
    E = synth.voltages(ant, f, g, sky, T, 1.0, rng)
    flags = np.zeros(Na, bool)
    flags[4] = True
    plan = O.Plan(ant, f, N, 0.5, flags=flags)
    gcur = synth.true_gains(2, Na, rng)
    img, _ = O.image_interval(plan, E, gcur, block=17)
    for c in range(2):
        A = _explicit_A(plan, c)
        Ec = E[:, c, :] / gcur[c]
        V = Ec.T @ np.conj(Ec) / T
        ref = np.einsum("yxa,ab,yxb->yx", A, V, np.conj(A)).real
        assert np.max(np.abs(img[c] - ref)) <= 1e-12 * np.max(ref)


def _offcentre_case(rng, Na=7, N=16, T=45, K=5):
    """Small off-centre case with a flagged antenna, support K and a calibrator
    away from the phase centre (shared by the sampled-checker pins)."""
    ant = synth.layout_disc(Na, 6.0, rng, 1.0)
    f = [47e6, 66e6]
    g = synth.true_gains(2, Na, rng)
    sky = np.array([[0.19, -0.31, 3.0], [-0.27, 0.12, 1.5]])
    E = synth.voltages(ant, f, g, sky, T, 1.0, rng)
    flags = np.zeros(Na, bool)
    flags[3] = True
    cal = (0.25, -0.375)                      # pixel (12, 5) at N = 16, du = 0.5
    plan = O.Plan(ant, f, N, 0.5, support=K, param=0.8, flags=flags, cal_lm=cal,
                  model_lmS=sky)
    return plan, E, synth.true_gains(2, Na, rng)


def test_image_pixels_equal_visibility_route_every_pixel():
    """image_pixels, the checker of every full-size image test, at all N^2
    pixels of a small case (two channels, flags, K = 5, T not a multiple of
    the block) equals the Sec. 2.1 statement I_k = sum_ab A_ka conj(A_kb) V'_ab
    with explicit A, and the full-transform image_interval.  A swapped axis
    or a wrong centring offset in its single-pixel DFT fails here."""
    rng = np.random.default_rng(31)
    plan, E, gcur = _offcentre_case(rng)
    N = plan.N
    T = E.shape[0]
    pix = [(kx, ky) for ky in range(N) for kx in range(N)]
    full, _ = O.image_interval(plan, E, gcur)
    for c in range(2):
        got = O.image_pixels(plan, E, gcur, c, pix, block=16).reshape(N, N)
        A = _explicit_A(plan, c)
        Ec = E[:, c, :] / gcur[c]
        V = Ec.T @ np.conj(Ec) / T
        ref = np.einsum("yxa,ab,yxb->yx", A, V, np.conj(A)).real
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(ref)
        assert np.max(np.abs(got - full[c])) <= 1e-12 * np.max(full[c])
    # a non-square pixel list keeps (kx, ky) order: (kx, ky) != (ky, kx)
    got = O.image_pixels(plan, E, gcur, 1, [(3, 11), (11, 3)])
    assert np.allclose(got, [full[1][11, 3], full[1][3, 11]], rtol=1e-12, atol=0)


def test_correlate_sampled_equals_visibility_route():
    """correlate_sampled (K_a, P_a of selected antennas with the calibrator
    pixel from the single-pixel sum) gives C_a of Eq. 15 equal to the
    visibility route sum_{b != a} conj(A_{0,b}) V_ab / conj(g_b), and K, P
    equal to correlate() on image_interval's pixel series."""
    rng = np.random.default_rng(32)
    plan, E, gcur = _offcentre_case(rng)
    Na = plan.Na
    ants = [6, 0, 3, 4]
    _, pixser = O.image_interval(plan, E, gcur)
    for c in range(2):
        Kc, P = O.correlate_sampled(plan, E, gcur, c, ants, block=13)
        Kf, Pf = O.correlate(E[:, c, :], pixser[:, c])
        assert np.allclose(Kc, Kf[ants], rtol=1e-12, atol=1e-14)
        assert np.allclose(P, Pf[ants], rtol=1e-12, atol=0)
        V = O.visibilities(E[:, c, :])
        for i, a in enumerate(ants):
            Ca = Kc[i] - np.conj(plan.A0[c, a]) * P[i] / np.conj(gcur[c, a])
            ref = sum(np.conj(plan.A0[c, b]) * V[a, b] / np.conj(gcur[c, b])
                      for b in range(Na) if b != a and not plan.flags[b])
            assert abs(Ca - ref) <= 1e-12 * abs(ref), (c, a)


def test_epical_interval_pixel_only_equals_full_image_route():
    """epical_interval's single-pixel branch (no image) gives the same gains
    and sums as the branch through the full image."""
    rng = np.random.default_rng(33)
    plan, E, gcur = _offcentre_case(rng)
    a = O.epical_interval(plan, E, gcur, 0.4, with_image=True)
    b = O.epical_interval(plan, E, gcur, 0.4, with_image=False)
    for x, y in zip((a[0], a[1], a[2]), (b[0], b[1], b[2])):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-14)
    assert np.array_equal(a[4], b[4])


# --------------------------------------------------------------------------
# EPICal (Eqs. 12-17)
# --------------------------------------------------------------------------
def _tiny_plan_and_data(rng, Na=8, N=16, T=200, cal=(0.0, 0.0), noise=0.5, unit=False,
                        sky=None, flags=None):
    ant = synth.layout_disc(Na, 8.0, rng, 1.0)
    f = [50e6]
    g = synth.true_gains(1, Na, rng)
    if sky is None:
        sky = np.array([[cal[0], cal[1], 4.0], [0.25, 0.1, 1.0]])
    E = synth.voltages(ant, f, g, sky, T, noise, rng, unit_modulus=unit)
    plan = O.Plan(ant, f, N, 0.5, cal_lm=cal, model_lmS=sky, flags=flags)
    return plan, E, g


def test_correlation_equals_visibility_route():
    """Eqs. 13 -> 15 are exact sample-average algebra: C_a from the image
    pixel equals sum_{b != a} conj(A_{0,b}) V_ab / conj(g_b)."""
    rng = np.random.default_rng(2)
    k0 = (19, 13)
    cal = ((k0[0] - 16) / 16.0, (k0[1] - 16) / 16.0)
    flags = np.zeros(9, bool)
    flags[2] = True
    plan, E, g = _tiny_plan_and_data(rng, Na=9, N=32, cal=cal, flags=flags)
    gcur = synth.true_gains(1, 9, rng)[0]
    _, pix = O.image_interval(plan, E, gcur[None])
    Kc, P = O.correlate(E[:, 0, :], pix[:, 0])
    Cc = Kc - np.conj(plan.A0[0]) * P / np.conj(gcur)
    V = O.visibilities(E[:, 0, :])
    ref = np.array([sum(np.conj(plan.A0[0, b]) * V[a, b] / np.conj(gcur[b])
                        for b in range(9) if b != a and not flags[b]) for a in range(9)])
    assert np.max(np.abs(Cc - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_zenith_single_source_limit():
    """Eqs. 18-19: for s0 at the phase centre A_{0,b} = 1/Na exactly, and
    Na C_a = sum_{b != a} V_ab / conj(g_b); the undamped update is that sum
    over (Na - 1) S (Eq. 16 literally; Eq. 19's Na S is its large-Na form)."""
    rng = np.random.default_rng(4)
    Na = 10
    sky = np.array([[0.0, 0.0, 2.5]])
    plan, E, g = _tiny_plan_and_data(rng, Na=Na, sky=sky)
    assert np.allclose(plan.A0[0], 1.0 / Na, atol=1e-15)
    gcur = synth.true_gains(1, Na, rng)[0]
    _, pix = O.image_interval(plan, E, gcur[None])
    Kc, P = O.correlate(E[:, 0, :], pix[:, 0])
    V = O.visibilities(E[:, 0, :])
    Cc = Kc - np.conj(plan.A0[0]) * P / np.conj(gcur)
    ref = np.array([sum(V[a, b] / np.conj(gcur[b]) for b in range(Na) if b != a)
                    for a in range(Na)])
    assert np.allclose(Na * Cc, ref, rtol=1e-12, atol=0)
    gn, _ = O.epical_update(Kc, P, plan.A0[0], plan.D[0], gcur, 0.0)
    assert np.allclose(gn, ref / ((Na - 1) * 2.5), rtol=1e-12)


@pytest.mark.parametrize("cal", [(0.0, 0.0), (0.25, -0.125)])
def test_noise_free_converges_to_true_gains(cal):
    """One unit-modulus source at the calibrator pixel, no noise, injected
    gains: EPICal from g = 1 converges to g e^{i phi}."""
    rng = np.random.default_rng(7)
    Na = 12
    sky = np.array([[cal[0], cal[1], 3.0]])
    plan, E, g = _tiny_plan_and_data(rng, Na=Na, N=16, T=32, sky=sky, noise=0.0,
                                     unit=True)
    gcur = np.ones((1, Na), complex)
    for _ in range(80):
        gcur, *_ = O.epical_interval(plan, E, gcur, 0.35, with_image=False)
    ga = O.align_phase(gcur[0], g[0])
    assert np.max(np.abs(ga - g[0]) / np.abs(g[0])) < 1e-10


def test_damping_closed_form_and_effective_time():
    """Eq. 17 with a fixed C/D = x gives g^(n) = x + gamma^n (g0 - x); the
    weights (1-gamma) gamma^k give t_eff / t_cal = (1+gamma)/(1-gamma)
    (Eq. 20) for the variance of i.i.d. inputs."""
    gamma = 0.35
    A0 = np.array([0.0j, 0.0j])
    D = np.array([2.0 + 1.0j, -1.0 + 0.5j])
    Kc = np.array([1.0 - 2.0j, 0.5 + 0.25j])
    P = np.zeros(2)
    g0 = np.array([1.0 + 0j, 1.0 + 0j])
    x = Kc / D
    g = g0.copy()
    for n in range(1, 30):
        g, _ = O.epical_update(Kc, P, A0, D, g, gamma)
        assert np.allclose(g, x + gamma ** n * (g0 - x), rtol=1e-13)
    # impulse responses: weight of the input j steps back
    n_steps = 200
    w = []
    for j in range(n_steps):
        gg = np.ones(1, complex)   # start value decays as gamma^n_steps ~ 0
        for n in range(n_steps):
            k = np.array([1.0 + 0j]) if n == n_steps - 1 - j else np.zeros(1, complex)
            gg, _ = O.epical_update(k, np.zeros(1), np.zeros(1, complex),
                                    np.ones(1, complex), gg, gamma)
        w.append(gg[0].real)
    w = np.array(w)
    assert np.isclose(w.sum(), 1.0, atol=1e-12)
    assert np.isclose(1.0 / np.sum(w ** 2), (1 + gamma) / (1 - gamma), rtol=1e-10)


def test_update_holds_flagged_and_bad_antennas():
    A0 = np.full(4, 0.25 + 0j)
    D = np.array([1.0 + 0j, 0.0 + 0j, 1.0 + 0j, 1.0 + 0j])
    Kc = np.array([1.0 + 0j, 1.0 + 0j, np.nan + 0j, 1.0 + 0j])
    g = np.array([2.0 + 0j, 3.0 + 0j, 4.0 + 0j, 5.0 + 0j])
    gn, held = O.epical_update(Kc, np.zeros(4), A0, D, g, 0.5, flags=[0, 0, 0, 1])
    assert held.tolist() == [False, True, True, True]
    assert gn[1:].tolist() == g[1:].tolist()
    with pytest.raises(ValueError):
        O.epical_update(Kc, np.zeros(4), A0, D, g, 1.0)


def test_epical_agrees_with_visibility_solve_noise_free():
    """Sec. 4 comparison: on noise-free single-source data both the EPICal
    loop and the Eq. 21 visibility solve recover the true gains up to a
    global phase."""
    rng = np.random.default_rng(8)
    Na = 10
    sky = np.array([[0.0, 0.0, 2.0]])
    plan, E, g = _tiny_plan_and_data(rng, Na=Na, N=16, T=24, sky=sky, noise=0.0, unit=True)
    V = O.visibilities(E[:, 0, :])
    VM = O.model_visibilities(plan.ant, plan.freqs[0], sky)
    gv = O.visibility_solve(V, VM, np.ones(Na, complex))
    gcur = np.ones((1, Na), complex)
    for _ in range(80):
        gcur, *_ = O.epical_interval(plan, E, gcur, 0.35, with_image=False)
    ge = O.align_phase(gcur[0], g[0])
    gvv = O.align_phase(gv, g[0])
    assert np.max(np.abs(ge - gvv) / np.abs(g[0])) < 1e-10
    assert O.gain_error(gvv, g[0]) < 1e-10


def test_visibility_solve_noisy_reduces_chi2():
    rng = np.random.default_rng(9)
    Na = 12
    plan, E, g = _tiny_plan_and_data(rng, Na=Na, N=16, T=400, noise=1.0)
    sky = np.array([[0.0, 0.0, 4.0], [0.25, 0.1, 1.0]])
    V = O.visibilities(E[:, 0, :])
    VM = O.model_visibilities(plan.ant, plan.freqs[0], sky)
    off = ~np.eye(Na, dtype=bool)

    def chi2(gg):
        return np.sum(np.abs(V - np.outer(gg, np.conj(gg)) * VM)[off] ** 2)

    gv = O.visibility_solve(V, VM, np.ones(Na, complex))
    assert chi2(gv) < chi2(g[0]) * 1.0000001
    # stationarity: small perturbations do not lower chi^2
    for d in (1e-4, 1e-4j):
        for a in range(3):
            gp = gv.copy()
            gp[a] += d
            assert chi2(gp) >= chi2(gv) - 1e-12


def test_visibility_solve_baseline_cut():
    """Sec. 5 leaves short baselines out of Eq. 21.  The mask keeps exactly
    the pairs at least min_baseline apart (symmetric, no autos); with
    noise-free data the truth is still the solution, and the masked chi^2
    is stationary at the noisy solution."""
    rng = np.random.default_rng(19)
    Na = 14
    ant = synth.layout_disc(Na, 12.0, rng, 1.0)
    f = 55e6
    uv = O.antenna_uv(ant, f)
    m = O.baseline_mask(uv, 0.7)
    for a in range(Na):
        for b in range(Na):
            want = a != b and np.hypot(*(uv[a] - uv[b])) >= 0.7
            assert m[a, b] == want
    assert m.sum() < Na * (Na - 1) and m.any(axis=1).all()
    sky = np.array([[0.0, 0.0, 3.0], [0.2, -0.3, 1.0]])
    g = synth.true_gains(1, Na, rng)[0]
    E = synth.voltages(ant, [f], g[None], sky, 64, 0.0, rng, tones=True)
    V = O.visibilities(E[:, 0, :])
    VM = O.model_visibilities(ant, f, sky)
    gv = O.visibility_solve(V, VM, np.ones(Na, complex), pair_mask=m)
    assert O.gain_error(O.align_phase(gv, g), g) < 1e-10
    En = synth.voltages(ant, [f], g[None], sky, 300, 1.0, rng)
    Vn = O.visibilities(En[:, 0, :])
    gn = O.visibility_solve(Vn, VM, np.ones(Na, complex), pair_mask=m)

    def chi2(gg):
        return np.sum(np.abs(Vn - np.outer(gg, np.conj(gg)) * VM)[m] ** 2)

    for d in (1e-4, 1e-4j):
        for a in range(3):
            gp = gn.copy()
            gp[a] += d
            assert chi2(gp) >= chi2(gn) - 1e-12


def test_gain_error_metric():
    gt = np.array([[1 + 1j, 2.0 + 0j]])
    ge = np.array([[1.1 + 1.1j, 2.0 + 0.2j]])
    # |0.1(1+i)|^2/|1+i|^2 = 0.01 ; |0.2i|^2/4 = 0.01
    assert np.isclose(O.gain_error(ge, gt), 0.1)


# --------------------------------------------------------------------------
# differentiation form (chi^2 gradient)
# --------------------------------------------------------------------------
def _diff_case(seed=12, Na=9, N=16, T=40):
    rng = np.random.default_rng(seed)
    ant = synth.layout_disc(Na, 8.0, rng, 1.0)
    f = [48e6, 66e6]
    g_true = synth.true_gains(2, Na, rng)
    sky = np.array([[0.0, 0.0, 3.0], [0.2, -0.15, 1.5], [-0.3, 0.25, 0.7]])
    E = synth.voltages(ant, f, g_true, sky, T, 0.3, rng)
    flags = np.zeros(Na, bool)
    flags[4] = True
    plan = O.Plan(ant, f, N, 0.5, flags=flags)
    M = O.model_image(plan, sky)
    return plan, E, g_true, M, rng


def test_model_image_equals_noise_free_unit_modulus_image():
    """The model image is the dirty image of perfectly calibrated, noise-free
    unit-modulus data of one source (Sec. 2.1 image of visibilities)."""
    rng = np.random.default_rng(13)
    ant = synth.layout_disc(10, 8.0, rng, 1.0)
    sky = np.array([[0.25, -0.1, 2.0]])
    g = synth.true_gains(1, 10, rng)
    E = synth.voltages(ant, [55e6], g, sky, 16, 0.0, rng, unit_modulus=True)
    plan = O.Plan(ant, [55e6], 16, 0.5)
    img, _ = O.image_interval(plan, E, g)
    M = O.model_image(plan, sky)
    assert np.max(np.abs(img - M)) <= 1e-12 * np.max(M)
    # so the chi^2 gradient vanishes at the true gains
    assert np.max(np.abs(O.chi2_gradient(plan, E, g, M))) < 1e-10


def test_chi2_gradient_matches_finite_differences():
    """dL = Re(conj(grad) dg) for real and imaginary steps of 1e-6 (central
    differences of the oracle's own loss)."""
    plan, E, g_true, M, rng = _diff_case()
    g = g_true * (1 + 0.1 * (rng.normal(size=g_true.shape) + 1j * rng.normal(size=g_true.shape)))
    grad = O.chi2_gradient(plan, E, g, M)
    h = 1e-6
    for c, a in [(0, 0), (1, 3), (1, 8), (0, 4)]:
        for d in (h, 1j * h):
            gp = g.copy()
            gm = g.copy()
            gp[c, a] += d
            gm[c, a] -= d
            fd = (O.chi2_loss(plan, E, gp, M) - O.chi2_loss(plan, E, gm, M)) / 2
            pred = np.real(np.conj(grad[c, a]) * d)
            assert abs(fd - pred) <= 1e-6 * abs(grad[c, a]) * h + 1e-12, (c, a, d, fd, pred)
    assert np.all(grad[:, 4] == 0)


# --------------------------------------------------------------------------
# gains constant across a band of channels (Sec. 5, LWA demonstration)
# --------------------------------------------------------------------------
def test_average_channels_invariants():
    """In-band channels all take one value per antenna whose band sum equals
    the input's; out-of-band channels and flagged antennas are untouched;
    averaging twice changes nothing; gains already constant across the band
    are left as they are."""
    rng = np.random.default_rng(12)
    C, Na = 7, 9
    g = rng.normal(size=(C, Na)) + 1j * rng.normal(size=(C, Na))
    flags = np.zeros(Na, bool)
    flags[4] = True
    out = O.average_channels(g, 2, 6, flags)
    assert np.array_equal(out[:2], g[:2]) and np.array_equal(out[6:], g[6:])
    assert np.array_equal(out[:, 4], g[:, 4])
    live = ~flags
    assert np.allclose(out[2:6, live], out[2, live][None], rtol=0, atol=0)
    assert np.allclose(out[2:6, live].sum(axis=0), g[2:6, live].sum(axis=0), rtol=1e-14)
    assert np.array_equal(O.average_channels(out, 2, 6, flags), out)
    const = np.repeat(g[:1], C, axis=0)
    assert np.allclose(O.average_channels(const, 0, C), const, rtol=1e-15)
    with pytest.raises(ValueError):
        O.average_channels(g, 3, 3)


def test_channel_averaging_reduces_gain_noise():
    """The reason the paper averages across channels: with the same true
    gains in every channel and independent noise, feedback calibration with
    the per-interval channel average ends closer to the truth than the
    per-channel solutions (same data, same loops)."""
    rng = np.random.default_rng(31)
    Na, C = 10, 6
    ant = synth.layout_disc(Na, 8.0, rng, 1.0)
    f = np.linspace(49e6, 51e6, C)
    g1 = synth.true_gains(1, Na, rng)
    g = np.repeat(g1, C, axis=0)
    sky = np.array([[0.0, 0.0, 4.0], [0.25, 0.1, 1.0]])
    plan = O.Plan(ant, f, 16, 0.5, model_lmS=sky)
    err = {}
    for avg in (False, True):
        rr = np.random.default_rng(5)
        gc = np.ones((C, Na), complex)
        for _ in range(30):
            E = synth.voltages(ant, f, g, sky, 64, 2.0, rr)
            gc, *_ = O.epical_interval(plan, E, gc, 0.5, with_image=False)
            if avg:
                gc = O.average_channels(gc, 0, C)
        err[avg] = np.mean([O.gain_error(O.align_phase(gc[c], g1[0]), g1[0]) for c in range(C)])
    assert err[True] < 0.7 * err[False], err


# --------------------------------------------------------------------------
# heterogeneous illumination patterns (one kernel parameter per antenna)
# --------------------------------------------------------------------------
def test_grid_table_per_antenna_parameters():
    """A per-antenna parameter array equal to the scalar gives the scalar's
    table; with different values, each antenna's stencil is the one it gets
    alone with its own value (antennas do not interact in Eq. 9's weights);
    a wider Gaussian puts less weight on the nearest cell."""
    rng = np.random.default_rng(17)
    ant = rng.uniform(-8, 8, size=(12, 2))
    freqs = [45e6, 70e6]
    b0, W0 = O.grid_table(ant, freqs, 64, 0.5, "gaussian", 5, 0.6)
    b1, W1 = O.grid_table(ant, freqs, 64, 0.5, "gaussian", 5, np.full(12, 0.6))
    assert np.array_equal(b0, b1) and np.array_equal(W0, W1)
    sig = rng.uniform(0.3, 1.2, 12)
    b2, W2 = O.grid_table(ant, freqs, 64, 0.5, "gaussian", 5, sig)
    for a in range(12):
        ba, Wa = O.grid_table(ant[a:a + 1], freqs, 64, 0.5, "gaussian", 5, sig[a])
        assert np.array_equal(b2[:, a], ba[:, 0]) and np.array_equal(W2[:, a], Wa[:, 0])
    narrow, wide = np.argmin(sig), np.argmax(sig)
    for c in range(2):
        assert W2[c, narrow, 2, 2] > W2[c, wide, 2, 2]


def test_noise_free_converges_with_per_antenna_kernels_off_centre():
    """With one Gaussian width per antenna and the calibrator off the phase
    centre, A_{0,a} differs antenna by antenna; the noise-free feedback
    loop still converges to the injected gains (up to a global phase),
    which holds only if the discrete A_0 uses each antenna's own stencil."""
    rng = np.random.default_rng(23)
    Na, N = 12, 32
    ant = synth.layout_disc(Na, 8.0, rng, 1.0)
    f = [50e6]
    k0 = (19, 13)
    cal = ((k0[0] - N / 2) / (N * 0.5), (k0[1] - N / 2) / (N * 0.5))
    sky = np.array([[cal[0], cal[1], 3.0]])
    g = synth.true_gains(1, Na, rng)
    E = synth.voltages(ant, f, g, sky, 32, 0.0, rng, unit_modulus=True)
    sig = rng.uniform(0.35, 0.9, Na)
    plan = O.Plan(ant, f, N, 0.5, support=5, param=sig, cal_lm=cal, model_lmS=sky)
    assert np.ptp(np.abs(plan.A0[0])) > 1e-3           # the stencils matter here
    gcur = np.ones((1, Na), complex)
    for _ in range(80):
        gcur, *_ = O.epical_interval(plan, E, gcur, 0.35, with_image=False)
    ga = O.align_phase(gcur[0], g[0])
    assert np.max(np.abs(ga - g[0]) / np.abs(g[0])) < 1e-9


# --------------------------------------------------------------------------
# multiple-pixel and direction-dependent EPICal (Sec. 6)
# --------------------------------------------------------------------------
def _mp_case(rng, Na=9, N=32, T=120, noise=0.5, tones=False, flags=None, sky=None, dd=None):
    ant = synth.layout_disc(Na, 10.0, rng, 1.0)
    f = [50e6, 58e6]
    g = synth.true_gains(2, Na, rng)
    if sky is None:
        sky = np.array([[0.0, 0.0, 4.0], [0.3125, -0.1875, 2.0], [-0.25, 0.375, 1.5]])
    gv = g if dd is None else dd
    E = synth.voltages(ant, f, gv, sky, T, noise, rng, tones=tones)
    plan = O.MultiPixelPlan(ant, f, N, 0.5, sky[:, :2], sky, flags=flags)
    return plan, E, g, sky


def test_multipixel_single_pixel_reduces_to_epical():
    """P = 1: the least-squares combination over pixels is Eq. 16 itself and
    the per-direction update equals the joint one."""
    rng = np.random.default_rng(60)
    ant = synth.layout_disc(8, 9.0, rng, 1.0)
    sky = np.array([[0.125, -0.0625, 3.0], [0.3, 0.2, 1.0]])
    E = synth.voltages(ant, [52e6], synth.true_gains(1, 8, rng), sky, 90, 0.7, rng)
    mp = O.MultiPixelPlan(ant, [52e6], 16, 0.5, sky[:1, :2], sky, cal_lm=sky[0, :2])
    sp = O.Plan(ant, [52e6], 16, 0.5, cal_lm=sky[0, :2], model_lmS=sky)
    assert mp.pix == [sp.k0]
    assert np.array_equal(mp.Ap[0, 0], sp.A0[0]) and np.array_equal(mp.Dp[0, 0], sp.D[0])
    g = synth.true_gains(1, 8, rng)
    ref, *_ = O.epical_interval(sp, E, g, 0.3, with_image=False)
    got, gd, *_ = O.multipixel_interval(mp, E, g, g[:, :, None], 0.3)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)
    assert np.allclose(gd[:, :, 0], ref, rtol=1e-13, atol=0)


def test_multipixel_correlation_equals_visibility_route():
    """Eqs. 13 -> 15 per pixel: C_{a,p} from the pixel correlations equals
    sum_{b != a} conj(A_{p,b}) V_ab / conj(g_b) for every antenna and pixel
    (flagged antenna included), and the joint update is the least-squares
    formula evaluated on that route."""
    rng = np.random.default_rng(61)
    flags = np.zeros(9, bool)
    flags[5] = True
    plan, E, g, sky = _mp_case(rng, flags=flags)
    gcur = synth.true_gains(2, 9, rng)
    for c in range(2):
        taps = O.pixel_taps(plan, E[:, c, :] / gcur[c], c, plan.pix)
        Kc, P = O.correlate_multi(E[:, c, :], taps)
        gn, held, Cc = O.multipixel_update(Kc, P, plan.Ap[c], plan.Dp[c], gcur[c], 0.25, flags)
        V = O.visibilities(E[:, c, :])
        ref = np.array([[sum(np.conj(plan.Ap[c, p, b]) * V[a, b] / np.conj(gcur[c, b])
                             for b in range(9) if b != a and not flags[b])
                         for p in range(3)] for a in range(9)])
        assert np.max(np.abs(Cc - ref)) <= 1e-12 * np.max(np.abs(ref))
        D = plan.Dp[c].T
        ls = np.array([np.vdot(D[a], ref[a]) / np.vdot(D[a], D[a]) for a in range(9)])
        want = np.where(flags, gcur[c], 0.75 * ls + 0.25 * gcur[c])
        assert np.allclose(gn, want, rtol=1e-12, atol=0)
        assert held[5] and not held[np.arange(9) != 5].any()


def test_multipixel_noise_free_converges_joint_and_per_direction():
    """Three sources with mutually orthogonal tone signals, no noise: the
    sample visibilities equal g_a conj(g_b) V^M_ab exactly, so the joint
    solution and every per-direction solution converge to the true gains
    up to one global phase."""
    rng = np.random.default_rng(62)
    plan, E, g, sky = _mp_case(rng, Na=10, N=32, T=64, noise=0.0, tones=True)
    gc = np.ones((2, 10), complex)
    gd = np.ones((2, 10, 3), complex)
    for _ in range(120):
        gc, gd, *_ = O.multipixel_interval(plan, E, gc, gd, 0.35)
    for c in range(2):
        ga = O.align_phase(gc[c], g[c])
        assert np.max(np.abs(ga - g[c]) / np.abs(g[c])) < 1e-9
        for p in range(3):
            gp = O.align_phase(gd[c, :, p], g[c])
            assert np.max(np.abs(gp - g[c]) / np.abs(g[c])) < 1e-9


def test_multipixel_tracks_direction_dependent_gains():
    """Gains that differ by direction (one set per source): with two
    well-separated, equally bright sources and the imaging gains held at
    the mean response, each per-direction solution lies much closer to its
    own source's gains than to the other source's.  The residual is the
    array's sidelobe response to the other source, which falls with Na
    (ratio about 0.3-0.5 at Na = 24, below 0.25 at Na = 64)."""
    rng = np.random.default_rng(63)
    Na = 64
    sky = np.array([[0.25, 0.0, 3.0], [-0.25, 0.125, 3.0]])
    g0 = synth.true_gains(1, Na, rng)[0]
    dd = np.empty((2, Na, 2), complex)
    for c in range(2):
        dd[c, :, 0] = g0 * (1 + 0.15 * rng.normal(size=Na)) * np.exp(0.2j * rng.normal(size=Na))
        dd[c, :, 1] = g0 * (1 + 0.15 * rng.normal(size=Na)) * np.exp(0.2j * rng.normal(size=Na))
    ant = synth.layout_disc(Na, 20.0, rng, 1.0)
    f = [50e6, 58e6]
    E = synth.voltages(ant, f, dd, sky, 256, 0.0, rng, tones=True)
    plan = O.MultiPixelPlan(ant, f, 64, 0.5, sky[:, :2], sky)
    gimg = 0.5 * (dd[:, :, 0] + dd[:, :, 1])
    gd = np.repeat(gimg[:, :, None], 2, axis=2)
    for _ in range(40):
        _, gd, *_ = O.multipixel_interval(plan, E, gimg, gd, 0.35)
    for c in range(2):
        for p, q in ((0, 1), (1, 0)):
            own = O.gain_error(O.align_phase(gd[c, :, p], dd[c, :, p]), dd[c, :, p])
            other = O.gain_error(O.align_phase(gd[c, :, p], dd[c, :, q]), dd[c, :, q])
            assert own < 0.3 * other, (c, p, own, other)


# --------------------------------------------------------------------------
# bandpass model fitted across channels (Sec. 6, "Fitting gain models")
# --------------------------------------------------------------------------
def test_fit_bandpass_recovers_polynomial_gains_exactly():
    """Gains that are exactly a degree-2 amplitude and a degree-3 phase
    polynomial in frequency (phase wrapping several times across the band)
    are returned unchanged by the fit of those degrees; channels outside the
    band and a flagged antenna are untouched."""
    rng = np.random.default_rng(70)
    C, Na = 24, 7
    freqs = np.linspace(40e6, 80e6, C)
    g = synth.true_gains(C, Na, rng)
    c_lo, c_hi = 3, 21
    x = O.bandpass_x(freqs, c_lo, c_hi)
    assert np.isclose(x[0], -1) and np.isclose(x[-1], 1)
    want = g.copy()
    for a in range(Na):
        amp = 1.0 + 0.1 * a + 0.2 * x - 0.05 * x ** 2
        ph = 0.3 * a + 9.0 * x + 1.5 * x ** 2 - 2.0 * x ** 3       # > 2 pi across the band
        want[c_lo:c_hi, a] = amp * np.exp(1j * ph)
    flags = np.zeros(Na, bool)
    flags[4] = True
    got = O.fit_bandpass(want, freqs, c_lo, c_hi, 2, 3, flags)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    noisy = want.copy()
    noisy[c_lo:c_hi] *= 1 + 0.05 * rng.normal(size=(c_hi - c_lo, Na))
    fit = O.fit_bandpass(noisy, freqs, c_lo, c_hi, 2, 3, flags)
    assert np.array_equal(fit[:c_lo], noisy[:c_lo]) and np.array_equal(fit[c_hi:], noisy[c_hi:])
    assert np.array_equal(fit[:, 4], noisy[:, 4])


def test_fit_bandpass_degree_zero_is_mean_amplitude_and_phase():
    """Degree 0 in both: every channel of the band gets the mean amplitude and
    the mean unwrapped phase of the antenna's solutions there."""
    rng = np.random.default_rng(71)
    C, Na = 10, 5
    freqs = np.linspace(50e6, 60e6, C)
    g = synth.true_gains(C, Na, rng)
    fit = O.fit_bandpass(g, freqs, 2, 9, 0, 0)
    for a in range(Na):
        band = g[2:9, a]
        want = np.mean(np.abs(band)) * np.exp(1j * np.mean(np.unwrap(np.angle(band))))
        assert np.allclose(fit[2:9, a], want, rtol=1e-13, atol=0)


def test_fit_bandpass_reduces_gain_noise():
    """Noisy per-channel solutions around a smooth bandpass (the situation
    Sec. 6 describes): the fitted gains lie closer to the truth."""
    rng = np.random.default_rng(72)
    C, Na = 64, 32
    freqs = np.linspace(40e6, 80e6, C)
    x = O.bandpass_x(freqs, 0, C)
    true = np.empty((C, Na), complex)
    for a in range(Na):
        c0, c1 = rng.normal(size=2)
        true[:, a] = (1.0 + 0.1 * c0 * x) * np.exp(1j * (rng.uniform(-np.pi, np.pi) + 3.0 * c1 * x))
    noisy = true * (1 + 0.1 * (rng.normal(size=(C, Na)) + 1j * rng.normal(size=(C, Na))))
    fit = O.fit_bandpass(noisy, freqs, 0, C, 2, 2)
    assert O.gain_error(fit, true) < 0.4 * O.gain_error(noisy, true)


# --------------------------------------------------------------------------
# phasing off zenith (Sec. 2.1 footnote)
# --------------------------------------------------------------------------
def test_phased_image_is_the_shifted_sky():
    """A planar array phased to s0 images a sky exactly as the unphased array
    images that sky moved by -s0 (same source signals, no noise), and the
    calibration response of the phase-centre pixel is p_a / Na."""
    rng = np.random.default_rng(80)
    Na, N, T = 20, 32, 40
    ant = synth.layout_disc(Na, 12.0, rng, 1.0)
    f = [50e6, 66e6]
    s0 = (0.3125, -0.21875)
    sky = np.array([[0.35, -0.2, 3.0], [0.1, 0.05, 1.0], [0.5, -0.4, 2.0]])
    g = synth.true_gains(2, Na, rng)
    E = synth.voltages(ant, f, g, sky, T, 0.0, np.random.default_rng(5))
    shifted = sky - np.array([s0[0], s0[1], 0.0])
    Es = synth.voltages(ant, f, g, shifted, T, 0.0, np.random.default_rng(5))
    pp = O.Plan(ant, f, N, 0.5, phase_lm=s0, cal_lm=s0)
    p0 = O.Plan(ant, f, N, 0.5)
    img, _ = O.image_interval(pp, E, g)
    ref, _ = O.image_interval(p0, Es, g)
    assert np.max(np.abs(img - ref)) <= 1e-12 * np.max(ref)
    assert pp.k0 == (N // 2, N // 2)
    assert np.allclose(pp.A0, pp.phase / Na, rtol=1e-13, atol=0)


def test_phased_epical_converges_off_zenith():
    """Calibrator at 40 degrees from zenith, array phased to it: noise-free
    EPICal from g = 1 converges to the true gains (global phase)."""
    rng = np.random.default_rng(81)
    Na = 14
    ant = synth.layout_disc(Na, 10.0, rng, 1.0)
    s0 = (0.5, 0.375)                        # sin(theta) ~ 0.63
    sky = np.array([[s0[0], s0[1], 3.0]])
    g = synth.true_gains(1, Na, rng)
    E = synth.voltages(ant, [52e6], g, sky, 32, 0.0, rng, unit_modulus=True)
    plan = O.Plan(ant, [52e6], 16, 0.5, cal_lm=s0, model_lmS=sky, phase_lm=s0)
    gc = np.ones((1, Na), complex)
    for _ in range(80):
        gc, *_ = O.epical_interval(plan, E, gc, 0.35, with_image=False)
    ga = O.align_phase(gc[0], g[0])
    assert np.max(np.abs(ga - g[0]) / np.abs(g[0])) < 1e-10

