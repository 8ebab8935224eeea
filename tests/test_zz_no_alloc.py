"""epic_image_host_static: the imaging call that allocates no device memory.

Callers such as a real-time loop that may not insert a device-synchronising
cudaMalloc between intervals, or a process confined to a device-memory
budget fixed at start-up, use this entry point; it stages through the
library's fixed 32 MiB device array instead of plan buffers grown with
cudaMalloc.  It must give the same images as epic_image_host, call after
call, although every call reuses (and must first clear) the same array.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import epic_synth as synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5   # the FP32 image bar of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_scratch_matches_image_host_two_calls():
    from paper_1603_02126_gb300 import Plan
    # 64 channels x 2500 samples: the 8 MiB image leaves room for 1536
    # samples per chunk, so each call runs two chunks
    w = synth.workload("lwa", n_time=2500)
    rng = np.random.default_rng(3)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:60], 2500,
                       w["noise_power"], rng)
    b1 = synth.quantise_ci4(E, w["lsb"])
    b2 = synth.quantise_ci4(E[::-1].copy() * 0.7, w["lsb"])
    p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
             voltage_scale=w["lsb"])
    for b in (b1, b2):
        ref = p.image_host(b)
        got = p.image_host_static(b)
        assert got.shape == ref.shape
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) <= IMG_TOL
    # accumulate: starts from the caller's image, not from the array's leftovers
    base = p.image_host(b1)
    acc = p.image_host_static(b2, base.copy(), accumulate=True)
    assert _rel(acc, base + p.image_host(b2)) <= IMG_TOL


def test_static_scratch_rejects_oversized_image():
    from paper_1603_02126_gb300 import EpicError, Plan
    rng = np.random.default_rng(4)
    ant = synth.layout_disc(16, 10.0, rng, 1.0)
    freqs = np.linspace(40e6, 60e6, 260)      # 260 x 128^2 x 8 B > 32 MiB
    p = Plan(ant, freqs, 128, 0.5, input="ci4")
    v = np.zeros((2, 260, 16), np.uint8)
    with pytest.raises(EpicError) as ei:
        p.image_host_static(v)
    assert "static scratch" in str(ei.value)


def test_static_scratch_epical_interval_matches_image_host():
    """EPICal armed: one interval imaged in two chunks through the static
    array accumulates the same K_a, P_a and frame count as epic_image_host,
    so the gain updates agree within the parity bar (1e-4)."""
    from paper_1603_02126_gb300 import Plan
    w = synth.workload("lwa", n_time=2500)
    rng = np.random.default_rng(5)
    E = synth.voltages(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:60], 2500,
                       w["noise_power"], rng)
    b = synth.quantise_ci4(E, w["lsb"])
    plans = [Plan(w["ant_xy"], w["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
                  voltage_scale=w["lsb"]) for _ in range(2)]
    for p in plans:
        p.configure((0.0, 0.0), w["model"], w["gamma"])
    img_ref = plans[0].image_host(b)
    img_got = plans[1].image_host_static(b)
    assert _rel(img_got, img_ref) <= IMG_TOL
    assert plans[0].info()["frames_pending"] == plans[1].info()["frames_pending"] == 2500
    for p in plans:
        p.update()
        assert p.sync() == 0
    g_ref, g_got = plans[0].gains(), plans[1].gains()
    amp = np.max(np.abs(np.abs(g_got) - np.abs(g_ref)) / np.abs(g_ref))
    ph = np.max(np.abs(np.angle(g_got * np.conj(g_ref))))
    assert amp <= 1e-4 and ph <= 1e-4, (amp, ph)


def test_static_scratch_refuses_non_fused_plan():
    """A plan on any other path needs its own scratch: UNSUPPORTED, before
    the size check (this unfused plan's image would also exceed the array)."""
    from paper_1603_02126_gb300 import EpicError, Plan
    rng = np.random.default_rng(6)
    ant = synth.layout_disc(16, 10.0, rng, 1.0)
    freqs = np.linspace(40e6, 60e6, 260)
    p = Plan(ant, freqs, 128, 0.5, input="ci4", path="unfused")
    with pytest.raises(EpicError) as ei:
        p.image_host_static(np.zeros((2, 260, 16), np.uint8))
    assert ei.value.status == 7           # EPIC_ERR_UNSUPPORTED
