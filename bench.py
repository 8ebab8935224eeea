"""Throughput of the EPIC imaging + EPICal calibration hot path on GB300.

One step = one calibration interval of the LWA-like workload (Na = 256
antennas in a 100 m x 90 m ellipse, 64 channels in 40-80 MHz, 128 x 128
grid, 3 x 3 Gaussian kernel, T = 10^4 samples of 4-bit complex voltages):
epic_image (unpack, gain correction, gridding, 2D FFT, square-accumulate and
the antenna-pixel correlation, one fused launch) followed by epical_update
(the damped gain update).  Metric: calibrated E-field frames per second,
frames = channels x time samples.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank images its own interval
(channels are independent), no collective on the data path; value = all
frames / slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import epic_synth as synth  # noqa: E402

METRIC = "calibrated E-field frames/s (Na=256, 128^2 grid) & gain-solve ms, vs plain FP32"
WORKLOAD = ("LWA-like: Na=256 in a 100 m x 90 m ellipse, C=64 channels 40-80 MHz, N=128, "
            "du=0.5 wavelength, 3x3 Gaussian (sigma 0.5 cell), T=10000 4-bit complex samples "
            "per calibration interval, EPICal armed (calibrator at the phase centre, 50-source "
            "model, gamma=0.5)")
NUM_SMS = 152
FP32_LANES_PER_SM = 128
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one fused image launch
# on this workload, with kernel_sha() of the sources it was taken at;
# ignored when those sources have changed since.
TRAFFIC = {"kernel_sha": "ffbd609a2fe4", "bytes_per_launch": 182208512}


def kernel_sha() -> str:
    """sha256 (first 12 hex) of the fused kernel's sources (kernel file and
    the FFT helpers it inlines)."""
    h = hashlib.sha256()
    for f in ("epic_kernels.cu", "epic_fft.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1603_02126_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def algorithmic_flops_per_frame(na, n, k):
    """Algorithmic FP32 work of one frame: radix-2 count of the N x N
    complex FFT 5 N^2 log2(N^2), gain + gridding 6 Na + 4 Na K^2,
    square-accumulate 3 N^2, EPICal correlation 11 Na."""
    return 5 * n * n * math.log2(n * n) + 6 * na + 4 * na * k * k + 3 * n * n + 11 * na


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(device, n_time=None):
    w = synth.workload("lwa", n_time=n_time)
    volt = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"], w["n_time"],
                                    w["noise_power"], w["lsb"], seed=1, device=device)
    return w, volt


def aggregate_ranks(total_ms, frames_per_rank, steps, dist=None, device=None):
    """Whole-job figures: the slowest rank's time bounds the job (every rank
    images its own channels, so no data moves between ranks); value = all
    ranks' frames per second.  Returns (ms_per_step, value, world)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    return ms_per_step, frames_per_rank * world / (ms_per_step / 1e3), world


def cpu_baseline(w, volt_cpu, budget_s=15.0):
    """The FP64 oracle as it stands, one channel of the same interval, on as
    many frames as fit the time budget (frames/s)."""
    import oracle as O
    c = 0
    oplan = O.Plan(w["ant_xy"], [w["freqs"][c]], w["grid_n"], w["cell"], support=3, param=0.5,
                   model_lmS=w["model"])
    g = np.ones((1, w["ant_xy"].shape[0]), complex)
    frames = 0
    t0 = time.perf_counter()
    blk = 64
    while time.perf_counter() - t0 < budget_s and frames + blk <= volt_cpu.shape[0]:
        E = O.unpack_ci4(volt_cpu[frames:frames + blk, c:c + 1, :]) * w["lsb"][c]
        O.epical_interval(oplan, E, g, w["gamma"], with_image=True)
        frames += blk
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {"value": frames / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"channel 0 of the interval, first {frames} frames "
                      f"(image + EPICal correlation and update, FP64 NumPy), {dt:.1f} s"}


def _timer(torch, flush, stream):
    """Median CUDA-event time (ms) of fn() over reps, L2 flushed before each."""
    def run(fn, reps):
        out = []
        for _ in range(reps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))
    return run


def forms(torch, Plan, dev, stream, flush, w1, volt1, steps):
    """The other forms of the hot path, each on its own workload, timed as
    speedups over the plain FP32 form of the same workload."""
    run = _timer(torch, flush, stream)
    reps = max(3, min(steps, 5))
    out = {}
    sc = stream.cuda_stream
    kw1 = dict(support=3, param=0.5, input="ci4", voltage_scale=w1["lsb"], stream=sc)
    C1 = len(w1["freqs"])
    img1 = torch.empty((C1, 128, 128), dtype=torch.float64, device=dev)

    # -- LWA-like interval: plain unfused FP32 vs fused FP32 vs graph + autotune
    pu = Plan(w1["ant_xy"], w1["freqs"], 128, 0.5, path="unfused", workspace_bytes=4 << 30, **kw1)
    pu.configure((0.0, 0.0), w1["model"], w1["gamma"])
    pf = Plan(w1["ant_xy"], w1["freqs"], 128, 0.5, path="fused", **kw1)
    pf.configure((0.0, 0.0), w1["model"], w1["gamma"])
    gout = torch.empty((C1, 256), dtype=torch.complex128, device=dev)
    for p in (pu, pf):
        p.image(volt1, img1)
        p.update(gout)
    ms_plain = run(lambda: (pu.image(volt1, img1), pu.update(gout)), reps)
    ms_fused = run(lambda: (pf.image(volt1, img1), pf.update(gout)), reps)
    info_u = pu.info()
    rows = info_u["window_rows"]
    # plain path bytes per frame: row spectra written by the gather + row-FFT
    # kernel and read back by the column FFTs (window rows of the widest
    # channel), voltages read twice (gridding, correlation)
    per_frame = 2 * rows * 128 * 8 + 2 * 256
    plain_gbs = per_frame * C1 * w1["n_time"] / (ms_plain / 1e3) / 1e9
    hbm_peak = float(peaks()[0].get("hbm_gbs", 6800.0))
    tune = pf.autotune(volt1, img1)
    pf.graph_capture(volt1, img1, gout)
    ms_graph = run(pf.graph_launch, reps)
    frames1 = C1 * w1["n_time"]
    out["lwa256_n128"] = {
        "workload": "LWA-like interval, Na=256, C=64, N=128, T=10000 (as the headline)",
        "plain_fp32_unfused": {"ms": ms_plain, "frames_per_s": frames1 / ms_plain * 1e3,
                               "hbm_gbs": plain_gbs, "hbm_frac": plain_gbs / hbm_peak},
        "fused_fp32": {"ms": ms_fused, "frames_per_s": frames1 / ms_fused * 1e3,
                       "speedup_vs_plain": ms_plain / ms_fused},
        "batched_graph_autotuned": {"ms": ms_graph, "frames_per_s": frames1 / ms_graph * 1e3,
                                    "speedup_vs_plain": ms_plain / ms_graph, "tune": tune},
    }
    pu.close()
    pf.close()

    # -- precision: Na=1024, C=32, N=256, T=4096 (4-bit), FP16/BF16 tensor cores vs plain FP32
    w2 = synth.workload("compact1024")
    v2 = synth.voltages_ci4_torch(w2["ant_xy"], w2["freqs"], w2["gains"], w2["sky"], w2["n_time"],
                                  w2["noise_power"], w2["lsb"], seed=2, device=dev)
    C2 = len(w2["freqs"])
    img2 = torch.empty((C2, 256, 256), dtype=torch.float64, device=dev)
    kw2 = dict(support=3, param=0.5, input="ci4", voltage_scale=w2["lsb"], stream=sc)
    res2 = {"workload": "Na=1024 in a 200 m disc, C=32 ch 40-80 MHz, N=256, T=4096, 4-bit"}
    ref_img = None
    frames2 = C2 * w2["n_time"]
    ms_p2 = None
    for prec in ("fp32", "fp16", "bf16"):
        p = Plan(w2["ant_xy"], w2["freqs"], 256, 0.5, path="unfused", precision=prec,
                 workspace_bytes=4 << 30, **kw2)
        p.image(v2, img2)
        ms = run(lambda: p.image(v2, img2), reps)
        p.image(v2, img2)
        torch.cuda.synchronize()
        img = img2.clone()
        entry = {"ms": ms, "frames_per_s": frames2 / ms * 1e3}
        if prec == "fp32":
            ref_img = img
            ms_p2 = ms
        else:
            entry["speedup_vs_plain_fp32"] = ms_p2 / ms
            entry["image_rel_l2_vs_fp32"] = float(torch.linalg.norm(img - ref_img) /
                                                  torch.linalg.norm(ref_img))
        res2[prec] = entry
        p.close()
    out["compact1024_n256"] = res2
    del v2, img2

    # -- batching: Na=2048 hex, C=256, N=512, T=4096 (complex64), plain vs graph + autotune
    w3 = synth.workload("hex2048")
    v3 = synth.voltages_c64_torch(w3["ant_xy"], w3["freqs"], w3["gains"], w3["sky"], w3["n_time"],
                                  w3["noise_power"], seed=3, device=dev)
    C3 = len(w3["freqs"])
    img3 = torch.empty((C3, 512, 512), dtype=torch.float64, device=dev)
    g3 = torch.empty((C3, 2048), dtype=torch.complex128, device=dev)
    kw3 = dict(support=3, param=0.5, input="c64", stream=sc)
    frames3 = C3 * w3["n_time"]
    # plain and batched forms with the same 8 GiB batch scratch
    p3 = Plan(w3["ant_xy"], w3["freqs"], 512, 0.5, path="unfused", workspace_bytes=8 << 30, **kw3)
    p3.configure((0.0, 0.0), w3["model"], w3["gamma"])
    p3.image(v3, img3)
    p3.update(g3)
    ms_p3 = run(lambda: (p3.image(v3, img3), p3.update(g3)), 2)
    p3b = Plan(w3["ant_xy"], w3["freqs"], 512, 0.5, path="unfused", workspace_bytes=8 << 30, **kw3)
    p3b.configure((0.0, 0.0), w3["model"], w3["gamma"])
    tune3 = p3b.autotune(v3[:256], img3)
    p3b.graph_capture(v3, img3, g3)
    p3b.graph_launch()
    ms_b3 = run(p3b.graph_launch, 2)
    # one persistent cooperative launch per interval (+ the update) in a graph
    p3p = Plan(w3["ant_xy"], w3["freqs"], 512, 0.5, path="unfused", workspace_bytes=8 << 30,
               batch_persistent=True, **kw3)
    p3p.configure((0.0, 0.0), w3["model"], w3["gamma"])
    p3p.graph_capture(v3, img3, g3)
    p3p.graph_launch()
    ms_pg3 = run(p3p.graph_launch, 2)
    out["hex2048_n512"] = {
        "workload": "Na=2048 hexagonal 8 m pitch +-0.5 m jitter, C=256 ch 50-100 MHz, N=512, "
                    "T=4096 complex64, EPICal armed",
        "plain_fp32": {"ms": ms_p3, "frames_per_s": frames3 / ms_p3 * 1e3},
        "batched_graph_autotuned": {"ms": ms_b3, "frames_per_s": frames3 / ms_b3 * 1e3,
                                    "speedup_vs_plain": ms_p3 / ms_b3, "tune": tune3},
        "persistent_graph": {"ms": ms_pg3, "frames_per_s": frames3 / ms_pg3 * 1e3,
                             "speedup_vs_plain": ms_p3 / ms_pg3, "launches_per_interval": 2},
    }
    p3.close()
    p3b.close()
    p3p.close()
    del v3, img3

    # -- differentiation: Na=256, N=128, C=16, T=4096; chi^2 to the 50-source model image
    from paper_1603_02126_gb300.autograd import EpicImageFn, chi2, solve_gains
    w4 = synth.workload("lwa_diff")
    v4 = synth.voltages_ci4_torch(w4["ant_xy"], w4["freqs"], w4["gains"], w4["sky"][:50],
                                  w4["n_time"], w4["noise_power"], w4["lsb"], seed=4, device=dev)
    C4 = len(w4["freqs"])
    mf = torch.from_numpy(synth.model_frames_c64(w4["ant_xy"], w4["freqs"], w4["model"])).to(dev)
    pm = Plan(w4["ant_xy"], w4["freqs"], 128, 0.5, input="c64", stream=sc)
    M = pm.image(mf) * mf.shape[0]
    pm.close()
    p4 = Plan(w4["ant_xy"], w4["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
              voltage_scale=w4["lsb"], stream=sc)
    g_true = torch.from_numpy(w4["gains"]).to(dev)

    def fwd_bwd():
        g = g_true.clone().requires_grad_(True)
        chi2(EpicImageFn.apply(g, v4, p4), M).backward()

    fwd_bwd()
    ms_fb = run(fwd_bwd, reps)
    ms_f = run(lambda: p4.image(v4), reps)
    # gradient solve vs EPICal, both from gains within ~10 % / 0.2 rad of the truth
    rng = np.random.default_rng(44)
    pert = (1 + 0.1 * rng.normal(size=w4["gains"].shape)) * np.exp(0.2j * rng.normal(size=w4["gains"].shape))
    g0 = torch.from_numpy(w4["gains"] * pert).to(dev)
    # first use of autograd and of the optimiser initialises torch's
    # machinery once (seconds): warm it up outside the timed solve
    solve_gains(p4, v4, M, g0, steps=2, lr=0.01, decay=0.97)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_adam = solve_gains(p4, v4, M, g0, steps=60, lr=0.01, decay=0.97)
    torch.cuda.synchronize()
    adam_s = time.perf_counter() - t0
    # the BF16 option of the adjoint's transforms: gradient vs the FP32 one
    # (itself within 1e-4 of the FP64 oracle in the tests), timing, solve
    def grad_at(prec):
        p4.set_adjoint_precision(prec)
        g = g_true.clone().requires_grad_(True)
        chi2(EpicImageFn.apply(g, v4, p4), M).backward()
        return g.grad

    gr32, gr16 = grad_at("fp32"), grad_at("bf16")
    bf16_grad_err = float(torch.linalg.norm(gr16 - gr32) / torch.linalg.norm(gr32))
    ms_fb16 = run(fwd_bwd, reps)
    t0 = time.perf_counter()
    g_adam16 = solve_gains(p4, v4, M, g0, steps=60, lr=0.01, decay=0.97)
    torch.cuda.synchronize()
    adam16_s = time.perf_counter() - t0
    p4.set_adjoint_precision("fp32")
    pe = Plan(w4["ant_xy"], w4["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
              voltage_scale=w4["lsb"], stream=sc)
    pe.configure((0.0, 0.0), w4["model"], w4["gamma"], g0=w4["gains"] * pert)
    t0 = time.perf_counter()
    for _ in range(60):
        pe.image(v4)
        pe.update()
    pe.sync()
    epical_s = time.perf_counter() - t0

    def sig(g):
        """sigma_g (Eq. 22) after removing each channel's global phase."""
        gt = w4["gains"]
        ph = np.angle(np.sum(g * np.conj(gt), axis=1, keepdims=True))
        ga = g * np.exp(-1j * ph)
        return float(np.sqrt(np.mean(np.abs(ga - gt) ** 2 / np.abs(gt) ** 2)))

    out["lwa_diff_n128"] = {
        "workload": "Na=256 (LWA-like), N=128, C=16, T=4096, 4-bit; loss = chi^2 to the 50-source "
                    "model image",
        "forward_ms": ms_f, "forward_backward_ms": ms_fb,
        "adam_60_steps": {"s": adam_s, "ms_per_step": adam_s / 60 * 1e3, "sigma_g": sig(g_adam.cpu().numpy())},
        "bf16_adjoint": {"forward_backward_ms": ms_fb16, "backward_speedup": (ms_fb - ms_f) / (ms_fb16 - ms_f),
                         "grad_rel_l2_vs_fp32": bf16_grad_err,
                         "adam_60_steps": {"s": adam16_s, "sigma_g": sig(g_adam16.cpu().numpy())}},
        "epical_60_loops": {"s": epical_s, "sigma_g": sig(pe.gains())},
        "sigma_g_start": sig(w4["gains"] * pert),
    }
    p4.close()
    pe.close()
    out["noise_trends"] = noise_trends(torch, Plan, dev, stream, run)
    return out


def noise_trends(torch, Plan, dev, stream, run):
    """Sec. 4 noise-trend sweep on the LWA-like array (64 channels, 4-bit):
    EPICal (10 loops of t_cal from the true gains, gamma = 0.35) against the
    visibility solve of Eq. 21 on visibilities of the last t_eff = t_cal (1 +
    gamma) / (1 - gamma) samples of the same stream, each with the full sky
    model and with the calibrator alone; sigma_g of Eq. 22 after removing
    each channel's global phase, and the GPU time of each stage."""
    w = synth.workload("noise")
    C, Na = len(w["freqs"]), w["ant_xy"].shape[0]
    gam = w["gamma"]
    sc = stream.cuda_stream

    def sig(g):
        ph = np.angle(np.sum(g, axis=1, keepdims=True))     # true gains are 1
        return float(np.sqrt(np.mean(np.abs(g * np.exp(-1j * ph) - 1.0) ** 2)))

    res = {"workload": "Sec. 4 sky (5 Jy calibrator + 49 sources of 0.2-0.5 Jy) on the LWA-like array, "
                       "C=64, N=128, 4-bit, true gains 1", "rows": []}
    for noise in (10.0, 100.0):
        rms = np.sqrt((w["sky"][:, 2].sum() + noise) / 2)
        lsb = np.full(C, rms / 2.0)
        for t_cal in (128, 512, 2048):
            t_eff = int(round(t_cal * (1 + gam) / (1 - gam)))
            T = 10 * t_cal
            v = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"], T, noise, lsb,
                                         seed=int(noise) * 7919 + t_cal, device=dev)
            row = {"sigma_r": noise, "t_cal": t_cal, "t_eff": t_eff}
            for name, model in (("full", w["model"]), ("single", w["model_single"])):
                p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, input="ci4", voltage_scale=lsb, stream=sc)
                p.configure((0.0, 0.0), model, gam)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for k in range(10):
                    p.image(v[k * t_cal:(k + 1) * t_cal])
                    p.update()
                e1.record(stream)
                e1.synchronize()
                row[f"epical_{name}_sigma_g"] = sig(p.gains())
                row[f"epical_{name}_ms"] = e0.elapsed_time(e1)
                vwin = v[T - t_eff:]
                vis = p.visibilities(vwin)
                ms_x = run(lambda: p.visibilities(vwin, vis), 3)
                gv = torch.ones((C, Na), dtype=torch.complex128, device=dev)
                p.visibility_solve(vis, gv.clone(), max_iter=2000, tol=1e-10)   # forms V^M once
                e0.record(stream)
                it = p.visibility_solve(vis, gv, max_iter=2000, tol=1e-10)
                e1.record(stream)
                e1.synchronize()
                row[f"vis_{name}_sigma_g"] = sig(gv.cpu().numpy())
                row[f"xengine_ms"] = ms_x
                row[f"solve_{name}_ms"] = e0.elapsed_time(e1)
                row[f"solve_{name}_iters_max"] = int(it.max())
                p.close()
            row["epical_over_vis_full"] = row["epical_full_sigma_g"] / row["vis_full_sigma_g"]
            row["epical_over_vis_single"] = row["epical_single_sigma_g"] / row["vis_single_sigma_g"]
            res["rows"].append(row)
            del v
    # algorithmic X-engine work: the Na (Na + 1) / 2 distinct complex products per sample
    last = res["rows"][-1]
    res["xengine_tflops"] = 8.0 * Na * (Na + 1) / 2 * C * last["t_eff"] / (last["xengine_ms"] / 1e3) / 1e12
    return res


def profile_case(name):
    """One untimed workload per name, the target of the ncu captures kept in
    profiles/ (the plan, data and launch shapes of the timed forms)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1603_02126_gb300 import Plan
    if name == "fused_lwa":            # headline interval, fused kernel
        w = synth.workload("lwa")
        d = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"], w["n_time"],
                                     w["noise_power"], w["lsb"], seed=1)
        p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
                 voltage_scale=w["lsb"], path="fused")
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        img = p.image(d)
        p.update()
        p.image(d, img)
        p.update()
    elif name == "tc_compact":         # FP16 tensor-core form, Na=1024 / N=256, 256 samples
        w = synth.workload("compact1024", n_time=256)
        d = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:100], 256,
                                     w["noise_power"], w["lsb"], seed=2)
        p = Plan(w["ant_xy"], w["freqs"], 256, 0.5, support=3, param=0.5, input="ci4",
                 voltage_scale=w["lsb"], path="unfused", precision="fp16", workspace_bytes=4 << 30)
        img = p.image(d)
        p.image(d, img)
    elif name == "unfused_lwa":        # plain unfused path, LWA-like array, 1000 samples
        w = synth.workload("lwa", n_time=1000)
        d = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"], w["n_time"],
                                     w["noise_power"], w["lsb"], seed=1)
        p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
                 voltage_scale=w["lsb"], path="unfused", workspace_bytes=4 << 30)
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        img = p.image(d)
        p.update()
        p.image(d, img)
        p.update()
    elif name in ("grad_lwa", "grad_lwa_bf16"):   # differentiation form, 16 channels, 1024 samples
        from paper_1603_02126_gb300.autograd import EpicImageFn, chi2
        w = synth.workload("lwa_diff", n_time=1024)
        v = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:50], w["n_time"],
                                     w["noise_power"], w["lsb"], seed=4)
        mf = torch.from_numpy(synth.model_frames_c64(w["ant_xy"], w["freqs"], w["model"])).cuda()
        pm = Plan(w["ant_xy"], w["freqs"], 128, 0.5, input="c64")
        M = pm.image(mf) * mf.shape[0]
        p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
                 voltage_scale=w["lsb"])
        if name == "grad_lwa_bf16":
            p.set_adjoint_precision("bf16")
        for _ in range(2):
            g = torch.from_numpy(w["gains"]).cuda().requires_grad_(True)
            chi2(EpicImageFn.apply(g, v, p), M).backward()
    elif name == "cluster_compact":    # cluster path, Na=1024 / N=256, 64 samples
        w = synth.workload("compact1024", n_time=64)
        d = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"][:100], 64,
                                     w["noise_power"], w["lsb"], seed=2)
        p = Plan(w["ant_xy"], w["freqs"], 256, 0.5, support=3, param=0.5, input="ci4",
                 voltage_scale=w["lsb"], path="cluster")
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        img = p.image(d)
        p.update()
        p.image(d, img)
        p.update()
    elif name == "multipix_lwa":       # headline interval with 16 calibration pixels (Sec. 6)
        w = synth.workload("lwa", n_time=2000)
        d = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"], w["n_time"],
                                     w["noise_power"], w["lsb"], seed=1)
        p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, support=3, param=0.5, input="ci4",
                 voltage_scale=w["lsb"], path="fused")
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        p.configure_pixels(w["model"][:16, :2])
        img = p.image(d)
        p.update()
        p.image(d, img)
        p.update()
    elif name == "noise_lwa":          # Sec. 4 comparison path: X-engine and StEFCal, 64 channels
        w = synth.workload("noise")
        lsb = np.full(len(w["freqs"]), np.sqrt((w["sky"][:, 2].sum() + 10.0) / 2) / 2.0)
        v = synth.voltages_ci4_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"], 4096, 10.0, lsb, seed=7)
        p = Plan(w["ant_xy"], w["freqs"], 128, 0.5, input="ci4", voltage_scale=lsb)
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        for _ in range(2):
            vis = p.visibilities(v)
            g = torch.ones((len(w["freqs"]), w["ant_xy"].shape[0]), dtype=torch.complex128, device="cuda")
            p.visibility_solve(vis, g, max_iter=2000, tol=1e-10)
    elif name == "hex_unfused":        # Na=2048 hex, N=512, 128 samples, plain unfused path
        w = synth.workload("hex2048", n_time=128)
        v = synth.voltages_c64_torch(w["ant_xy"], w["freqs"], w["gains"], w["sky"], w["n_time"],
                                     w["noise_power"], seed=3)
        p = Plan(w["ant_xy"], w["freqs"], 512, 0.5, support=3, param=0.5, input="c64",
                 path="unfused", workspace_bytes=2 << 30)
        p.configure((0.0, 0.0), w["model"], w["gamma"])
        img = p.image(v)
        p.update()
        p.image(v, img)
        p.update()
    else:
        raise SystemExit(f"unknown case {name}")
    torch.cuda.synchronize()
    print(json.dumps({"case": name, "ok": True}))


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, bounded samples."""
    if rank != 0:
        return
    w = synth.workload("lwa")
    rng = np.random.default_rng(1)
    import oracle as O
    T = 64
    E = synth.voltages(w["ant_xy"], w["freqs"][:1], w["gains"][:1], w["sky"][:50], T,
                       w["noise_power"], rng)
    b = synth.quantise_ci4(E, w["lsb"][:1])
    oplan = O.Plan(w["ant_xy"], w["freqs"][:1], w["grid_n"], w["cell"], model_lmS=w["model"])
    g = np.ones((1, 256), complex)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        Eint = O.unpack_ci4(b) * w["lsb"][0]
        g, *_ = O.epical_interval(oplan, Eint, g, w["gamma"], with_image=True)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = T / (ms / 1e3)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"channel 0, {T} frames per step"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": f"channel 0, {T} frames per step"},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision / batching / differentiation forms")
    ap.add_argument("--case", default=None,
                    help="run one untimed profiling workload (fused_lwa, tc_compact, unfused_lwa, "
                         "grad_lwa, grad_lwa_bf16, hex_unfused, cluster_compact, multipix_lwa, noise_lwa) and exit")
    ap.add_argument("--n-time", type=int, default=None,
                    help="samples per interval (default: the workload's 10000)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.case:
        profile_case(args.case)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1603_02126_gb300 import Plan

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)     # a real stream: graphs cannot capture the legacy one
    torch.cuda.set_stream(stream)

    w, volt = make_inputs(dev, args.n_time)
    C, Na, N, K, T = len(w["freqs"]), 256, 128, 3, w["n_time"]
    frames = C * T
    plan = Plan(w["ant_xy"], w["freqs"], N, w["cell"], support=K, param=w["kernel_sigma"],
                input="ci4", voltage_scale=w["lsb"], stream=stream.cuda_stream)
    plan.configure((0.0, 0.0), w["model"], w["gamma"])
    image = torch.empty((C, N, N), dtype=torch.float64, device=dev)
    gains_out = torch.empty((C, Na), dtype=torch.complex128, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step():
        plan.image(volt, image)
        plan.update(gains_out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_ms, img_ms, upd_ms = [], [], []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        plan.image(volt, image)
        e1.record(stream)
        plan.update(gains_out)
        e2.record(stream)
        e2.synchronize()
        step_ms.append(e0.elapsed_time(e2))
        img_ms.append(e0.elapsed_time(e1))
        upd_ms.append(e1.elapsed_time(e2))
    torch.cuda.synchronize()
    clk = clocks.stop()
    held = plan.sync()
    total_ms = float(np.sum(step_ms))
    ms_per_step, value, _ = aggregate_ranks(total_ms, frames, args.steps, dist, dev)
    if dist:
        dist.barrier()

    # EPICal increment: the same interval without the correlation
    plain = Plan(w["ant_xy"], w["freqs"], N, w["cell"], support=K, param=w["kernel_sigma"],
                 input="ci4", voltage_scale=w["lsb"], stream=stream.cuda_stream)
    plain.image(volt, image)
    nocal = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1)
        e0, e1 = ev(), ev()
        e0.record(stream)
        plain.image(volt, image)
        e1.record(stream)
        e1.synchronize()
        nocal.append(e0.elapsed_time(e1))

    # end to end through the host-buffer entry point (pinned host memory)
    hv = volt.cpu().pin_memory()
    himg = torch.empty((C, N, N), dtype=torch.float64).pin_memory()
    hg = torch.empty((C, Na), dtype=torch.complex128).pin_memory()
    for _ in range(2):
        plan.image_host(hv, himg)
        plan.update(gains_out)
        hg.copy_(gains_out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.image_host(hv, himg)
        plan.update(gains_out)
        hg.copy_(gains_out, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = frames * world / (float(np.mean(e2e_ms)) / 1e3)

    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    nominal_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
    from paper_1603_02126_gb300.api import measure_fma_peak
    alu_peak = measure_fma_peak(False, stream)
    fp64_peak = measure_fma_peak(True, stream)
    fl = algorithmic_flops_per_frame(Na, N, K) * frames
    img_avg = float(np.mean(img_ms))
    achieved = fl / (img_avg / 1e3) / 1e12
    sha = kernel_sha()
    traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["kernel_sha"] == sha else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_step": frames,
                       "l2": "flushed between timed steps (256 MiB write); voltages 164 MB > L2",
                       "path": "fused FP32 (epic_image + epical_update)",
                       "parallelism": f"{world} GPU(s), channels independent, no collective"},
            "gain_solve_ms": {"update_kernel": float(np.mean(upd_ms)),
                              "epical_increment_in_image": img_avg - float(np.mean(nocal)),
                              "interval_voltages_to_gains": ms_per_step},
            "image_ms_without_epical": float(np.mean(nocal)),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": traffic,
                         "kernel": "epic_image_fused<128,1>",
                         "peak_source": "measured in this run: FP32 FMA microbenchmark "
                                        "(epic_measure_fma_peak, 152 x 8 CTAs x 256 threads, "
                                        "8 independent chains per thread, CUDA events)",
                         "peak_nominal": nominal_peak,
                         "fp64_fma_peak_measured": fp64_peak,
                         "hbm_gbs_of_launch": (volt.numel() + C * N * N * 8 * 3) / (img_avg / 1e3) / 1e9},
            "e2e": {"value": e2e_value, "unit": "frames/s",
                    "h2d_bytes_per_step": int(volt.numel()),
                    "d2h_bytes_per_step": int(C * N * N * 8 + C * Na * 16)},
            "gpu_launches": 2 * args.steps,
            "clocks": clk,
            "held_gains": held,
            "kernel_sha": sha,
        }
        if not args.no_forms and world == 1:
            line["forms"] = forms(torch, Plan, dev, stream, flush, w, volt, args.steps)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(w, volt[:, :1].cpu().numpy())
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
