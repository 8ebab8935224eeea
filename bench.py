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
# on this workload, with the sha256 (first 12 hex) of the kernel source it
# was taken at; ignored when the kernel source has changed since.
TRAFFIC = {"kernel_sha": "c8dfb121f750", "bytes_per_launch": 183435520}


def kernel_sha() -> str:
    p = os.path.join(ROOT, "paper_1603_02126_gb300", "csrc", "epic_kernels.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:12]


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
    ap.add_argument("--n-time", type=int, default=None,
                    help="samples per interval (default: the workload's 10000)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
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
    stream = torch.cuda.current_stream()

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
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = frames * world / (ms_per_step / 1e3)

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
    alu_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
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
                         "peak_source": f"derived: {NUM_SMS} SMs x {FP32_LANES_PER_SM} FP32 "
                                        f"lanes x 2 x {sm_max:.0f} MHz ({pk_kind} max clock)",
                         "hbm_gbs_of_launch": (volt.numel() + C * N * N * 8 * 3) / (img_avg / 1e3) / 1e9},
            "e2e": {"value": e2e_value, "unit": "frames/s",
                    "h2d_bytes_per_step": int(volt.numel()),
                    "d2h_bytes_per_step": int(C * N * N * 8 + C * Na * 16)},
            "gpu_launches": 2 * args.steps,
            "clocks": clk,
            "held_gains": held,
            "kernel_sha": sha,
        }
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(w, volt[:, :1].cpu().numpy())
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
