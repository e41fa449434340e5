#!/usr/bin/env python
"""Benchmark of the projected-EM hot path (E-step + M-step + denoiser) on GB300.

One *step* is one projected-EM iteration (Algorithm 2 with F = 1): E-step over all N
observations x L^2 shifts, M-step, block-DCT projection.  The metric is observation x
shift pairs per second, N * L^2 * steps / device time.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl srmra|reference]
                    [--workload NAME] [--prec fp32|bf16|bf16x3]

Under torchrun (N > 1) every rank runs an independent replica of the workload (its own
seeded instance): the method has no data exchange between independent problems, so
the scaling is weak and the only collective is the timing max/barrier.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "E+M obs x shift pairs/s"
DEFAULT_WORKLOAD = "proj_em_L64_K2_N1e4"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="srmra", choices=["srmra", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", default=None, help="fp32 | bf16 | bf16x3 (default: workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# GB300: 152 SMs x 128 FP32 lanes x 2 flops per FFMA at the maximum SM clock.
FP32_LANES_PER_SM = 128
NUM_SMS = 152


def fp32_peak_tflops(sm_mhz: float) -> float:
    return NUM_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


KERNEL_SOURCE = {"fp32": "k_simt.cu", "bf16": "k_tc.cu", "bf16x3": "k_tc.cu"}


def traffic_from_profiles(kernel: str, workload: str, prec: str):
    """DRAM bytes per launch recorded from an ncu capture in profiles/traffic.txt, or
    None.  Lines: `traffic <kernel> <workload> <bytes_per_launch> <source sha1 prefix>`;
    a line counts only while the kernel's source file still has that hash."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_2204_04754_gb300", "csrc", KERNEL_SOURCE[prec])
    if not os.path.exists(path) or not os.path.exists(src):
        return None
    with open(src, "rb") as f:
        digest = hashlib.sha1(f.read()).hexdigest()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 5 and parts[0] == "traffic" and parts[1] == kernel \
                    and parts[2] == workload and digest.startswith(parts[4]):
                return float(parts[3])
    return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = []
        smax = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(problem, budget_s: float, n_sub: int | None = None):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload: one EM
    iteration over the first n_sub observations, repeated for ~budget_s seconds."""
    import numpy as np
    from oracle import srmra_oracle as O
    p = problem
    if n_sub is None:
        n_sub = 256
        t0 = time.perf_counter()
        O.em_iter(p.y[:n_sub], p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
        dt = time.perf_counter() - t0
        n_sub = int(max(64, min(p.N, n_sub * (budget_s / 4.0) / max(dt, 1e-3))))
    reps = 0
    t0 = time.perf_counter()
    while True:
        O.em_iter(p.y[:n_sub], p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 50:
            break
    pairs = n_sub * p.L * p.L * reps
    _ = np
    return {"value": pairs / el, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} dense FP64 oracle EM iteration(s) over the first {n_sub} of "
                      f"{p.N} observations (all {p.L * p.L} shifts), {el:.1f} s",
            "n_sub": n_sub}


def run_reference(args, rank):
    from paper_2204_04754_gb300 import synth
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    p = synth.workload_problem(args.workload)
    cal = cpu_oracle_rate(p, 3.0)
    n_sub = cal["n_sub"]
    from oracle import srmra_oracle as O
    x, r1, r2 = p.x0, p.rho1_0, p.rho2_0
    for _ in range(args.warmup):
        O.em_iter(p.y[:n_sub], x, r1, r2, p.sigma, p.K)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xn, r1n, r2n, _, _ = O.em_iter(p.y[:n_sub], x, r1, r2, p.sigma, p.K)
        if w["F"]:
            xn, _ = O.dct_denoise(xn, 1.0)
    el = time.perf_counter() - t0
    value = n_sub * p.L * p.L * args.steps / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "L_high": p.L, "K": p.K, "N": p.N,
                      "sigma": p.sigma, "F": w["F"], "sample_observations": n_sub},
           "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": os.cpu_count(),
                            "kind": "oracle",
                            "sample": f"each step: one dense FP64 oracle projected-EM "
                                      f"iteration over the first {n_sub} of {p.N} "
                                      f"observations"},
           "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    from paper_2204_04754_gb300 import srmra, synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = synth.WORKLOADS[args.workload]
    prec = args.prec or "fp32"
    p = synth.workload_problem(args.workload, instance=rank)
    F = w["F"]
    stream = torch.cuda.current_stream()
    y = torch.from_numpy(p.y).cuda()
    s = srmra.Solver(p.L, p.K, p.sigma, y, prec=prec, x0=p.x0, rho1=p.rho1_0,
                     rho2=p.rho2_0, stream=stream.cuda_stream)
    del y
    # warm-up (starts Algorithm 2's sigma_BM schedule at 1)
    s.solve(args.warmup, F, sigma_bm1=1.0, loglik=False)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    s.profile(True)
    s.profile_read()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = s.launches
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit()
                          else local)
    clocks.start()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.solve(1, F, sigma_bm1=0.0, loglik=False)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = s.launches - launches0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = float(sum(step_ms))
    phase_ms, phase_n = s.profile_read()
    s.profile(False)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()

    pairs_per_step = p.N * p.L * p.L
    value = world * pairs_per_step * args.steps / (total_ms / 1e3)

    # roofline of the dominant kernel (phase), from the live CUDA events
    peaks, peak_src = load_peaks()
    dom = max(("pass1", "pass2"), key=lambda k: phase_ms[k])
    per_pair_flops = {"pass1": 2 * p.l * p.l, "pass2": 4 * p.l * p.l}[dom]
    avg_launch_s = phase_ms[dom] / max(1, phase_n[dom]) / 1e3
    achieved = per_pair_flops * pairs_per_step / avg_launch_s / 1e12
    if prec == "fp32":
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak = fp32_peak_tflops(sm_max)
        bound = "alu"
        peak_note = (f"FP32 FFMA peak derived: {NUM_SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 "
                     f"flops x {sm_max:.0f} MHz (max SM clock, {peak_src} peaks file)")
    else:
        peak = float(peaks["bf16_tflops_sustained"])
        bound = "tensor"
        peak_note = f"dense bf16, sustained, of {peak_src}"
    kern = {"pass1": f"k_p1_{prec}", "pass2": f"k_p2_{prec}"}[dom]
    roof = {"bound": bound, "kernel": kern, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic_from_profiles(kern, args.workload, prec),
            "algorithmic_flops_per_launch": per_pair_flops * pairs_per_step,
            "avg_launch_ms": avg_launch_s * 1e3, "peak_source": peak_note}

    out = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3"}[prec],
           "data": "synthetic (seeded blob image, mixture shift distributions, Gaussian noise)",
           "config": {"workload": args.workload, "L_high": p.L, "K": p.K, "L_low": p.l,
                      "N": p.N, "sigma": p.sigma, "F": F, "precision": prec,
                      "step": "one projected-EM iteration (E-step, M-step, DCT projection)",
                      "l2": "256 MiB buffer zeroed before every timed step",
                      "parallelism": f"{world} independent replica(s)"},
           "roofline": roof, "gpu_launches": launches,
           "phases_ms_per_step": {k: v / args.steps for k, v in phase_ms.items()},
           "clocks": clk}

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_run(p, prec, w, srmra, torch)
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_oracle_rate(p, args.cpu_seconds)
        cb.pop("n_sub", None)
        out["cpu_baseline"] = cb
    s.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def e2e_run(p, prec, w, srmra, torch):
    """End to end through the public API with pinned host buffers: create (uploads y),
    a full solve of the workload's iteration count with the log-likelihood read back
    every iteration, read the final state, destroy."""
    import numpy as np
    iters = int(w["iters"])
    yh = torch.from_numpy(p.y).pin_memory()

    def once():
        t0 = time.perf_counter()
        s = srmra.Solver(p.L, p.K, p.sigma, yh, prec=prec, x0=p.x0, rho1=p.rho1_0,
                         rho2=p.rho2_0, y_on_device=False)
        ll = s.solve(iters, w["F"], loglik=True)
        x, r1, r2, _, _ = s.state()
        s.close()
        return time.perf_counter() - t0, ll

    once()  # warm
    el, ll = once()
    h2d = p.y.nbytes + p.x0.nbytes + 16 * p.L
    d2h = 8 * iters + 4 * p.L * p.L + 16 * p.L
    _ = np
    return {"value": p.N * p.L * p.L * iters / el, "unit": "pairs/s",
            "h2d_bytes_per_step": h2d / iters, "d2h_bytes_per_step": d2h / iters,
            "step": f"one solve of {iters} iterations per upload; per-step bytes are "
                    f"per-iteration averages", "seconds": el}


if __name__ == "__main__":
    main()
