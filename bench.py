#!/usr/bin/env python
"""Benchmark of the projected-EM hot path (E-step + M-step + denoiser) on GB300.

One *step* is one projected-EM iteration (Algorithm 2 with F = 1): E-step over all N
observations x L^2 shifts, M-step, block-DCT projection.  The metric is observation x
shift pairs per second, N * L^2 * steps / device time.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl srmra|reference]
                    [--workload NAME] [--prec fp32|bf16|bf16x3|fft32]
    python bench.py --study precision [--study-iters 40]   (per-iteration errors)

The default workload is the largest single-GPU one: L = 96, K = 3 (l = 32), N = 5e4,
sigma = 0.2, timed in the float32 form.  Beside the headline the line carries, for the
same workload, the tensor-core forms (bf16x3, bf16) with their speedup over float32
and their error against the FP64 oracle after one iteration from a common state; the
same for sigma = 1.0; the projected-EM workload L = 64, K = 2, N = 1e4; 64 uneven
problems in grouped launches; and a short serving trace.

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
DEFAULT_WORKLOAD = "precision_L96_K3_N5e4_s0.2"
# the second noise level of the precision workload, reported beside the first
COMPANION = {"precision_L96_K3_N5e4_s0.2": "precision_L96_K3_N5e4_s1.0"}
SECONDARY = "proj_em_L64_K2_N1e4"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="srmra", choices=["srmra", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", default=None, help="fp32 | bf16 | bf16x3 | fft32 (default: workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--requests", type=int, default=12, help="serve: trace length")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-pool", type=int, default=16,
                    help="serve: distinct seeded problems the requests draw from")
    ap.add_argument("--rates", default=None,
                    help="serve: comma-separated arrival rates per second (a sweep)")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the blocks beside the headline (other forms, workloads)")
    ap.add_argument("--no-extra", action="store_true",
                    help="keep the other forms of the workload, skip the other workloads")
    ap.add_argument("--oracle-threads", type=int, default=0,
                    help="threads of the FFT oracle error checks (0 = all host cores)")
    ap.add_argument("--study", default=None, choices=[None, "precision"],
                    help="precision: per-iteration one-step errors of every form against "
                         "the FP64 oracle over a projected run")
    ap.add_argument("--flags", type=int, default=0,
                    help="context flags of the timed forms (srmra.SRMRA_FLAG_*; e.g. 32 asks "
                         "for the pair form of the tensor-core pass 2)")
    ap.add_argument("--n-obs", type=int, default=None,
                    help="fewer observations than the workload's (small profiling runs)")
    ap.add_argument("--study-iters", type=int, default=40)
    ap.add_argument("--study-forms", default="fp32,bf16x3,bf16",
                    help="forms of the study (bf16x3-comp: the compensated M-step forced)")
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


KERNEL_SOURCE = {"fp32": "k_simt.cu", "bf16": "k_tc.cu", "bf16x3": "k_tc.cu", "fft32": "k_fft.cu"}


def profile_record(field: str, kernel: str, workload: str, prec: str):
    """A per-launch figure recorded from an ncu capture in profiles/traffic.txt, or None.
    Lines: `<field> <kernel> <workload> <value> <source sha1 prefix>`, field `traffic`
    (DRAM bytes per launch) or `tensor` (sm__pipe_tensor_cycles_active, fraction of
    elapsed cycles); a line counts only while the kernel's source file still has that
    hash."""
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
            if len(parts) == 5 and parts[0] == field and parts[1] == kernel \
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


def gpu_index(local: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    return int(vis) if vis.isdigit() else local


def cpu_oracle_rate(problem, budget_s: float, n_sub: int | None = None):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload: one EM
    iteration over the first n_sub observations, repeated for ~budget_s seconds."""
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
    return {"value": pairs / el, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} dense FP64 oracle EM iteration(s) over the first {n_sub} of "
                      f"{p.N} observations (all {p.L * p.L} shifts), {el:.1f} s",
            "n_sub": n_sub}


def run_reference(args, rank):
    from paper_2204_04754_gb300 import synth
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    if args.workload in ("batched_64", "serve"):
        sp = synth.batched_instances(1)[0] if args.workload == "batched_64" else \
            dict(L=96, K=2, N=10_000, sigma=0.5, seed=synth.seed_for(5, 0))
        p = synth.make_problem(sp["L"], sp["K"], sp["N"], sp["sigma"], sp["seed"])
    else:
        p = synth.workload_problem(args.workload)
    # each step a sample of about 2 s of oracle work (per-call fixed costs, such as
    # building the L^2 templates, are then a small part of it)
    cal = cpu_oracle_rate(p, 8.0)
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


def reduce_max(value: float, dist, device) -> float:
    """Maximum of `value` over all ranks (the job's time is its slowest rank's)."""
    import torch
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job units per second: every rank processes its own replica (weak scaling)."""
    return world * units_per_rank_step * steps / (max_ms / 1e3)


def time_steps(run_step, steps, stream, torch, flush):
    """Device time (ms) of each step, L2 flushed before every step (outside the events)."""
    evs = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


# ------------------------------------------------------------------- work accounting

def padded(p):
    """Padded sizes the kernels execute over: (Npad, Spad, ldk, pixel chunks)."""
    l2 = p.l * p.l
    return (-(-p.N // 128) * 128, -(-(p.L * p.L) // 256) * 256, -(-l2 // 64) * 64,
            -(-l2 // 256))


def kernel_names(prec: str, plan: dict, l: int):
    """The pass-1 and pass-2 kernels as they are launched."""
    if prec == "fp32":
        return "k_p1_f32", "k_p2_f32"
    if prec == "fft32":
        return f"k_fft_p1<{l}>", f"k_fft_p2<{l}>"
    n = 3 if prec == "bf16x3" else 1
    p2 = {"per_chunk": f"k_p2_tc<{n},false>", "per_chunk_comp": f"k_p2_tc<{n},true>",
          "ring": f"k_p2c_tc<{n}>", "interleaved": f"k_p2i_tc<{n}>",
          "pair": f"k_p2p_tc<{n}>"}[plan["p2_form"]]
    return f"k_p1_tc<{n},{plan.get('p1_shift_tile', 256)}>", p2


def tc_executed_flops(p, prec: str, plan: dict):
    """Tensor-core flops the two passes issue per launch (padding included): pass 1 NPROD
    MMAs per logit tile; pass 2 the same logits once per chunk group plus the fp16 M-step
    product Z' = W^T Y' over every 256-pixel chunk (three products with the compensated
    M-step)."""
    nprod = 3 if prec == "bf16x3" else 1
    nz = 3 if plan["p2_form"] == "per_chunk_comp" else 1
    Npad, Spad, ldk, nch = padded(p)
    p1 = nprod * 2.0 * Npad * Spad * ldk
    p2 = (nprod * 2.0 * Spad * Npad * ldk * plan["p2_chunk_groups"] +
          nz * 2.0 * Spad * Npad * nch * 256)
    return p1, p2


def roofline_of(p, prec: str, plan: dict, workload: str, phase_ms: dict, phase_n: dict):
    """Roofline of the dominant pass: algorithmic flops (Sec. 2 E- and M-step: 2 l^2 per
    pair for the logits of pass 1; 4 l^2 for pass 2, the logit recompute plus the M-step
    sum) over its average CUDA-event launch time, against the FP32 FFMA peak (float32 and
    FFT forms) or the sustained bf16 tensor peak (tensor-core forms).  Tensor-core forms
    add the executed tensor flops (padding and recompute included) of each pass and of
    the two passes together, time-weighted."""
    peaks, src = load_peaks()
    dom = max(("pass1", "pass2"), key=lambda k: phase_ms[k])
    l2 = p.l * p.l
    pairs = p.N * p.L * p.L
    if prec == "fft32":
        lg = math.log2(l2)
        per_pair = {"pass1": 5 * lg + 6, "pass2": 10 * lg + 14}[dom]
    else:
        per_pair = {"pass1": 2 * l2, "pass2": 4 * l2}[dom]
    t_ms = {k: phase_ms[k] / max(1, phase_n[k]) for k in ("pass1", "pass2")}
    k1, k2 = kernel_names(prec, plan, p.l)
    kern = {"pass1": k1, "pass2": k2}[dom]
    achieved = per_pair * pairs / (t_ms[dom] / 1e3) / 1e12
    if prec in ("fp32", "fft32"):
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak = fp32_peak_tflops(sm_max)
        bound = "alu"
        note = (f"FP32 FFMA peak derived: {NUM_SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 "
                f"flops x {sm_max:.0f} MHz (max SM clock, {src} peaks file)")
    else:
        peak = float(peaks["bf16_tflops_sustained"])
        bound = "tensor"
        note = f"dense bf16, sustained, of {src}"
    traffic = profile_record("traffic", kern, workload, prec)
    roof = {"bound": bound, "kernel": kern, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "algorithmic_flops_per_launch": per_pair * pairs, "avg_launch_ms": t_ms[dom],
            "peak_source": note}
    if traffic:
        hbm = float(peaks["hbm_gbs"])
        roof["dram_gbs"] = traffic / (t_ms[dom] / 1e3) / 1e9
        roof["dram_frac_of_hbm_peak"] = roof["dram_gbs"] / hbm
    if bound == "tensor":
        e1, e2 = tc_executed_flops(p, prec, plan)
        ex = {"pass1": e1, "pass2": e2}
        roof["executed_flops_per_launch"] = ex[dom]
        roof["executed_tflops"] = ex[dom] / (t_ms[dom] / 1e3) / 1e12
        roof["executed_frac"] = roof["executed_tflops"] / peak
        both = t_ms["pass1"] + t_ms["pass2"]
        roof["passes"] = {
            "pass1": {"kernel": k1, "ms": t_ms["pass1"],
                      "executed_frac": e1 / (t_ms["pass1"] / 1e3) / 1e12 / peak,
                      "algorithmic_frac": 2 * l2 * pairs / (t_ms["pass1"] / 1e3) / 1e12 / peak},
            "pass2": {"kernel": k2, "ms": t_ms["pass2"],
                      "executed_frac": e2 / (t_ms["pass2"] / 1e3) / 1e12 / peak,
                      "algorithmic_frac": 4 * l2 * pairs / (t_ms["pass2"] / 1e3) / 1e12 / peak},
            "both_time_weighted": {"ms": both,
                                   "executed_frac": (e1 + e2) / (both / 1e3) / 1e12 / peak,
                                   "algorithmic_frac": 4 * l2 * pairs / (both / 1e3) / 1e12 / peak}}
        tp = profile_record("tensor", kern, workload, prec)
        if tp is not None:
            roof["ncu_tensor_pipe_active"] = tp
        roof["algorithmic_frac_of_burst_peak"] = achieved / float(peaks["bf16_tflops"])
    return roof


# ------------------------------------------------------------------- one form, timed

class FormRun:
    """One precision form of a workload on the GPU: a context created from device-
    resident observations, warmed up (Algorithm 2's sigma_BM schedule started at 1), then
    `steps` projected-EM iterations timed with CUDA events (L2 flushed before each)."""

    def __init__(self, p, w, workload, prec, steps, warmup, srmra, torch, stream, flush,
                 clocks=False, local=0, barrier=None, flags=0):
        self.p, self.prec = p, prec
        y = torch.from_numpy(p.y).cuda()
        self.s = srmra.Solver(p.L, p.K, p.sigma, y, prec=prec, x0=p.x0, rho1=p.rho1_0,
                              rho2=p.rho2_0, stream=stream.cuda_stream, flags=flags)
        del y
        F = w["F"]
        self.s.solve(warmup, F, sigma_bm1=1.0, loglik=False)
        self.s.profile(True)
        self.s.profile_read()
        torch.cuda.synchronize()
        if barrier:  # all ranks start the timed steps together
            barrier()
        l0 = self.s.launches
        cs = ClockSampler(gpu_index(local)) if clocks else None
        if cs:
            cs.start()
        self.step_ms = time_steps(lambda: self.s.solve(1, F, sigma_bm1=0.0, loglik=False),
                                  steps, stream, torch, flush)  # synchronises at the end
        if barrier:
            barrier()
        self.clocks = cs.stop() if cs else None
        self.launches = self.s.launches - l0
        ms, n = self.s.profile_read()
        self.s.profile(False)
        self.phase_ms = {k: float(v) for k, v in ms.items()}
        self.phase_n = {k: int(v) for k, v in n.items()}
        self.steps = steps
        self.total_ms = float(sum(self.step_ms))
        self.value = p.N * p.L * p.L * steps / (self.total_ms / 1e3)
        self.plan = self.s.plan()
        self.roof = roofline_of(p, prec, self.plan, workload, self.phase_ms, self.phase_n)

    def summary(self, fp32_value=None):
        d = {"precision": self.prec, "value": self.value, "unit": "pairs/s",
             "ms_per_step": self.total_ms / self.steps,
             "phases_ms_per_step": {k: v / self.steps for k, v in self.phase_ms.items()},
             "plan": self.plan, "roofline": self.roof, "gpu_launches": self.launches}
        if fp32_value:
            d["speedup_vs_fp32"] = self.value / fp32_value
        return d

    def close(self):
        self.s.close()


def rel(a, b):
    import numpy as np
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def errors_vs_oracle(p, runs, threads):
    """One EM iteration of every form from one common state (the first run's current
    estimate), each compared with the FP64 FFT oracle's iteration from the same state:
    relative 2-norm errors of x, rho1, rho2, |dLL| / |LL|, and the largest |d lse_i| /
    |lse_i| (and the same over ||y_i||^2 / (2 sigma^2) + |lse_i| + 1, the scale of the
    terms that cancel in lse_i)."""
    import numpy as np
    from oracle import fft_oracle as FO
    x, r1, r2, sbm, t = runs[0].s.state()
    t0 = time.perf_counter()
    xo, r1o, r2o, llo, aux = FO.em_iter_fft(p.y, x, r1, r2, p.sigma, p.K, workers=threads)
    oracle_s = time.perf_counter() - t0
    yscale = (p.y.astype(np.float64) ** 2).sum(axis=(1, 2)) / (2 * p.sigma ** 2)
    out = {}
    for r in runs:
        r.s.set_state(x, r1, r2, sbm, t)
        ll = r.s.em_iter(1)[0]
        lse, _ = r.s.estep()
        xg, r1g, r2g, _, _ = r.s.state()
        out[r.prec] = {
            "x": rel(xg, xo), "rho1": rel(r1g, r1o), "rho2": rel(r2g, r2o),
            "LL": abs(ll - llo) / abs(llo),
            "lse_max_rel": float(np.max(np.abs(lse - aux["lse"]) / np.abs(aux["lse"]))),
            "lse_max_scaled": float(np.max(np.abs(lse - aux["lse"]) /
                                           (1.0 + np.abs(aux["lse"]) + yscale)))}
    return out, {"oracle": "FP64 polyphase-FFT oracle (pinned to the dense definition), all "
                           f"{p.N} observations, {threads} threads, {oracle_s:.1f} s",
                 "state": f"the float32 run's estimate after its timed iterations (t = {t})"}


def workload_block(name, steps, warmup, srmra, torch, stream, flush, threads, local=0,
                   forms=("fp32", "bf16x3", "bf16"), clocks=False):
    """Every form of one workload: timed runs, and errors against the oracle."""
    from paper_2204_04754_gb300 import synth
    w = synth.WORKLOADS[name]
    p = synth.workload_problem(name)
    runs = [FormRun(p, w, name, f, steps, warmup, srmra, torch, stream, flush,
                    clocks=(clocks and f == forms[0]), local=local) for f in forms]
    err, how = errors_vs_oracle(p, runs, threads)
    base = runs[0].value
    block = {"workload": name, "L_high": p.L, "K": p.K, "N": p.N, "sigma": p.sigma,
             "forms": {}, "error_vs_oracle": how}
    for r in runs:
        d = r.summary(None if r.prec == forms[0] else base)
        d["error_vs_oracle"] = err[r.prec]
        if r.prec != "fp32":
            worst = max(err[r.prec][k] for k in ("x", "rho1", "rho2", "LL"))
            d["rel_err_max"] = worst
            d["within_1e-4"] = bool(worst <= 1e-4)
        block["forms"][r.prec] = d
    return p, w, runs, block


# ------------------------------------------------------------------- other blocks

def online_block(p, w, steps, warmup, srmra, torch, stream, flush, fp32_value, n_shards=10):
    """Online (mini-batch) EM on the same workload: the observations split into n_shards
    device-resident shards, one shard per step (cyclic), gamma_t = (t + 1)^-0.6; pairs/s
    of the steps (shard observations x L^2 shifts per step)."""
    cuts = [p.N * k // n_shards for k in range(n_shards + 1)]
    shards = [srmra.Solver(p.L, p.K, p.sigma, p.y[a:b], prec="fp32", x0=p.x0, rho1=p.rho1_0,
                           rho2=p.rho2_0, stream=stream.cuda_stream)
              for a, b in zip(cuts[:-1], cuts[1:])]
    on = srmra.Online(shards)
    t = [0]

    def one():
        on.step(t[0] % n_shards, (t[0] + 1) ** -0.6, loglik=False)
        t[0] += 1
    for _ in range(warmup):
        one()
    ms = time_steps(one, steps, stream, torch, flush)
    pairs = sum(b - a for a, b in zip(cuts[:-1], cuts[1:])) / n_shards * p.L * p.L
    value = pairs * steps / (sum(ms) / 1e3)
    on.close()
    for s_ in shards:
        s_.close()
    return {"shards": n_shards, "obs_per_step": p.N // n_shards, "value": value,
            "unit": "pairs/s", "ms_per_step": sum(ms) / steps,
            "per_pair_vs_full_iteration": value / fp32_value,
            "note": "mini-batch EM with stochastic-approximation statistics (fp32 form); "
                    "steps checked against the oracle in tests/test_gpu_online.py"}


def mom_block(p, steps, warmup, srmra, torch, stream, flush, sm_max):
    """Projected MoM (Algorithm 1) on the same observations: the one-pass empirical
    moments and the projected gradient iterations, against the FP32 FFMA peak.  Flops
    counted are the algorithmic ones of the products: M2^ = Y^T Y / N is symmetric, so
    N l^2 (l^2 + 1) (one multiply-add per unique entry and observation); per iteration
    the symmetric T^T diag(rho) T, L^2 l^2 (l^2 + 1), plus T R, 2 L^2 l^4."""
    import numpy as np
    s = srmra.Solver(p.L, p.K, p.sigma, p.y, prec="fp32", x0=p.x0, rho1=p.rho1_0,
                     rho2=p.rho2_0, stream=stream.cuda_stream)
    m = srmra.Mom(s)
    for _ in range(warmup):
        m.recompute_moments()
    ms_mom = time_steps(m.recompute_moments, steps, stream, torch, flush)
    _, gx, g1, g2 = m.eval()
    mu_x = 0.003 / float(np.abs(gx).max())
    mu_r = 0.003 / float(max(np.abs(g1).max(), np.abs(g2).max()))
    m.run(warmup, 0, mu_x, mu_r, objective=False)
    fs = []
    ms_it = time_steps(lambda: fs.append(m.run(1, 0, mu_x, mu_r)), steps, stream, torch, flush)
    l2 = float(p.l) ** 2
    peak = fp32_peak_tflops(sm_max)
    mom_tf = p.N * l2 * (l2 + 1) / (float(np.mean(ms_mom)) / 1e3) / 1e12
    it_tf = p.L * p.L * l2 * (3 * l2 + 1) / (float(np.mean(ms_it)) / 1e3) / 1e12
    m.close()
    s.close()
    return {"moments_ms": float(np.mean(ms_mom)), "moments_tflops": mom_tf,
            "moments_frac_fp32_peak": mom_tf / peak,
            "iteration_ms": float(np.mean(ms_it)), "iteration_tflops": it_tf,
            "iteration_frac_fp32_peak": it_tf / peak,
            "objective_first_last": [float(fs[0][0]), float(fs[-1][0])],
            "note": "float32 SIMT products (k_mom_gemm); each timed iteration includes its "
                    "host synchronisation; checked against the oracle in "
                    "tests/test_gpu_mom.py"}


def secondary_block(steps, warmup, srmra, torch, stream, flush, threads):
    """The projected-EM workload L = 64, K = 2, N = 1e4, sigma = 0.3 (F = 1): the float32,
    bf16x3 and polyphase-FFT forms with errors against the oracle, online EM and
    projected MoM on the same observations."""
    p, w, runs, block = workload_block(SECONDARY, steps, warmup, srmra, torch, stream, flush,
                                       threads, forms=("fp32", "bf16x3", "fft32"))
    fp32_value = runs[0].value
    for r in runs:
        r.close()
    block["online"] = online_block(p, w, steps, warmup, srmra, torch, stream, flush,
                                   fp32_value)
    block["mom"] = mom_block(p, steps, warmup, srmra, torch, stream, flush,
                             float(load_peaks()[0].get("sm_max_mhz", 2070.0)))
    return block


def batched_block(steps, warmup, rank, prec, srmra, synth, torch, stream, flush, count=64,
                  clocks=None):
    """`count` uneven problems (L in {32,48,64,96}, K in {2,4}, N ~ U[1e3, 2e4], sigma ~
    U[0.1, 1]) advanced together: grouped persistent launches replayed as a CUDA graph,
    decomposition and tile shape picked by the autotuner."""
    specs = synth.batched_instances(count, seed=synth.seed_for(4) + 1000 * rank)
    t0 = time.perf_counter()
    probs = [synth.make_problem(sp["L"], sp["K"], sp["N"], sp["sigma"], sp["seed"])
             for sp in specs]
    gen_s = time.perf_counter() - t0
    solvers = [srmra.Solver(p.L, p.K, p.sigma, p.y, prec=prec, x0=p.x0, rho1=p.rho1_0,
                            rho2=p.rho2_0, stream=stream.cuda_stream) for p in probs]
    t0 = time.perf_counter()
    batch = srmra.Batch(solvers, autotune=True)
    tune_s = time.perf_counter() - t0
    batch.solve(warmup, 1, sigma_bm1=1.0)
    l0 = sum(s.launches for s in solvers)
    if clocks:
        clocks.start()
    ms = time_steps(lambda: batch.solve(1, 1, sigma_bm1=0.0), steps, stream, torch, flush)
    clk = clocks.stop() if clocks else None
    launches = sum(s.launches for s in solvers) - l0
    # per-pass device times: one more iteration enqueued without the graph (events
    # recorded inside a captured graph cannot be timed)
    probe = srmra.Batch(solvers, autotune=False, graph=False)
    probe.solve(1, 1, sigma_bm1=0.0)
    p1_ms, p2_ms = probe.pass_ms()
    probe.close()
    total_ms = float(sum(ms))
    pairs = sum(p.N * p.L * p.L for p in probs)
    alg2 = sum(4 * p.l * p.l * p.N * p.L * p.L for p in probs)
    peaks, peak_src = load_peaks()
    peak = float(peaks["bf16_tflops_sustained"])
    achieved = alg2 / (p2_ms / 1e3) / 1e12
    d = {"value": pairs * steps / (total_ms / 1e3), "unit": "pairs/s",
         "ms_per_step": total_ms / steps, "steps": steps, "warmup": warmup,
         "problems": len(probs), "L_high": sorted({p.L for p in probs}),
         "K": sorted({p.K for p in probs}), "N_total": int(sum(p.N for p in probs)),
         "precision": prec,
         "step": "one projected-EM iteration (F = 1) of all problems (grouped launches, "
                 "CUDA graph replay)",
         "autotuner": batch.tuning(), "autotune_seconds": tune_s,
         "data_generation_s": gen_s,
         "roofline": {"bound": "tensor", "kernel": f"grouped pass 2 ({prec})",
                      "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                      "frac": achieved / peak, "traffic": None,
                      "algorithmic_flops_per_launch": alg2, "avg_launch_ms": p2_ms,
                      "peak_source": f"dense bf16, sustained, of {peak_src}"},
         "phases_ms_last_step": {"pass1_grouped": p1_ms, "pass2_grouped": p2_ms},
         "gpu_launches": launches, "clocks": clk}
    batch.close()
    for s_ in solvers:
        s_.close()
    return d


def run_batched(args, rank, world, local):
    """The batched workload as the bench line."""
    import torch
    from paper_2204_04754_gb300 import srmra, synth
    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload]
    prec = args.prec or w["prec"]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    d = batched_block(args.steps, args.warmup, rank, prec, srmra, synth, torch, stream, flush,
                      count=w["count"], clocks=ClockSampler(gpu_index(local)))
    out = {"metric": METRIC, "value": world * d["value"], "unit": "pairs/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": d["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
           "data": "synthetic (64 seeded problems)",
           "config": {"workload": args.workload, "problems": d["problems"],
                      "L_high": d["L_high"], "K": d["K"], "N_total": d["N_total"], "F": 1,
                      "step": d["step"], "l2": "256 MiB buffer zeroed before every timed step",
                      "autotuner": d["autotuner"], "autotune_seconds": d["autotune_seconds"],
                      "parallelism": f"{world} independent replica(s)"},
           "roofline": d["roofline"], "phases_ms_last_step": d["phases_ms_last_step"],
           "gpu_launches": d["gpu_launches"], "clocks": d["clocks"]}
    if rank == 0:
        print(json.dumps(out), flush=True)


def serve_trace(srmra, srv, probs, arrivals, iters, F):
    """Submit probs[k] at arrivals[k] (seconds from the start) and step the server until
    every request has finished.  Returns (latencies in ms, makespan s, server steps);
    latency = completion - planned arrival (queueing included)."""
    import numpy as np
    n = len(probs)
    ids = {}
    done = {}
    pending = list(range(n))
    steps = 0
    start = time.perf_counter()
    while len(done) < n:
        now = time.perf_counter() - start
        while pending and arrivals[pending[0]] <= now:
            k = pending.pop(0)
            p = probs[k]
            ids[k] = srv.submit(p.L, p.K, p.sigma, p.y, iters, F=F)
        running, queued, finished = srv.step()
        steps += 1
        if finished:
            tnow = time.perf_counter() - start
            for k, rid in ids.items():
                if k not in done and srv.result(rid, probs[k].L)["state"] == 2:
                    done[k] = tnow
        if running == 0 and queued == 0 and pending:
            wait = arrivals[pending[0]] - (time.perf_counter() - start)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    makespan = time.perf_counter() - start
    lat = np.array([1e3 * (done[k] - arrivals[k]) for k in range(n)])
    return lat, makespan, steps


def serve_block(requests, rates, pool_size, slots, budget_gb, prec, srmra, synth, torch,
                stream, iters=30, F=1, clocks=None):
    """Poisson arrivals of projected-EM solve requests (L in {64,96,128}, K in {2,4},
    N in {1e4, 5e4, 1e5}, sigma ~ U[0.2, 1], 30 projected iterations) served with
    continuous batching.  Latency = completion - planned arrival (queueing included).
    The requests draw their data from a pool of `pool_size` distinct seeded problems
    (request k uses pool entry k mod pool size), so that long traces fit in host memory;
    several rates run the same trace at each (a sweep that shows where the offered load
    exceeds capacity)."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(synth.seed_for(5)))
    n = requests
    unit_gaps = rng.exponential(1.0, size=n)  # arrivals at rate r: cumsum(unit_gaps) / r
    pool = min(n, pool_size)
    specs = []
    for k in range(pool):
        L = int(rng.choice([64, 96, 128]))
        K = int(rng.choice([2, 4]))
        N = int(rng.choice([10_000, 50_000, 100_000]))
        sigma = float(rng.uniform(0.2, 1.0))
        specs.append((L, K, N, sigma))
    t0 = time.perf_counter()
    pool_probs = [synth.make_problem(L, K, N, sg, seed=synth.seed_for(5, k))
                  for k, (L, K, N, sg) in enumerate(specs)]
    probs = [pool_probs[k % pool] for k in range(n)]
    gen_s = time.perf_counter() - t0
    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.8, budget_gb * 2 ** 30))
    srv = srmra.Server(budget, max_active=slots, prec=prec, stream=stream.cuda_stream)
    # warm the kernels and graph machinery on tiny requests (not part of the trace; with
    # "auto" one of each form)
    warm = [(64, 4)] + ([(48, 2)] if prec == "auto" else [])
    wps = [synth.make_problem(L, K, 2000, 0.5, seed=synth.seed_for(5, 999)) for L, K in warm]
    wids = [srv.submit(wp.L, wp.K, wp.sigma, wp.y, 2, F=F) for wp in wps]
    while srv.step()[0] > 0:
        pass
    for wp, wid in zip(wps, wids):
        srv.result(wid, wp.L)
    pairs = sum(p.N * p.L * p.L * iters for p in probs)
    sweep = []
    if clocks:
        clocks.start()
    for rate in rates:
        arrivals = np.cumsum(unit_gaps) / rate
        lat, makespan, steps = serve_trace(srmra, srv, probs, arrivals, iters, F)
        sweep.append({"rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                      "solves_per_s": n / makespan, "pairs_per_s": pairs / makespan,
                      "makespan_s": makespan, "server_steps": steps})
    clk = clocks.stop() if clocks else None
    srv.close()
    head = sweep[0]
    d = {"metric": "serve p99 latency", "unit": "ms", "precision": prec, "requests": n,
         "rate_per_s": head["rate_per_s"], "iters_per_request": iters, "F": F,
         "mix": "L {64,96,128} x K {2,4} x N {1e4,5e4,1e5}, sigma U[0.2,1]",
         "distinct_problems": pool,
         "problems": [{"L": L, "K": K, "N": N, "sigma": sg} for L, K, N, sg in specs],
         "slots": slots, "budget_bytes": budget, "data_generation_s": gen_s,
         "forms": ({"fft32": sum(1 for p in probs if p.L // p.K in (8, 16, 32)),
                    "bf16x3": sum(1 for p in probs if p.L // p.K not in (8, 16, 32))}
                   if prec == "auto" else {prec: n}),
         "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "max_ms": head["max_ms"],
         "solves_per_s": head["solves_per_s"], "pairs_per_s": head["pairs_per_s"],
         "makespan_s": head["makespan_s"], "server_steps": head["server_steps"],
         "clocks": clk}
    if len(sweep) > 1:
        d["sweep"] = sweep
    return d


def run_serve(args, rank, local):
    """The serving workload as the bench line (λ = 50/s unless --rates is given)."""
    import torch
    from paper_2204_04754_gb300 import srmra, synth
    if rank != 0:
        return
    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload]
    prec = args.prec or w["prec"]
    rates = [float(r) for r in args.rates.split(",")] if args.rates else [w["rate"]]
    d = serve_block(args.requests, rates, args.serve_pool, args.serve_slots,
                    args.serve_budget_gb, prec, srmra, synth, torch,
                    torch.cuda.current_stream(), iters=w["iters"], F=w["F"],
                    clocks=ClockSampler(gpu_index(local)))
    out = {"metric": "serve p99 latency", "value": d["p99_ms"], "unit": "ms",
           "n_gpus": 1, "steps": d["server_steps"], "warmup": 1, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": prec,
           "data": "synthetic (seeded requests)",
           "config": {"workload": args.workload, "requests": d["requests"],
                      "rate_per_s": d["rate_per_s"], "iters_per_request": d["iters_per_request"],
                      "F": d["F"], "mix": d["mix"], "distinct_problems": d["distinct_problems"],
                      "slots": d["slots"], "budget_bytes": d["budget_bytes"],
                      "data_generation_s": d["data_generation_s"]},
           "p50_ms": d["p50_ms"], "p99_ms": d["p99_ms"], "max_ms": d["max_ms"],
           "solves_per_s": d["solves_per_s"], "pairs_per_s": d["pairs_per_s"],
           "makespan_s": d["makespan_s"], "clocks": d["clocks"]}
    if "sweep" in d:
        out["sweep"] = d["sweep"]
    print(json.dumps(out), flush=True)


def e2e_run(p, prec, w, srmra, torch):
    """End to end through the public API with pinned host buffers: create (uploads y),
    a full solve of the workload's iteration count with the log-likelihood read back
    every iteration, read the final state, destroy."""
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
    return {"value": p.N * p.L * p.L * iters / el, "unit": "pairs/s",
            "h2d_bytes_per_step": h2d / iters, "d2h_bytes_per_step": d2h / iters,
            "step": f"one solve of {iters} iterations per upload; per-step bytes are "
                    f"per-iteration averages", "seconds": el}


# ------------------------------------------------------------------- precision study

def run_study(args, local):
    """Per-iteration one-step errors over a projected run of the precision workload, both
    noise levels: every form runs Algorithm 2 (F = 1, sigma_BM_1 = 1) from the workload's
    initial guess; before each of its iterations the FP64 oracle takes the form's own
    current state, runs the same iteration and projection (Eq. decaying_function
    schedule), and the form's result is compared with it.  Prints one JSON line per
    noise level, with the maxima over the iterations and the smallest threshold margin
    of the denoiser seen by the oracle."""
    import numpy as np
    import torch
    from oracle import fft_oracle as FO
    from oracle import srmra_oracle as O
    from paper_2204_04754_gb300 import srmra, synth
    torch.cuda.set_device(local)
    threads = args.oracle_threads or os.cpu_count()
    names = [args.workload] + ([COMPANION[args.workload]] if args.workload in COMPANION else [])
    decay = 2.0 ** -0.1
    for name in names:
        p = synth.workload_problem(name)
        res = {}
        t_start = time.perf_counter()
        for form in args.study_forms.split(","):
            prec = form.split("-")[0]
            flags = {"comp": srmra.SRMRA_FLAG_MSTEP_COMP,
                     "fp16": srmra.SRMRA_FLAG_MSTEP_FP16}.get(form.partition("-")[2], 0)
            s = srmra.Solver(p.L, p.K, p.sigma, p.y, prec=prec, x0=p.x0, rho1=p.rho1_0,
                             rho2=p.rho2_0, flags=flags)
            per = []
            sbm = 1.0
            margin = math.inf
            for it in range(args.study_iters):
                x, r1, r2, _, _ = s.state()
                ll = s.solve(1, 1, sigma_bm1=sbm, decay=decay)[0]
                xg, r1g, r2g, _, _ = s.state()
                xo, r1o, r2o, llo, _ = FO.em_iter_fft(p.y, x, r1, r2, p.sigma, p.K,
                                                      workers=threads)
                xo, mg = O.dct_denoise(xo, sbm)
                margin = min(margin, mg)
                per.append({"x": rel(xg, xo), "rho1": rel(r1g, r1o), "rho2": rel(r2g, r2o),
                            "LL": abs(ll - llo) / abs(llo), "margin": mg})
                sbm *= decay
            s.close()
            res[form] = {"max": {k: max(q[k] for q in per) for k in ("x", "rho1", "rho2", "LL")},
                         "last": per[-1], "min_threshold_margin": margin,
                         "per_iteration": per}
        print(json.dumps({"study": "precision", "workload": name, "iters": args.study_iters,
                          "mode": "one-step (oracle restarted from each form's state)",
                          "seconds": time.perf_counter() - t_start, "forms": res}), flush=True)


# ------------------------------------------------------------------- main

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.study:
        if rank == 0:
            run_study(args, local)
        return
    if args.workload.startswith("batched"):
        run_batched(args, rank, world, local)
        return
    if args.workload.startswith("serve"):
        run_serve(args, rank, local)
        return

    import torch
    from paper_2204_04754_gb300 import srmra, synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = synth.WORKLOADS[args.workload]
    prec = args.prec or "fp32"
    p = synth.workload_problem(args.workload, N=args.n_obs, instance=rank)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    threads = args.oracle_threads or os.cpu_count()
    head = FormRun(p, w, args.workload, prec, args.steps, args.warmup, srmra, torch, stream,
                   flush, clocks=True, local=local, barrier=dist.barrier if dist else None,
                   flags=args.flags)
    total_ms = head.total_ms
    if dist:
        total_ms = reduce_max(total_ms, dist, "cuda")
    value = job_throughput(p.N * p.L * p.L, args.steps, world, total_ms)

    out = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3", "fft32": "f32"}[prec],
           "data": "synthetic (seeded blob image, mixture shift distributions, Gaussian noise)",
           "config": {"workload": args.workload, "L_high": p.L, "K": p.K, "L_low": p.l,
                      "N": p.N, "sigma": p.sigma, "F": w["F"], "precision": prec,
                      "step": "one projected-EM iteration (E-step, M-step, DCT projection)",
                      "l2": "256 MiB buffer zeroed before every timed step",
                      "parallelism": f"{world} independent replica(s)"},
           "roofline": head.roof, "gpu_launches": head.launches,
           "phases_ms_per_step": {k: v / args.steps for k, v in head.phase_ms.items()},
           "plan": head.plan, "clocks": head.clocks}

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_run(p, prec, w, srmra, torch)
    if rank == 0 and prec == "fp32" and not args.no_mixed:
        # the tensor-core forms of the same workload, and the errors of every form
        # against the FP64 oracle after one iteration from a common state
        forms = ("bf16x3", "bf16") + (("fft32",) if p.l in (8, 16, 32) else ())
        runs = [head] + [FormRun(p, w, args.workload, f, args.steps, args.warmup, srmra,
                                 torch, stream, flush, flags=args.flags) for f in forms]
        err, how = errors_vs_oracle(p, runs, threads)
        out["error_vs_oracle"] = dict(err["fp32"], how=how)
        out["forms"] = {}
        for r in runs[1:]:
            d = r.summary(value)
            d["error_vs_oracle"] = err[r.prec]
            worst = max(err[r.prec][k] for k in ("x", "rho1", "rho2", "LL"))
            d["rel_err_max"] = worst
            d["within_1e-4"] = bool(worst <= 1e-4)
            out["forms"][r.prec] = d
            r.close()
        if "bf16x3" in out["forms"]:
            out["roofline"]["bf16x3"] = out["forms"]["bf16x3"]["roofline"]
            out["bf16x3_speedup_vs_fp32"] = out["forms"]["bf16x3"]["speedup_vs_fp32"]
            out["bf16x3_rel_err_max_vs_oracle"] = out["forms"]["bf16x3"]["rel_err_max"]
    head.close()
    if rank == 0 and prec == "fp32" and not args.no_mixed and not args.no_extra:
        if args.workload in COMPANION:
            _, _, runs2, blk = workload_block(COMPANION[args.workload], args.steps,
                                              args.warmup, srmra, torch, stream, flush,
                                              threads, local=local,
                                              forms=("fp32", "bf16x3", "bf16", "fft32"))
            for r in runs2:
                r.close()
            out[COMPANION[args.workload]] = blk
        if args.workload != SECONDARY:
            out[SECONDARY] = secondary_block(args.steps, args.warmup, srmra, torch, stream,
                                             flush, threads)
        del flush
        torch.cuda.empty_cache()
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        out["batched_64"] = batched_block(min(args.steps, 5), args.warmup, rank, "bf16x3",
                                          srmra, synth, torch, stream, flush)
        out["serve"] = serve_block(16, [2.0], 6, args.serve_slots, args.serve_budget_gb,
                                   "bf16x3", srmra, synth, torch, stream)
        # the same trace with each request in the form the server picks for it
        out["serve_auto"] = serve_block(16, [2.0], 6, args.serve_slots, args.serve_budget_gb,
                                        "auto", srmra, synth, torch, stream)
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_oracle_rate(p, args.cpu_seconds)
        cb.pop("n_sub", None)
        out["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
