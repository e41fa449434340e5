#!/usr/bin/env python
"""Benchmark of the projected-EM hot path (E-step + M-step + denoiser) on GB300.

One *step* is one projected-EM iteration (Algorithm 2 with F = 1): E-step over all N
observations x L^2 shifts, M-step, block-DCT projection.  The metric is observation x
shift pairs per second, N * L^2 * steps / device time.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl srmra|reference]
                    [--workload NAME] [--prec fp32|bf16|bf16x3|fft32]

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
                    help="skip the bf16x3-vs-fp32 comparison block")
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
    if args.workload in ("batched_64", "serve"):
        sp = synth.batched_instances(1)[0] if args.workload == "batched_64" else \
            dict(L=96, K=2, N=10_000, sigma=0.5, seed=synth.seed_for(5, 0))
        p = synth.make_problem(sp["L"], sp["K"], sp["N"], sp["sigma"], sp["seed"])
    else:
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


def mixed_block(p, w, steps, warmup, srmra, torch, stream, flush, fp32_value, form="bf16x3"):
    """The same workload in another form (split-bf16 tensor cores, or the polyphase FFT):
    pairs/s and speedup over the fp32 form; and the error at which that speedup holds:
    one EM iteration of each form from the same state (the fp32 run's state after the
    warm-up), compared."""
    import numpy as np
    s3 = srmra.Solver(p.L, p.K, p.sigma, p.y, prec=form, x0=p.x0, rho1=p.rho1_0,
                      rho2=p.rho2_0, stream=stream.cuda_stream)
    s3.solve(warmup, w["F"], sigma_bm1=1.0, loglik=False)
    ms = time_steps(lambda: s3.solve(1, w["F"], sigma_bm1=0.0, loglik=False), steps,
                    stream, torch, flush)
    s1 = srmra.Solver(p.L, p.K, p.sigma, p.y, prec="fp32", x0=p.x0, rho1=p.rho1_0,
                      rho2=p.rho2_0, stream=stream.cuda_stream)
    s1.solve(warmup, w["F"], sigma_bm1=1.0, loglik=False)
    st = s1.state()
    s3.set_state(*st)
    s1.em_iter(1, loglik=False)
    s3.em_iter(1, loglik=False)
    (x1, r11, r21, _, _), (x3, r13, r23, _, _) = s1.state(), s3.state()
    s1.close()
    s3.close()
    value = p.N * p.L * p.L * steps / (sum(ms) / 1e3)
    rel = lambda a, b: float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))
    note = {"bf16x3": "per-iteration parity with the FP64 oracle (<= 1e-4) is tested in "
                      "tests/test_gpu_tc.py",
            "fft32": "exact reformulation (polyphase correlation by l x l FFTs) in float32; "
                     "per-iteration parity with the FP64 oracle (<= 1e-5) is tested in "
                     "tests/test_gpu_fft.py"}[form]
    return {"precision": form, "value": value, "unit": "pairs/s",
            "ms_per_step": sum(ms) / steps, "speedup_vs_fp32": value / fp32_value,
            "one_step_rel_diff_vs_fp32": {"x": rel(x3, x1), "rho1": rel(r13, r11),
                                          "rho2": rel(r23, r21)},
            "note": note}


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


def run_batched(args, rank, world, local):
    """64 uneven problems advanced together: grouped launches in a CUDA graph."""
    import numpy as np
    import torch
    from paper_2204_04754_gb300 import srmra, synth
    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload]
    prec = args.prec or w["prec"]
    specs = synth.batched_instances(w["count"], seed=synth.seed_for(4) + 1000 * rank)
    stream = torch.cuda.current_stream()
    probs = [synth.make_problem(sp["L"], sp["K"], sp["N"], sp["sigma"], sp["seed"])
             for sp in specs]
    solvers = [srmra.Solver(p.L, p.K, p.sigma, p.y, prec=prec, x0=p.x0, rho1=p.rho1_0,
                            rho2=p.rho2_0, stream=stream.cuda_stream) for p in probs]
    t0 = time.perf_counter()
    batch = srmra.Batch(solvers, autotune=True)
    tune_s = time.perf_counter() - t0
    batch.solve(args.warmup, w["F"], sigma_bm1=1.0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    l0 = sum(s.launches for s in solvers)
    clocks = ClockSampler(local)
    clocks.start()
    ms = time_steps(lambda: batch.solve(1, w["F"], sigma_bm1=0.0), args.steps, stream, torch,
                    flush)
    clk = clocks.stop()
    launches = sum(s.launches for s in solvers) - l0
    # per-pass device times: one more iteration enqueued without the graph (events
    # recorded inside a captured graph cannot be timed)
    probe = srmra.Batch(solvers, autotune=False, graph=False)
    probe.solve(1, w["F"], sigma_bm1=0.0)
    p1_ms, p2_ms = probe.pass_ms()
    probe.close()
    total_ms = float(sum(ms))
    pairs = sum(p.N * p.L * p.L for p in probs)
    alg2 = sum(4 * p.l * p.l * p.N * p.L * p.L for p in probs)
    peaks, peak_src = load_peaks()
    peak = float(peaks["bf16_tflops_sustained"])
    achieved = alg2 / (p2_ms / 1e3) / 1e12
    out = {"metric": METRIC, "value": world * pairs * args.steps / (total_ms / 1e3),
           "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": prec, "data": "synthetic (64 seeded problems)",
           "config": {"workload": args.workload, "problems": len(probs),
                      "L_high": sorted({p.L for p in probs}), "K": sorted({p.K for p in probs}),
                      "N_total": int(sum(p.N for p in probs)), "F": w["F"],
                      "step": "one projected-EM iteration of all problems (grouped launches, "
                              "CUDA graph replay)",
                      "l2": "256 MiB buffer zeroed before every timed step",
                      "autotuner": batch.tuning(), "autotune_seconds": tune_s,
                      "parallelism": f"{world} independent replica(s)"},
           "roofline": {"bound": "tensor", "kernel": f"k_p2_tc grouped ({prec})",
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": None,
                        "algorithmic_flops_per_launch": alg2, "avg_launch_ms": p2_ms,
                        "peak_source": f"dense bf16, sustained, of {peak_src}"},
           "phases_ms_last_step": {"pass1_grouped": p1_ms, "pass2_grouped": p2_ms},
           "gpu_launches": launches, "clocks": clk}
    batch.close()
    for s_ in solvers:
        s_.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    _ = np


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


def run_serve(args, rank, local):
    """Poisson arrivals of projected-EM solve requests (L in {64,96,128}, K in {2,4},
    N in {1e4, 5e4, 1e5}, sigma ~ U[0.2, 1], 30 projected iterations) served with
    continuous batching.  Latency = completion - planned arrival (queueing included).
    The requests draw their data from a pool of --serve-pool distinct seeded problems
    (request k uses pool entry k mod pool size), so that long traces fit in host memory;
    --rates runs the same trace at several arrival rates (a sweep that shows where the
    offered load exceeds capacity)."""
    import numpy as np
    import torch
    from paper_2204_04754_gb300 import srmra, synth
    if rank != 0:
        return
    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload]
    prec = args.prec or w["prec"]
    rng = np.random.Generator(np.random.PCG64(synth.seed_for(5)))
    n = args.requests
    rates = [float(r) for r in args.rates.split(",")] if args.rates else [w["rate"]]
    unit_gaps = rng.exponential(1.0, size=n)  # arrivals at rate r: cumsum(unit_gaps) / r
    pool = min(n, args.serve_pool)
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
    stream = torch.cuda.current_stream()
    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.8, args.serve_budget_gb * 2 ** 30))
    srv = srmra.Server(budget, max_active=args.serve_slots, prec=prec, stream=stream.cuda_stream)
    # warm the kernels and graph machinery on a tiny request (not part of the trace)
    wp = synth.make_problem(64, 4, 2000, 0.5, seed=synth.seed_for(5, 999))
    wid = srv.submit(wp.L, wp.K, wp.sigma, wp.y, 2, F=w["F"])
    while srv.step()[0] > 0:
        pass
    srv.result(wid, wp.L)
    pairs = sum(p.N * p.L * p.L * w["iters"] for p in probs)
    sweep = []
    clocks = ClockSampler(local)
    clocks.start()
    for rate in rates:
        arrivals = np.cumsum(unit_gaps) / rate
        lat, makespan, steps = serve_trace(srmra, srv, probs, arrivals, w["iters"], w["F"])
        sweep.append({"rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                      "solves_per_s": n / makespan, "pairs_per_s": pairs / makespan,
                      "makespan_s": makespan, "server_steps": steps})
    clk = clocks.stop()
    srv.close()
    head = sweep[0]
    out = {"metric": "serve p99 latency", "value": head["p99_ms"], "unit": "ms",
           "n_gpus": 1, "steps": head["server_steps"], "warmup": 1, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": prec,
           "data": "synthetic (seeded requests)",
           "config": {"workload": args.workload, "requests": n, "rate_per_s": head["rate_per_s"],
                      "iters_per_request": w["iters"], "F": w["F"],
                      "mix": "L {64,96,128} x K {2,4} x N {1e4,5e4,1e5}, sigma U[0.2,1]",
                      "distinct_problems": pool, "slots": args.serve_slots,
                      "budget_bytes": budget, "data_generation_s": gen_s},
           "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "max_ms": head["max_ms"],
           "solves_per_s": head["solves_per_s"], "pairs_per_s": head["pairs_per_s"],
           "makespan_s": head["makespan_s"], "clocks": clk}
    if len(sweep) > 1:
        out["sweep"] = sweep
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload.startswith("batched"):
        run_batched(args, rank, world, local)
        return
    if args.workload.startswith("serve"):
        run_serve(args, rank, local)
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
        total_ms = reduce_max(total_ms, dist, "cuda")
        dist.barrier()

    pairs_per_step = p.N * p.L * p.L
    value = job_throughput(pairs_per_step, args.steps, world, total_ms)

    # roofline of the dominant kernel (phase), from the live CUDA events
    peaks, peak_src = load_peaks()
    dom = max(("pass1", "pass2"), key=lambda k: phase_ms[k])
    if prec == "fft32":
        # per (observation, phase): one inverse l x l FFT (pass 1), plus the forward FFT
        # of the weight map and the products (pass 2), 5 n log2 n flops per complex
        # n-point FFT; spread over the l^2 lags (pairs) of the phase
        lg = math.log2(p.l * p.l)
        per_pair_flops = {"pass1": 5 * lg + 6, "pass2": 10 * lg + 14}[dom]
    else:
        per_pair_flops = {"pass1": 2 * p.l * p.l, "pass2": 4 * p.l * p.l}[dom]
    avg_launch_s = phase_ms[dom] / max(1, phase_n[dom]) / 1e3
    achieved = per_pair_flops * pairs_per_step / avg_launch_s / 1e12
    if prec in ("fp32", "fft32"):
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
    traffic = traffic_from_profiles(kern, args.workload, prec)
    roof = {"bound": bound, "kernel": kern, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "algorithmic_flops_per_launch": per_pair_flops * pairs_per_step,
            "avg_launch_ms": avg_launch_s * 1e3, "peak_source": peak_note}
    if traffic:
        # the same kernel's DRAM bandwidth: recorded bytes per launch over the live launch
        # time, against the measured HBM copy bandwidth
        hbm = float(peaks["hbm_gbs"])
        roof["dram_gbs"] = traffic / avg_launch_s / 1e9
        roof["dram_frac_of_hbm_peak"] = roof["dram_gbs"] / hbm

    out = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3", "fft32": "f32"}[prec],
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
    if rank == 0 and prec == "fp32" and not args.no_mixed:
        out["bf16x3"] = mixed_block(p, w, args.steps, args.warmup, srmra, torch, stream, flush,
                                    value)
        if p.l in (8, 16, 32):
            out["fft32"] = mixed_block(p, w, args.steps, args.warmup, srmra, torch, stream,
                                       flush, value, form="fft32")
        out["online"] = online_block(p, w, args.steps, args.warmup, srmra, torch, stream,
                                     flush, value)
        out["mom"] = mom_block(p, args.steps, args.warmup, srmra, torch, stream, flush,
                               float(load_peaks()[0].get("sm_max_mhz", 2070.0)))
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
