"""FastMNMF throughput on GB300: TF-bin*iterations per second.

One step = one whole FastMNMF job on the paper-scale single mixture (M=4 channels, N=4
sources, K=32 bases, F=513 bins, T=640 frames, 10 % of the bins with diffuse noise):
restore the seeded initial state, 100 iterations (W, H, g~ MU, V + IP, x~, normalisation,
log-likelihood), then the multichannel Wiener separation, all on device-resident data.  L2 is flushed (a 512 MB
write) between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun, one rank per GPU) every rank runs its own mixture (seed + rank): the
mixtures are independent problems, so the units shard with no collective ("weak").
--impl reference times the float64 CPU oracle on the host cores instead (rank 0 only).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FastMNMF TF-bin·iters/s vs plain FP32 on 1 GB300; serving p50/p99 latency"
UNIT = "TF-bin·iters/s"
WORKLOADS = {
    # paper-scale single mixture (the headline): 1024-point STFT at 16 kHz, ~10 s, 100 iterations
    "c1": dict(M=4, N=4, K=32, F=513, T=640, iters=100, diffuse=0.1),
    # large mixture (mixed-precision case): 2048-point STFT, ~65 s
    "c2": dict(M=8, N=6, K=64, F=1025, T=4096, iters=10, diffuse=0.0),
}
WORKLOAD = WORKLOADS["c1"]
PRECISIONS = {"fp32": 0, "bf16": 1, "tf32": 2}
# timed forms: (precision, schedule).  "fused": FP32 with the bin-fused schedule (two launches
# per iteration); "sweep": FP32 with one tiled launch per block (the plain form);
# "bf16" / "tf32": the mixed-precision forms (tensor-core contractions).
FORMS = {"fused": ("fp32", 2), "sweep": ("fp32", 1), "bf16": ("bf16", 0), "tf32": ("tf32", 0)}
DTYPES = {"fused": "f32", "sweep": "f32", "bf16": "bf16", "tf32": "tf32"}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock = 80.5 TFLOP/s


def kernel_flops(kind: str, F, T, M, N, K) -> float:
    """Algorithmic FLOPs of one launch of a plain-form kernel class (per TF bin x F*T)."""
    ft = F * T
    mm = M * M
    per_point = {
        # A, B (M rcp + 3M mul), P, R (4NM), contraction over t (4NK)
        "w_update": 4 * N * K + 4 * N * M + 4 * M,
        # lambda (2NK), y~ (2NM), A, B, P, R as above, contraction over f (4NK)
        "h_update": 6 * N * K + 6 * N * M + 4 * M,
        # lambda (2NK), y~ (2NM), A, B (4M), num/den over t (4NM)
        "g_update": 2 * N * K + 6 * N * M + 4 * M,
        # fused per-bin kernel: lambda of the bin (2NK), g~ update (y~ 2NM, A, B 4M, sums 4NM),
        # V_fm (y~ 2NM, 1/y~ M, products 2M^2, sums 2M^3), x~ (8M^2), y~ and the log-likelihood
        # terms (2NM + 3M), P, R of the W update (4NM + 4M), W sums over t (4NK), lambda of the
        # new W (2NK), P, R of the H update (y~ 2NM, A, B 4M, 4NM)
        "bin": 8 * N * K + 20 * N * M + 16 * M + 10 * M * M + 2 * M ** 3,
        # fused H GEMM: num and den sums over f (4NK)
        "hgemm": 4 * N * K,
        # lambda, y~, 1/y~, x x^H (3 M^2), V accumulation (2 M * M^2)
        "scm": 2 * N * K + 2 * N * M + M + 3 * mm + 2 * M * mm,
        # Q x (8 M^2), |.|^2, LL term (4M)
        "xt_loglik": 8 * mm + 7 * M,
    }
    return float(per_point.get(kind, 0)) * ft


# Mixtures of at most this many frames form x~, the log-likelihood terms and the P, R of the
# next W update inside the IP kernel (the library's choice); longer ones in the x~ kernel.
FUSE_XT_FRAMES = 1024


def kernel_bytes(kind: str, F, T, M, N, K) -> float:
    """Algorithmic DRAM bytes of one launch of a mixed-form kernel class (operands read
    once, results written once; float32 / complex64 storage)."""
    ft = F * T
    fused = T <= FUSE_XT_FRAMES
    mu = 8 * N * K * (F + T)                                      # W and H read and written
    xt = 20 * ft * M + 8 * N * ft                                 # X, y~ read, x~, y~ written; P, R of the next W update
    ip = 4 * F * M ** 4 + 64 * F * M * M                          # one V_fm set read; Q, Q^-1 read and written
    return float({
        "gemm_lambda": 4 * N * ft + 4 * N * K * (F + T),         # lambda written, W and H read
        "gemm_w": 8 * N * ft + 4 * N * K * T,                     # P, R and H read
        "gemm_h": 8 * N * ft + 4 * N * K * F,                     # P, R and W read
        "pr": 4 * ft * M + 4 * N * ft + 8 * N * ft,               # H update: x~, lambda read; P, R written
        "g_update": 4 * N * ft + 4 * ft * M,                      # lambda and x~ read
        "scm": 4 * N * ft + 8 * ft * M + 4 * ft * M,              # lambda, X read, y~ written
        "xt_loglik": (0 if fused else xt) + mu,                   # x~ part (long mixtures) and mu
        "wiener": 8 * ft * M + 4 * N * ft + 8 * N * ft * M,       # X, lambda read; images written
        "ip": ip + (xt if fused else 0),                         # x~ part inside the IP kernel (short mixtures)
        "apply": 8 * N * K * (F + T),                               # num/den (one split) read, W or H updated
    }.get(kind, 0))


def roofline_for(dom, avg_ms, precision, F, T, M, N, K, workload):
    peaks = read_peaks() or {}
    if precision in ("fp32", "fused", "sweep") and kernel_flops(dom, F, T, M, N, K) > 0:
        achieved = kernel_flops(dom, F, T, M, N, K) / (avg_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": read_traffic(dom, workload, precision), "kernel": dom,
                "avg_launch_us": avg_ms * 1e3,
                "peak_source": "derived: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2070 MHz (max SM clock)"}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = kernel_bytes(dom, F, T, M, N, K) / (avg_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": read_traffic(dom, workload, precision), "kernel": dom, "avg_launch_us": avg_ms * 1e3,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


def read_traffic(kernel: str, workload: str, precision: str):
    """DRAM bytes per launch from the committed ncu summary (None if not captured for this
    kernel, workload and form)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        for line in open(path):
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[2] == precision:
                return float(parts[3])
    except OSError:
        pass
    return None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id: str | None):
        self.dev_id = dev_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.dev_id:
            cmd += ["-i", self.dev_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, device) -> float:
    """The maximum of a per-rank figure over all ranks (a job lasts as long as its slowest
    rank); the value itself without a process group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput of replicas: the units all ranks processed over the slowest time."""
    return units_per_rank * world / max_seconds


def oracle_iteration_rate(mix, W, H, G, Q, n_iter: int, min_seconds: float = 0.0, max_iter: int = 100):
    """Times the float64 oracle (as it stands) on the host: n_iter iterations, continued in
    runs of n_iter from the state reached until min_seconds have passed (at most max_iter);
    returns (rate, cores, seconds, iterations)."""
    from oracle import fastmnmf_oracle as O
    X = mix.X.astype(np.complex128)
    W, H, G, Q = W.astype(np.float64), H.astype(np.float64), G.astype(np.float64), Q.astype(np.complex128)
    c0, t0 = time.process_time(), time.perf_counter()
    done = 0
    while True:
        W, H, G, Q, _ = O.iterate(X, W, H, G, Q, n_iter=n_iter)
        done += n_iter
        if time.perf_counter() - t0 >= min_seconds or done + n_iter > max_iter:
            break
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    F, T = X.shape[0], X.shape[1]
    return F * T * done / wall, max(1, int(math.ceil(cpu / wall - 0.05))), wall, done


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1903_03237_gb300.synth import make_mixture, make_state
    w = WORKLOAD
    mix = make_mixture(w["F"], w["T"], w["M"], w["N"], w["K"], 0, diffuse_frac=w["diffuse"])
    W, H, G, Q = make_state(w["F"], w["T"], w["M"], w["N"], w["K"], 0)
    for _ in range(args.warmup):
        oracle_iteration_rate(mix, W, H, G, Q, 1)
    rates, secs, cores = [], [], 1
    for _ in range(args.steps):
        r, c, s, _ = oracle_iteration_rate(mix, W, H, G, Q, 1)
        rates.append(r)
        secs.append(s)
        cores = max(cores, c)
    value = w["F"] * w["T"] * args.steps / sum(secs)
    sample = f"1 oracle iteration of the {w['F']}x{w['T']} M{w['M']} N{w['N']} K{w['K']} mixture per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        # the same config as this arm's line (impl and dtype tell the two apart)
        "data": "synthetic",
        "config": _config(args.form) | {"parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _config(form="bf16"):
    w = WORKLOAD
    prec = {"fused": "FP32, bin-fused schedule (two launches per iteration), float-float IP solve",
            "sweep": "FP32, one tiled launch per block (plain form), float-float IP solve",
            "bf16": "mixed: split-BF16 (hi + lo, three MMAs) tcgen05 contractions for lambda, the W/H sums, V_fm "
                    "and the g~ sums, FP32 accumulation in TMEM, float-float IP solve",
            "tf32": "mixed: TF32 tensor-core GEMMs for lambda and the W/H sums, split-BF16 tensor-core V_fm "
                    "and g~ sums, FP32 accumulation, float-float IP solve"}[form]
    name = "paper-scale single mixture" if WORKLOAD is WORKLOADS["c1"] else "large mixture"
    return {"workload": f"{name} M{w['M']} N{w['N']} K{w['K']} F{w['F']} T{w['T']}, "
                        f"{w['iters']} iterations + Wiener separation per step",
            "M": w["M"], "N": w["N"], "K": w["K"], "F": w["F"], "T": w["T"], "iters_per_step": w["iters"],
            "l2": "flushed between timed steps (512 MB write)", "precision": prec}


def _measure(fm, torch, mix, args, form, steps, warmup, rank, world, local, sample_clocks):
    """Times one form on the workload: each step is a whole job (fresh initial state, the
    workload's iterations, Wiener separation) with X resident in HBM; then the same job end
    to end through the C ABI with host buffers.  Returns the numbers of the bench line."""
    w = WORKLOAD
    F, T, M, N, K, iters = w["F"], w["T"], w["M"], w["N"], w["K"], w["iters"]
    stream = torch.cuda.Stream()
    Xd = torch.from_numpy(mix.X).cuda()
    torch.cuda.synchronize()
    precision, schedule = FORMS[form]
    ctx = fm.Context(Xd, N, K, seed=rank, stream=stream.cuda_stream, precision=PRECISIONS[precision],
                     schedule=schedule)
    out = torch.empty((N, F, T, M), dtype=torch.complex64, device="cuda")
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step():  # one whole job: fresh initial state, the iterations, Wiener separation
        ctx.restart()
        ctx.iterate(iters)
        ctx.separate(out)

    for _ in range(warmup):
        step()
    ctx.sync()
    tune = None
    if not args.no_autotune:
        # the library's tuner picks the launch shapes for this workload (state restored after)
        sp = ctx.autotune(3)
        tune = {"trial_speedup": sp, "scales": [round(v, 4) for v in ctx.get_tuning()]}
        for _ in range(warmup):
            step()
        ctx.sync()
    # calibration (untimed): which kernel class dominates the step
    ctx.set_timing(True)
    step()
    ctx.sync()
    cal = ctx.kernel_times()
    dom = max((k for k in cal if cal[k][1] > 0), key=lambda k: cal[k][0])
    shares = {k: round(v[0] / max(1e-12, sum(x[0] for x in cal.values())), 4) for k, v in cal.items() if v[1]}
    avg_all = {k: round(1e3 * v[0] / v[1], 2) for k, v in cal.items() if v[1]}
    ctx.set_timing(False)
    for _ in range(warmup):  # the graph variant without timing events
        step()
    ctx.sync()
    dev_id = None
    try:
        dev_id = str(torch.cuda.get_device_properties(local).uuid)
        dev_id = dev_id if dev_id.startswith("GPU-") else "GPU-" + dev_id
    except Exception:
        dev_id = None

    def timed_steps(evs):
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)

    # value: the steps as a user runs them (no events between the library's kernels)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = ctx.launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev_id if sample_clocks else None) as clocks:
        # NVTX range "timed" (main form only): lets ncu capture exactly the timed launches
        if sample_clocks:
            torch.cuda.nvtx.range_push("timed")
        timed_steps(evs)
        torch.cuda.synchronize()
        if sample_clocks:
            torch.cuda.nvtx.range_pop()
    ctx.sync()
    launches = ctx.launch_count() - launches0
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    total_ms = reduce_max(total_ms, "cuda")
    value = job_rate(F * T * iters * steps, world, total_ms / 1e3)

    # roofline of the dominant kernel: the same steps again, each of its launches bracketed by
    # events on the context stream (event nodes inside the captured graph)
    ctx.set_timing([dom])
    for _ in range(warmup):  # capture that graph variant first
        step()
    ctx.sync()
    ctx.kernel_times()
    evs2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    timed_steps(evs2)
    torch.cuda.synchronize()
    ctx.sync()
    kt = ctx.kernel_times()
    bracketed_ms = sum(a.elapsed_time(b) for a, b in evs2) / steps
    avg_ms = kt[dom][0] / kt[dom][1]
    roofline = roofline_for(dom, avg_ms, form, F, T, M, N, K, args.workload)
    roofline["launches_timed"] = kt[dom][1]
    roofline["ms_per_step_with_kernel_events"] = bracketed_ms

    # end to end through the C ABI with host buffers: H2D mixture, iterations, D2H images
    ctx.set_timing(False)
    # pinned host buffers (page-locked: the copies run as DMA at full link speed)
    Xp = torch.empty(mix.X.shape, dtype=torch.complex64, pin_memory=True)
    Xh = Xp.numpy()
    Xh[...] = mix.X
    outp = torch.empty((N, F, T, M), dtype=torch.complex64, pin_memory=True)
    outh = outp.numpy()
    ctx.reset(Xh, seed=rank)
    ctx.iterate(iters)
    ctx.separate(outh)
    e2e_s = []
    for _ in range(max(1, steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.reset(Xh, seed=rank)
        ctx.iterate(iters)
        ctx.separate(outh)  # synchronises (host output)
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = reduce_max(sum(e2e_s), "cuda")
    e2e_val = job_rate(F * T * iters * len(e2e_s), world, e2e_total)
    ctx.close()
    return {"value": value, "ms_per_step": total_ms / steps, "roofline": roofline, "launches": launches,
            "e2e": e2e_val, "shares": shares, "avg_us": avg_all, "clocks": clocks.summary(), "tune": tune}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1903_03237_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1903_03237_gb300 import fastmnmf as fm
    from paper_1903_03237_gb300.synth import make_mixture, make_state

    w = WORKLOAD
    F, T, M, N, K, iters = w["F"], w["T"], w["M"], w["N"], w["K"], w["iters"]
    mix = make_mixture(F, T, M, N, K, seed=rank, diffuse_frac=w["diffuse"])
    res = _measure(fm, torch, mix, args, args.form, args.steps, args.warmup, rank, world, local, True)
    # the plain FP32 form (one launch per block) and the mixed BF16 form on the same
    # workload, for the comparison the metric names
    others = {}
    if not args.no_compare:
        for name, form in (("plain_fp32", "sweep"), ("fused_fp32", "fused"), ("mixed_bf16", "bf16")):
            if form == args.form:
                continue
            psteps = max(2, min(args.steps, 3))
            pr = _measure(fm, torch, mix, args, form, psteps, max(3, args.warmup), rank, world, local, False)
            others[name] = {"value": pr["value"], "ms_per_step": pr["ms_per_step"], "e2e_value": pr["e2e"],
                            "steps": psteps, "autotune": pr["tune"], "dominant_kernel": pr["roofline"]["kernel"],
                            "roofline_frac": pr["roofline"]["frac"]}

    serving = None
    if rank == 0 and not args.no_serving:
        # the metric's serving half, bounded: 300 requests at 20 req/s, then a saturated burst
        # of 200 (every request queued at once), each with the one-at-a-time comparison
        cb, fifo = serving_replay(fm, 300, 20.0, args.max_active, args.form)
        cb2, fifo2 = serving_replay(fm, 200, 0.0, args.max_active, args.form)
        keep = ("p50_ms", "p99_ms", "throughput", "completed", "failed")
        serving = {"workload": "Poisson arrivals (seed 7), M4 N3 K16 F513, T lognormal (median 375, sigma 0.6, cap "
                               "6000), 50 iterations + Wiener per request; latency = completion - arrival",
                   "unit_throughput": UNIT, "max_active": args.max_active, "iters_per_step": 10,
                   "rate_20_per_s": {"requests": 300, "continuous_batching": {k: cb[k] for k in keep},
                                     "one_at_a_time": {k: fifo[k] for k in keep}},
                   "burst_200_at_once": {"requests": 200, "continuous_batching": {k: cb2[k] for k in keep},
                                         "one_at_a_time": {k: fifo2[k] for k in keep}}}

    dp = None
    if rank == 0 and not args.no_dp:
        dp = dp_measure(fm, torch, 20, 3)
        if not args.no_cpu_baseline:
            dp["oracle_s_per_iteration"] = dp_oracle_seconds()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # a bounded sample: all bins of c1 (2 iterations), the first 96 bins of larger mixtures
        Fs = F if F * T <= 513 * 640 else 96
        sub = type(mix)(X=mix.X[:Fs], W=None, H=None, G=None, Q=None, noisy_bins=None)
        W0, H0, G0, Q0 = make_state(Fs, T, M, N, K, 0)
        r, cores, secs, nit = oracle_iteration_rate(sub, W0, H0, G0, Q0, 2, min_seconds=10.0)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{nit} oracle iterations (runs of 2 until 10 s had passed) of {Fs} of the {F} bins x {T} "
                         f"frames of the same mixture ({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.form],
            "data": "synthetic",
            "config": _config(args.form) | {"parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": res["roofline"], "cpu_baseline": cpu,
            "e2e": {"value": res["e2e"], "unit": UNIT, "h2d_bytes_per_step": F * T * M * 8,
                    "d2h_bytes_per_step": N * F * T * M * 8},
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "kernel_share": res["shares"], "kernel_avg_us": res["avg_us"], "autotune": res["tune"],
        }
        for name, o in others.items():
            line[name] = o
        if serving is not None:
            line["serving"] = serving
        if dp is not None:
            line["fastmnmf_dp"] = dp
        if "plain_fp32" in others:
            line["speedup_vs_plain_fp32"] = res["value"] / others["plain_fp32"]["value"]
        # the whole iteration against HBM by the minimum traffic of one iteration with lambda,
        # y~, A, B, P, R on chip (X read twice, x~ written once and read three times: 32 F T M
        # bytes), over the step time per iteration (restart and Wiener filter included)
        hbm = float((read_peaks() or {}).get("hbm_gbs", 6800.0))
        it_us = 1e3 * res["ms_per_step"] / iters
        it_gbs = 32.0 * F * T * M / (it_us * 1e-6) / 1e9
        line["iteration_hbm_equiv"] = {"bytes_per_iteration": 32 * F * T * M, "us_per_iteration": it_us,
                                       "achieved_gbs": it_gbs, "peak_gbs": hbm, "frac": it_gbs / hbm}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# FastMNMF-DP at the paper's setting (Sec. IV-A): 8 s at 16 kHz with a 1024-point window and
# a 256-point shift (F = 513, T = 500), M = 5, speech + one noise source (N = 2) with K = 16
# noise bases, D = 16, 30 proposals per frame, eps = 1e-4; decoder width 128 (random weights).
DP_SETTING = dict(F=513, T=500, M=5, N=2, K=16, D=16, Hd=128, S=30, eps=1e-4)
DP_PAPER_GPU_MS = 98.0   # Table I (GPU, GTX 1080 Ti): FastMNMF-DP, N = 2, K = 16, 0.98 decisec per iteration


def dp_flops_mh(F, T, M, D, Hd, S):
    """Algorithmic flops of one Metropolis launch: per proposal and frame the decoder (hidden
    layer 2 D Hd, output layer 2 Hd F) and the log gamma terms (about 8 flops per (f, m) besides
    one exponential per f and one division pair and one logarithm per (f, m))."""
    return float(S) * T * (2.0 * D * Hd + 2.0 * Hd * F + 8.0 * F * M)


def dp_measure(fm, torch, steps, warmup):
    """ms per FastMNMF-DP iteration at the paper's setting, device-resident draws (timed with
    events on the context's stream over `steps` consecutive iterations), the Metropolis launch
    alone, and end to end with the draws copied from pinned host memory inside the timed region
    and the log-likelihood read back."""
    from paper_1903_03237_gb300.synth import make_mixture, make_dp_state, make_decoder, make_dp_draws
    c = DP_SETTING
    F, T, M, N, K, Dd, Hd, S = c["F"], c["T"], c["M"], c["N"], c["K"], c["D"], c["Hd"], c["S"]
    X = make_mixture(F, T, M, N, K, 0).X
    state = make_dp_state(F, T, M, N, K, Dd, 0)
    theta = make_decoder(F, Dd, Hd, 0)
    n = warmup + steps
    xi, logu = make_dp_draws(n, S, T, Dd, 0)
    xid, lud = torch.from_numpy(xi).cuda(), torch.from_numpy(logu).cuda()
    xih, luh = torch.from_numpy(xi).pin_memory(), torch.from_numpy(logu).pin_memory()
    st = torch.cuda.Stream()
    out = {"workload": "FastMNMF-DP, F513 T500 M5 N2 K16, D16, decoder width 128 (seeded random weights), "
                       "30 proposals per frame, eps 1e-4; consecutive iterations (state L2-resident, as in a run)",
           "unit": "ms per iteration", "paper_gtx1080ti_ms": DP_PAPER_GPU_MS}
    with fm.DPContext(X, N, K, D=Dd, Hd=Hd, n_proposals=S, eps=c["eps"], stream=st.cuda_stream) as dp:
        dp.set_decoder(*theta)
        dp.set_state(*state)
        dp.iterate(warmup, xid[:warmup], lud[:warmup])
        dp.sync()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        dp.iterate(steps, xid[warmup:], lud[warmup:])
        e1.record(st)
        dp.sync()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # the Metropolis launch alone (one iteration's proposals), bracketed by events on the
        # context's stream; the call also reads two 8-byte counters
        dp.set_state(*state)
        torch.cuda.synchronize()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(st)
        fm.lib().fmnmf_dp_metropolis(dp._dp, xid[0].data_ptr(), lud[0].data_ptr(), 1, None, None)
        e3.record(st)
        dp.sync()
        torch.cuda.synchronize()
        mh_ms = e2.elapsed_time(e3)
        # end to end: draws from pinned host memory, copied inside the timed region, and the
        # log-likelihood read back
        dp.set_state(*state)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xs = torch.empty_like(xid[:steps])
        ls = torch.empty_like(lud[:steps])
        with torch.cuda.stream(st):
            xs.copy_(xih[warmup:], non_blocking=True)
            ls.copy_(luh[warmup:], non_blocking=True)
        dp.iterate(steps, xs, ls)
        ll = dp.loglik()
        e2e_ms = 1e3 * (time.perf_counter() - t0) / steps
        acc = dp.accepted()
    fl = dp_flops_mh(F, T, M, Dd, Hd, S)
    ach = fl / (mh_ms * 1e-3) / 1e12
    out.update({"ms_per_iteration": ms, "iterations_per_s": 1e3 / ms, "e2e_ms_per_iteration": e2e_ms,
                "h2d_bytes_per_iteration": S * T * (Dd + 1) * 4, "d2h_bytes_per_call": 8,
                "vs_paper_gpu": DP_PAPER_GPU_MS / ms, "loglik_final": ll, "accepted_last_run": acc,
                "steps": steps, "warmup": warmup, "metropolis_ms": mh_ms, "metropolis_share": mh_ms / ms,
                "metropolis_roofline": {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                        "frac": ach / FP32_PEAK_TFLOPS, "flops_per_launch": fl,
                                        "kernel": "k_dp_mh"}})
    return out


def dp_oracle_seconds():
    """Seconds of the float64 oracle (as it stands) for one FastMNMF-DP iteration at the same
    setting, timed on the host."""
    from oracle import fastmnmf_dp_oracle as DPO
    from paper_1903_03237_gb300.synth import make_mixture, make_dp_state, make_decoder, make_dp_draws
    c = DP_SETTING
    F, T, M, N, K, Dd, Hd, S = c["F"], c["T"], c["M"], c["N"], c["K"], c["D"], c["Hd"], c["S"]
    X = make_mixture(F, T, M, N, K, 0).X.astype(np.complex128)
    state = [a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
             for a in make_dp_state(F, T, M, N, K, Dd, 0)]
    theta = tuple(a.astype(np.float64) for a in make_decoder(F, Dd, Hd, 0))
    xi, logu = make_dp_draws(1, S, T, Dd, 0)
    t0 = time.perf_counter()
    DPO.iterate_dp(X, *state, theta, xi.astype(np.float64), logu.astype(np.float64), c["eps"], n_iter=1)
    return time.perf_counter() - t0


def c3_instances(n=64, seed=0):
    """Batched workload: n mixtures, T ~ U{200..4000}, M in {2,4,8} with N = M, K = 16,
    F = 513, per-instance seeds 1000 + i (same generative model as the other configs)."""
    rng = np.random.default_rng(seed)
    Ts = rng.integers(200, 4001, size=n)
    Ms = rng.choice([2, 4, 8], size=n)
    return [(513, int(T), int(M), int(M), 16, 1000 + i) for i, (T, M) in enumerate(zip(Ts, Ms))]


def run_batched(args):
    """One step = every instance restarted from its seeded state and iterated 50 times, all
    members of one batch (one graph launch per step).  Also times the same step with the
    instances run one after another (sequential: each mixture's iterations finish before the
    next mixture's start), for comparison."""
    import torch
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf as fm
    from paper_1903_03237_gb300.synth import make_mixture
    iters = 50
    inst = c3_instances(args.instances)
    prec, sched = PRECISIONS[FORMS[args.form][0]], FORMS[args.form][1]
    ctxs = []
    for (F, T, M, N, K, sd) in inst:
        mix = make_mixture(F, T, M, N, K, sd)
        ctxs.append(fm.Context(mix.X, N, K, seed=sd, precision=prec, schedule=sched))
    units = sum(F * T * iters for (F, T, M, N, K, sd) in inst)
    batch = fm.Batch(ctxs)

    def step_batched():
        for c in ctxs:
            c.restart()
        batch.iterate(iters)

    def step_sequential():  # one mixture at a time: each finishes before the next starts
        for c in ctxs:
            c.restart()
            c.iterate(iters)
            c.sync()

    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for i in range(args.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            tot += time.perf_counter() - t0
        return tot
    t_u = timed(step_batched)           # launch shapes as planned for each mixture alone
    batch.sync()
    tune_speedup = batch.autotune(2)    # one split scale for all members, timed on the batch
    l0 = sum(c.launch_count() for c in ctxs)
    t_b = timed(step_batched)
    launches = sum(c.launch_count() for c in ctxs) - l0
    batch.sync()
    t_s = timed(step_sequential)
    for c in ctxs:
        c.sync()
    value = units * args.steps / t_b
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_b / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.form], "data": "synthetic",
        "config": {"workload": f"batched: {len(inst)} mixtures, T ~ U{{200..4000}}, M in {{2,4,8}}, N = M, K 16, "
                               f"F 513, {iters} iterations each, one graph launch per step, autotuned split scale",
                   "l2": "flushed between timed steps (512 MB write)", "form": args.form},
        "sequential_value": units * args.steps / t_s, "batched_over_sequential": t_s / t_b,
        "untuned_value": units * args.steps / t_u, "tuned_over_untuned": t_u / t_b,
        "tuner_trial_speedup": tune_speedup, "tuned_scales": ctxs[0].get_tuning(),
        "gpu_launches": launches,
    }), flush=True)
    batch.close()


def serving_replay(fm, requests, rate, max_active, form, iters=50):
    """Serving workload: Poisson arrivals (arrival seed 7; rate 0 = every request queued at
    once); each request M 4, N 3, K 16, F 513, T = min(6000, round(exp(ln 375 + 0.6 Z))),
    per-request seed 2000 + i, `iters` iterations then the Wiener separation.  Requests are
    submitted at their arrival times; latency = completion - arrival.  Runs the
    continuous-batching server and, for comparison, the same arrivals served one request at a
    time (FIFO, max_active 1).  Returns both summaries."""
    from paper_1903_03237_gb300.synth import make_mixture
    R = requests
    rng = np.random.default_rng(7)
    gaps = rng.exponential(1.0 / 20.0, size=R)
    arrivals = np.cumsum(gaps) - gaps[0]
    if rate > 0:
        arrivals = arrivals * (20.0 / rate)
    else:  # capacity: every request queued at once
        arrivals = np.zeros(R)
    Ts = np.minimum(6000, np.round(np.exp(np.log(375.0) + 0.6 * rng.standard_normal(R)))).astype(int)
    Ts = np.maximum(Ts, 8)
    # mixtures: slices of a few long seeded draws (the generator's cost stays out of the loop)
    pool = [make_mixture(513, int(Ts.max()), 4, 3, 16, 2000 + i).X for i in range(4)]
    reqs = [np.ascontiguousarray(pool[i % 4][:, :T, :]) for i, T in enumerate(Ts)]

    def serve(ma):
        with fm.Server(max_active=ma, iters_per_step=10, precision=PRECISIONS[FORMS[form][0]]) as srv:
            ids = []
            t0 = time.perf_counter()
            for i in range(R):
                now = time.perf_counter() - t0
                if arrivals[i] > now:
                    time.sleep(arrivals[i] - now)
                ids.append(srv.submit(reqs[i], 3, 16, iters, seed=2000 + i))
            lat, done_units, failed = [], 0.0, {}
            for i, j in enumerate(ids):
                srv.wait(j, 600.0)
                st, l = srv.poll(j)
                try:
                    srv.result(j)
                except fm.FastMNMFError as e:  # e.g. a very short request whose model degenerates
                    name = fm.STATUS_NAMES.get(e.status, str(e.status))
                    failed[name] = failed.get(name, 0) + 1
                    continue
                lat.append(l)
                done_units += 513 * int(Ts[i]) * iters
            wall = time.perf_counter() - t0
        lat = np.array(lat)
        return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "throughput": done_units / wall, "wall_s": wall, "completed": int(len(lat)), "failed": failed}

    return serve(max_active), serve(1)


def run_serving(args):
    """--workload c4: the serving replay at its full length (2000 requests by default)."""
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf as fm
    R = args.requests
    cb, fifo = serving_replay(fm, R, args.rate, args.max_active, args.form)
    print(json.dumps({
        "metric": METRIC, "value": cb["throughput"], "unit": UNIT, "n_gpus": 1, "steps": R, "warmup": 0,
        "ms_per_step": 1e3 * cb["wall_s"] / R, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.form], "data": "synthetic",
        "config": {"workload": f"serving: {R} requests, Poisson {args.rate:g}/s, M4 N3 K16 F513, T lognormal (median 375, "
                               "sigma 0.6, cap 6000), 50 iterations + Wiener each",
                   "max_active": args.max_active, "iters_per_step": 10, "form": args.form},
        "latency_p50_ms": cb["p50_ms"], "latency_p99_ms": cb["p99_ms"],
        "completed": cb["completed"], "failed": cb["failed"],
        "fifo": fifo,
    }), flush=True)


def profile_run(args):
    """A short run of the same workload for ncu captures: context, 3 iterations, separation
    (``--bins`` overrides F to keep the device footprint of a capture small)."""
    import torch
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf as fm
    from paper_1903_03237_gb300.synth import make_mixture
    if args.workload == "dp":
        # FastMNMF-DP at the paper's setting: 4 iterations with device-resident draws
        from paper_1903_03237_gb300.synth import make_dp_state, make_decoder, make_dp_draws
        c = DP_SETTING
        F, T, M, N, K, Dd, Hd, S = c["F"], c["T"], c["M"], c["N"], c["K"], c["D"], c["Hd"], c["S"]
        xi, logu = make_dp_draws(4, S, T, Dd, 0)
        with fm.DPContext(make_mixture(F, T, M, N, K, 0).X, N, K, D=Dd, Hd=Hd, n_proposals=S, eps=c["eps"]) as dp:
            dp.set_decoder(*make_decoder(F, Dd, Hd, 0))
            dp.set_state(*make_dp_state(F, T, M, N, K, Dd, 0))
            dp.iterate(4, torch.from_numpy(xi).cuda(), torch.from_numpy(logu).cuda())
            print("profile run ok, log-likelihood", dp.loglik(), "accepted", dp.accepted())
        return
    w = WORKLOAD
    F = args.bins or w["F"]
    mix = make_mixture(F, w["T"], w["M"], w["N"], w["K"], 0, diffuse_frac=w["diffuse"])
    with fm.Context(mix.X, w["N"], w["K"], seed=0, precision=PRECISIONS[FORMS[args.form][0]],
                    schedule=FORMS[args.form][1]) as ctx:
        ctx.iterate(3)
        ctx.separate()
        print("profile run ok, log-likelihood", ctx.loglik())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-run", action="store_true", help="short run for ncu captures, no JSON line")
    ap.add_argument("--bins", type=int, default=0, help="--profile-run: number of frequency bins (default: the workload's)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["c3", "c4", "dp"], default="c1",
                    help="c1 (default, the headline line), c2 (large mixture), c3 (batched mixtures), c4 (serving), "
                         "dp (FastMNMF-DP at the paper's setting; with --profile-run only)")
    ap.add_argument("--requests", type=int, default=2000, help="c4: number of requests")
    ap.add_argument("--max-active", type=int, default=16, help="c4: resident requests")
    ap.add_argument("--rate", type=float, default=20.0,
                    help="c4: arrival rate in requests/s (the same arrival pattern, rescaled); 0 = all at once")
    ap.add_argument("--instances", type=int, default=64, help="c3: number of mixtures")
    ap.add_argument("--form", choices=sorted(FORMS), default="bf16",
                    help="form to time: bf16 (default: split-BF16 tensor-core contractions), fused (FP32, bin-fused "
                         "schedule), sweep (plain FP32), tf32")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP32 comparison run")
    ap.add_argument("--no-autotune", action="store_true", help="keep the planned launch shapes (no tuner run)")
    ap.add_argument("--no-serving", action="store_true", help="skip the bounded serving replay of the default run")
    ap.add_argument("--no-dp", action="store_true", help="skip the FastMNMF-DP measurement of the default run")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = WORKLOADS.get(args.workload, WORKLOADS["c1"])
    if args.workload == "dp" and not args.profile_run:
        ap.error("--workload dp is a --profile-run workload; the default line measures FastMNMF-DP under fastmnmf_dp")
    if args.profile_run:
        profile_run(args)
    elif args.workload == "c3":
        run_batched(args)
    elif args.workload == "c4":
        run_serving(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
