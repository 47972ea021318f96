"""Benchmark of the m-Cubes VEGAS hot path on GB300.

One step = one VEGAS iteration of the whole hot path (sampling launch +
refinement/weighting launch) over one batch of N = m * p synthetic samples.
Default workload: the d=6 power-law x lognormal x ridge integrand on
[0.05, 2]^6, 1e8 calls per iteration (m = 19^6, p = 2), 500 bins per axis,
plain double precision.  Metric: integrand evaluations per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config cosmo6|gauss3|corner8|osc10] [--ncall C] [--no-cpu-baseline]

Other lines: --config batch4096 (integrals/s of 4096 batched integrals at
rel_tol 1e-4 against plain FP64 one by one), --config serve (Poisson stream
through the continuous-batching server: p50/p99 latency, integrals/s),
--config onedim (m-Cubes1D speed-up on the symmetric suite integrands),
--config accuracy (the Sec. 5.1 tolerance sweep on f2..f6).

Under torchrun (N > 1) every rank integrates its own independent copy of
the workload (own seed) on its own GPU: weak scaling, no collective on the
data path; the value is the samples of all ranks over the slowest rank's time.
--impl reference times the CPU oracle (the method as plainly written) on the
host cores, each step a bounded sample of one iteration.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2202_01753_gb300 import workloads as W  # noqa: E402
from paper_2202_01753_gb300 import closed_forms as CF  # noqa: E402

# Work per sample of the sampling kernel, from the ncu captures summarised in
# profiles/ (the per-unit figures of the roofline), keyed by (config,
# precision).  "fp64": FP64 instructions per sample (DFMA + DADD + DMUL) against
# the FP64 pipe (2 per clk per SM on GB300, ncu peak_sustained), and with
# "issue_per_sample" also all issued instructions against the issue slots, the
# larger fraction reported as the kernel's; "issue": issued warp
# instructions per 32 samples against 4 issue slots/clk/SM.  "traffic": DRAM
# bytes read + written by one full-size launch (one-pass ncu capture of
# dram__bytes_read.sum and dram__bytes_write.sum on the same kernel build).
# "fp32_flops": 2 FFMA + FADD + FMUL per sample (the FP32-pipe fraction shown
# beside the issue fraction).
ROOFLINE_UNITS = {
    ("cosmo6", "fp64"): {"kind": "fp64", "per_sample": 29.86, "issue_per_sample": 2032.5, "traffic": 277.2e3,
                         "pipe_busy": 0.781,
                         "source": "profiles/vsample_cosmo6_fp64.md"},
    ("gauss3", "fp64"): {"kind": "fp64", "per_sample": 26.92, "traffic": 101.4e3, "pipe_busy": 0.783,
                         "source": "profiles/vsample_gauss3_fp64.md"},
    ("table6", "fp64"): {"kind": "fp64", "per_sample": 43.74, "dram_bytes_per_sample": 409.2, "traffic": 38.5028e9,
                         "pipe_busy": 0.734,
                         "source": "profiles/vsample_table6_fp64.md"},
    ("corner8", "mixed"): {"kind": "issue", "per_sample": 533.1, "traffic": 598.8e3, "fp32_flops": 99.08,
                           "source": "profiles/vsample_corner8_mixed.md"},
    ("osc10", "mixed"): {"kind": "issue", "per_sample": 654.3, "traffic": 301.1e3, "fp32_flops": 134.87,
                         "source": "profiles/vsample_osc10_mixed.md"},
}
DFMA_PER_CLK_PER_SM = 2.0



def _measured_hbm_gbs() -> float:
    """HBM copy bandwidth measured on this machine's GPUs (GB/s), else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _measured_hbm_gbs()
ISSUE_PER_CLK_PER_SM = 4.0

L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2: written between timed steps


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cosmo6",
                    choices=sorted(W.CONFIGS) + ["batch4096", "serve", "onedim", "accuracy"])
    ap.add_argument("--sweep-runs", type=int, default=100, help="seeds per tolerance level (accuracy sweep)")
    ap.add_argument("--sweep-ncall0", type=float, default=1e5, help="calls per iteration at tau_rel = 1e-3")
    ap.add_argument("--sweep-ncall-cap", type=float, default=1.7e9, help="largest calls per iteration")
    ap.add_argument("--sweep-seconds", type=float, default=1800.0,
                    help="no deeper level of an integrand starts after its share of this time")
    ap.add_argument("--sweep-precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="length of the configured Poisson stream")
    ap.add_argument("--serve-burst", type=int, default=2000, help="requests offered at once (capacity)")
    ap.add_argument("--serve-steady-seconds", type=float, default=8.0,
                    help="length of the stream at a sustainable fraction of the capacity")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-iters", type=int, default=2, help="iterations per server step")
    ap.add_argument("--batch-n", type=int, default=4096)
    ap.add_argument("--batch-rel-tol", type=float, default=1e-4, help="relative tolerance of every batched integral")
    ap.add_argument("--seq-sample", type=int, default=96, help="integrals timed one by one in plain FP64")
    ap.add_argument("--ncall", type=float, default=None, help="override calls per iteration (profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--multi", default="auto", choices=["auto", "shard", "replicas"],
                    help="auto: N > 1 shards one integral's cubes over the ranks; shard: also at N = 1; "
                         "replicas: an independent integral per rank")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline only: skip the mixed-precision, batch and serving legs of the default run")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def workload(args, rank):
    w = W.CONFIGS[args.config](seed=rank)
    if w.fid == W.F_TABLE:
        w.meta["tables_from"] = (args.config, {"seed": rank})
    if args.ncall:
        w = w.scaled(int(args.ncall))
    return w


# ---------------------------------------------------------------------------
# cross-rank aggregation (weak scaling: every rank integrates its own copy)
# ---------------------------------------------------------------------------
def aggregate_ranks(local_ms, local_samples, device):
    """Whole-job throughput: the samples of all ranks over the slowest rank's
    time.  Returns (samples_per_s, max_ms, total_samples); works on any
    initialised process group (NCCL on GPUs, gloo on CPUs) or none."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(local_samples)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    max_ms, total = float(t.item()), float(n.item())
    return total / (max_ms / 1e3), max_ms, total


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a moment to start: wait for its first sample, so
            # that the samples kept (from here on) cover the timed region
            t_end = time.time() + 5.0
            while not self.lines and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines = self.lines[-1:]
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            t = [x.strip() for x in ln.split(",")]
            if len(t) < 7:
                continue
            try:
                sm.append(float(t[0]))
                smax.append(float(t[1]))
            except ValueError:
                continue
            for n, v in zip(names, t[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands on a bounded sample of the workload
# ---------------------------------------------------------------------------
def _oracle_pass(job):
    """One adjusting oracle pass over cubes [c0, c1) of a workload (runs in a
    spawned worker process); returns (seconds, samples)."""
    import oracle
    spec, c0, c1 = job
    if spec.get("tables_from"):                 # regenerate the (seeded) tables in this process
        name, kw = spec["tables_from"]
        oracle.set_tables(W.CONFIGS[name](**kw).meta["tables"])
    pb = oracle.Problem(spec["fid"], spec["params"], spec["lo"], spec["hi"], spec["ncall"], nb=spec["nb"],
                        g_override=spec["g_override"], seed=spec["seed"])
    B = oracle.init_grid(pb.d, pb.nb)
    t = time.perf_counter()
    pb.vsample(B, 0, True, c0, c1)
    return time.perf_counter() - t, (c1 - c0) * pb.p


def cpu_oracle_rate(w, seconds):
    """The oracle's adjusting pass on the host: one core over a cube range
    sized to about seconds/2, then every core (spawned processes, one cube
    range each) for about seconds/2.  Returns a cpu_baseline object."""
    import multiprocessing as mp

    import oracle
    if w.fid == W.F_TABLE:
        oracle.set_tables(w.meta["tables"])
    pb = oracle.Problem(w.fid, w.params, w.lo, w.hi, w.ncall, nb=w.nb, g_override=w.g_override, seed=w.seed)
    B = oracle.init_grid(pb.d, pb.nb)
    # calibrate on a small range, then one range sized to seconds / 2
    n0 = max(1, min(pb.m, 2000 if pb.p < 100 else 1))
    t = time.perf_counter()
    pb.vsample(B, 0, True, 0, n0)
    dt = max(time.perf_counter() - t, 1e-4)
    n = int(min(pb.m, max(n0, n0 * 0.5 * seconds / dt)))
    t = time.perf_counter()
    pb.vsample(B, 0, True, 0, n)
    dt1 = time.perf_counter() - t
    rate1 = n * pb.p / dt1
    cores = os.cpu_count() or 1
    spec = dict(fid=w.fid, params=[float(v) for v in w.params], lo=[float(v) for v in w.lo],
                hi=[float(v) for v in w.hi], ncall=w.ncall, nb=w.nb, g_override=w.g_override, seed=w.seed,
                tables_from=w.meta.get("tables_from"))
    per = max(1, min(n, pb.m // cores))
    jobs = [(spec, i * per, (i + 1) * per) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_pass, [(spec, 0, 1)] * cores)           # start-up and library load, untimed
        t = time.perf_counter()
        res = pool.map(_oracle_pass, jobs, chunksize=1)
        dtn = time.perf_counter() - t
    samples_n = sum(r[1] for r in res)
    return {"value": samples_n / dtn, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"one adjusting pass over cubes [0, {per * cores}) split into {cores} equal ranges, "
                      f"one process per core ({samples_n} samples, {dtn:.1f} s)",
            "single_core": {"value": rate1, "cores": 1,
                            "sample": f"cubes [0, {n}) ({n * pb.p} samples, {dt1:.1f} s)"}}


def _oracle_pass_it(job):
    """_oracle_pass for a given iteration index (reference arm steps)."""
    import oracle
    spec, c0, c1, it = job
    if spec.get("tables_from"):
        name, kw = spec["tables_from"]
        oracle.set_tables(W.CONFIGS[name](**kw).meta["tables"])
    pb = oracle.Problem(spec["fid"], spec["params"], spec["lo"], spec["hi"], spec["ncall"], nb=spec["nb"],
                        g_override=spec["g_override"], seed=spec["seed"])
    B = oracle.init_grid(pb.d, pb.nb)
    t = time.perf_counter()
    pb.vsample(B, it, True, c0, c1)
    return time.perf_counter() - t, (c1 - c0) * pb.p


def reference_arm(args):
    """The oracle (the method as plainly written) on the host: every step is
    one adjusting pass over a bounded cube range of the workload, split into
    one equal range per host core (spawned processes, started before
    timing)."""
    import multiprocessing as mp

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args, 0)
    import oracle
    g, m, p = oracle.geometry(w.d, w.ncall, w.g_override, w.nb)
    cores = os.cpu_count() or 1
    per = max(1, min(m // cores, (400_000 // p) if p < 1000 else 1))
    spec = dict(fid=w.fid, params=[float(v) for v in w.params], lo=[float(v) for v in w.lo],
                hi=[float(v) for v in w.hi], ncall=w.ncall, nb=w.nb, g_override=w.g_override, seed=w.seed,
                tables_from=w.meta.get("tables_from"))
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_pass_it, [(spec, 0, 1, 0)] * cores)      # start-up and library load, untimed
        for i in range(args.warmup):
            pool.map(_oracle_pass_it, [(spec, c * per, (c + 1) * per, i) for c in range(cores)], chunksize=1)
        t = time.perf_counter()
        for i in range(args.steps):
            pool.map(_oracle_pass_it, [(spec, c * per, (c + 1) * per, args.warmup + i) for c in range(cores)],
                     chunksize=1)
        dt = time.perf_counter() - t
    samples = per * cores * p * args.steps
    value = samples / dt
    line = {
        "impl": "reference", "metric": "integrand evaluations per second", "value": value,
        "unit": "evals/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "d": w.d, "ncall": w.ncall, "nbins": w.nb,
                   "sample_per_step": f"cubes [0, {per * cores}) of one iteration ({per * cores * p} samples) "
                                      f"in {cores} equal ranges, one process per core"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per * cores * p} samples per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# the mixed-precision configurations (d=8 corner peak, d=10 oscillatory at
# 1e9 calls per iteration): evaluations/s, issue and FP32 fractions, and the
# error against the FP64 oracle on a sampled cube range
# ---------------------------------------------------------------------------
MIXED_ORACLE_CUBES = 200_000


def mixed_oracle_sample(w, ctx, c0, n):
    """The FP64 oracle's pass over cubes [c0, c0 + n) of iteration 0 on the
    uniform grid (timed: the CPU baseline of this configuration), and the
    relative differences of the GPU mixed pass over the same cubes."""
    import numpy as np

    import oracle
    pb = oracle.Problem(w.fid, w.params, w.lo, w.hi, w.ncall, nb=w.nb, g_override=w.g_override, seed=w.seed)
    B = oracle.init_grid(pb.d, pb.nb)
    t = time.perf_counter()
    o_sums, o_C, _, _ = pb.vsample(B, 0, True, c0, c0 + n)
    dt = time.perf_counter() - t
    g_sums, g_C = ctx.sample_range(0, True, c0, c0 + n)
    o_C = np.asarray(o_C).reshape(w.d, w.nb)
    return {
        "error_vs_fp64_oracle": {
            "sum_of_cube_means_rel": abs(g_sums[0] - o_sums[0]) / abs(o_sums[0]),
            "sum_of_cube_means_rel_to_sum_abs": abs(g_sums[0] - o_sums[0]) / abs(o_sums[2]),
            "sum_of_cube_variances_rel": abs(g_sums[1] - o_sums[1]) / abs(o_sums[1]),
            "histogram_max_rel": float(np.max(np.abs(g_C - o_C) / np.maximum(np.abs(o_C), 1e-300))),
            "sample": f"cubes [{c0}, {c0 + n}) of iteration 0 on the uniform grid ({n * pb.p} samples)"},
        "cpu_baseline": {"value": n * pb.p / dt, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": f"one adjusting FP64 pass over cubes [{c0}, {c0 + n}) ({n * pb.p} samples, "
                                   f"{dt:.1f} s)"},
    }


def mixed_leg(args, name, local, stream, sms, steps):
    import torch

    from paper_2202_01753_gb300 import mcubes

    w = W.CONFIGS[name](seed=0)
    ctx = mcubes.Context(local, stream=stream.cuda_stream, nbins=w.nb, g_override=w.g_override, seed=w.seed,
                         precision=w.precision, ita=-1)
    ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, itmax=3 + steps)
    geom = ctx.geometry()
    N = geom["m"] * geom["p"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ctx.iterate(3)
    torch.cuda.synchronize()
    ctx.timing_reset(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(local)
    clocks.start()
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        ctx.iterate(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    kt = ctx.timing()
    res = ctx.result()
    ctx.close()
    sample_ms = kt["sample_ms"] / max(kt["sample_launches"], 1)
    unit = ROOFLINE_UNITS[(name, "mixed")]
    sm_mhz = clk.get("sm_mhz") or 0.0
    out = {"workload": w.name, "d": w.d, "ncall": w.ncall, "g": geom["g"], "m": geom["m"], "p": geom["p"],
           "samples_per_step": N, "evals_per_s": N / (step_ms / 1e3), "ms_per_step": step_ms,
           "sample_ms_avg": sample_ms, "steps": steps, "warmup": 3, "precision": "mixed",
           "l2": "flushed between timed steps (256 MB write)",
           "estimate": res["estimate"], "sigma": res["sigma"], "clocks": clk}
    if sm_mhz:
        t = sample_ms / 1e3
        issue = unit["per_sample"] * (N / 32.0) / t / (ISSUE_PER_CLK_PER_SM * sms * sm_mhz * 1e6)
        fp32 = unit["fp32_flops"] * N / t / (2 * 128 * sms * sm_mhz * 1e6)
        out["roofline"] = {"bound": "alu", "pipe": "issue", "frac": issue, "fp32_pipe_frac": fp32,
                           "per_sample": f"{unit['per_sample']} thread-instructions, {unit['fp32_flops']} FP32 "
                                         f"flops ({unit['source']})"}
    if not args.no_cpu_baseline:
        ctx2 = mcubes.Context(local, nbins=w.nb, g_override=w.g_override, seed=w.seed, precision="mixed")
        ctx2.setup(w.fid, w.params, w.lo, w.hi, w.ncall, itmax=1)
        c0 = geom["m"] // 2
        out.update(mixed_oracle_sample(w, ctx2, c0, min(MIXED_ORACLE_CUBES, geom["m"] - c0)))
        ctx2.close()
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def ours(args):
    import torch
    import torch.distributed as dist

    from paper_2202_01753_gb300 import build, mcubes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # N > 1: one integral sharded over the ranks by cube range (every rank the
    # same problem and seed), or with --multi replicas an independent copy per
    # rank; --multi shard also runs the sharded path (NCCL included) on one GPU
    sharded = args.multi == "shard" or (world > 1 and args.multi == "auto")
    if world > 1 or sharded:
        for k, v in (("MASTER_ADDR", "127.0.0.1"), ("MASTER_PORT", "29531"), ("RANK", "0"), ("WORLD_SIZE", "1")):
            os.environ.setdefault(k, v)
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    w = workload(args, 0 if sharded else rank)
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.current_stream()
    prec = w.precision

    def make_ctx(on_stream):
        c = mcubes.Context(local, stream=stream.cuda_stream if on_stream else None, nbins=w.nb,
                           g_override=w.g_override, seed=w.seed, precision=prec, ita=-1)
        if w.fid == W.F_TABLE:
            c.set_tables(w.meta["tables"])       # resident state, uploaded once before timing
        return c

    ctx = make_ctx(True)
    ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, itmax=Wm + K)
    geom = ctx.geometry()
    N = geom["m"] * geom["p"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    if sharded:
        from paper_2202_01753_gb300.shard import cube_ranges
        c0, c1 = cube_ranges(geom["m"], world)[rank]
        plen = ctx.shard_partial_len()
        part = torch.zeros(plen, dtype=torch.float64, device="cuda")
        gathered = torch.zeros(world * plen, dtype=torch.float64, device="cuda")
        local_N = (c1 - c0) * geom["p"]

        def step(c):
            c.shard_sample(c0, c1, part.data_ptr())
            dist.all_gather_into_tensor(gathered, part)   # NCCL, on the context's stream
            c.shard_finish(gathered.data_ptr(), world)
    else:
        local_N = N

        def step(c):
            c.iterate(1)

    for _ in range(Wm):
        step(ctx)
    torch.cuda.synchronize()
    ctx.timing_reset(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(K):
        flush.fill_(float(k))                 # L2 flush, outside the timed pair
        ev[k][0].record(stream)
        step(ctx)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    kt = ctx.timing()
    res = ctx.result()
    ctx.close()

    # slowest rank's time, all ranks' samples
    value, t_max, _ = aggregate_ranks(total_ms, local_N * K, "cuda")

    # end to end through the public calls with host buffers (copies inside)
    ctx2 = make_ctx(sharded)
    if sharded:
        ctx2.setup(w.fid, w.params, w.lo, w.hi, w.ncall, 2)
        for _ in range(2):
            step(ctx2)                        # warm
        ctx2.result()
        dist.barrier()
        t0 = time.perf_counter()
        ctx2.setup(w.fid, w.params, w.lo, w.hi, w.ncall, K)
        for _ in range(K):
            step(ctx2)
        r2 = ctx2.result()
    else:
        ctx2.integrate(w.fid, w.params, w.lo, w.hi, w.ncall, 2)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r2 = ctx2.integrate(w.fid, w.params, w.lo, w.hi, w.ncall, K)
    e2e_s = time.perf_counter() - t0
    ctx2.close()
    e2e_value, _, _ = aggregate_ranks(e2e_s * 1e3, local_N * K, "cuda")
    h2d = 8 * (len(w.params) + 2 * w.d)
    d2h = 88

    if rank != 0:
        if dist.is_initialized():
            dist.destroy_process_group()
        return 0

    from paper_2202_01753_gb300 import peaks
    pk = peaks.measure(local)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    avg_sample_ms = kt["sample_ms"] / max(kt["sample_launches"], 1)
    unit = ROOFLINE_UNITS.get((args.config, prec))
    sm_mhz = clk.get("sm_mhz") or 0.0
    t_launch = avg_sample_ms / 1e3
    if unit and unit["kind"] == "fp64" and sm_mhz:
        peak = DFMA_PER_CLK_PER_SM * sms * sm_mhz * 1e6 / 1e12              # T FP64 instructions/s
        achieved = unit["per_sample"] * local_N / t_launch / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP64-inst/s",
                "frac": achieved / peak, "traffic": unit.get("traffic"), "pipe": "fp64",
                "peak_how": "2 FP64 instructions/clk/SM (ncu peak_sustained) x SMs x median SM clock under load",
                "measured_dfma_per_s": pk["dfma_per_s"],
                "per_sample": f"{unit['per_sample']} FP64 instructions, DFMA+DADD+DMUL ({unit['source']})"}
        if unit.get("pipe_busy"):
            roof["ncu_fp64_pipe_busy"] = unit["pipe_busy"]   # sm__pipe_fp64_cycles_active, same kernel
        if unit.get("issue_per_sample"):
            # the kernel's time is bounded by its FP64 instructions on the FP64
            # pipe and by all its instructions on the issue slots; the larger
            # fraction is the limit it runs against
            ipeak = ISSUE_PER_CLK_PER_SM * sms * sm_mhz * 1e6 / 1e9          # G warp-instructions/s
            iach = unit["issue_per_sample"] * (local_N / 32.0) / t_launch / 1e9
            roof["fractions"] = {
                "fp64": {"frac": achieved / peak, "achieved": achieved, "peak": peak, "unit": "T FP64-inst/s"},
                "issue": {"frac": iach / ipeak, "achieved": iach, "peak": ipeak, "unit": "Gwarp-inst/s",
                          "per_sample": f"{unit['issue_per_sample']} thread-instructions ({unit['source']})",
                          "peak_how": "4 warp-instructions/clk/SM x SMs x median SM clock under load"}}
            if iach / ipeak > achieved / peak:
                roof.update({"achieved": iach, "peak": ipeak, "unit": "Gwarp-inst/s", "frac": iach / ipeak,
                             "pipe": "issue", "peak_how": roof["fractions"]["issue"]["peak_how"],
                             "per_sample": roof["fractions"]["issue"]["per_sample"]})
        if unit.get("dram_bytes_per_sample"):
            hbm = unit["dram_bytes_per_sample"] * local_N / t_launch / 1e9
            roof["hbm"] = {"achieved_gbs": hbm, "peak_gbs": HBM_PEAK_GBS, "frac": hbm / HBM_PEAK_GBS,
                           "bytes_per_sample": unit["dram_bytes_per_sample"],
                           "how": "ncu dram__bytes_read+write per launch / samples (full-size one-pass capture)"}
    elif unit and unit["kind"] == "issue" and sm_mhz:
        peak = ISSUE_PER_CLK_PER_SM * sms * sm_mhz * 1e6 / 1e9              # G warp-instructions/s
        achieved = unit["per_sample"] * (local_N / 32.0) / t_launch / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s", "frac": achieved / peak,
                "traffic": unit.get("traffic"), "pipe": "issue",
                "peak_how": "4 warp-instructions/clk/SM x SMs x median SM clock under load",
                "per_sample": f"{unit['per_sample']} thread-instructions ({unit['source']})"}
        if unit.get("fp32_flops"):
            fp32_peak = 2 * 128 * sms * sm_mhz * 1e6 / 1e12          # TFLOP/s: 128 FFMA lanes/SM
            fp32 = unit["fp32_flops"] * local_N / t_launch / 1e12
            roof["fp32"] = {"achieved_tflops": fp32, "peak_tflops": fp32_peak, "frac": fp32 / fp32_peak,
                            "flops_per_sample": unit["fp32_flops"],
                            "how": "(2 FFMA + FADD + FMUL) per sample from ncu x samples / kernel time against "
                                   "128 FMA lanes x 2 x SMs x clock"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "note": "no ncu per-sample count recorded for this configuration"}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_oracle_rate(w, args.cpu_seconds)

    # the metric's other parts, on the same GPU after the headline: the
    # mixed-precision configurations, the batch of 4096 integrals and the
    # served stream
    extra = {}
    if args.config == "cosmo6" and world == 1 and not args.no_extra and not args.ncall:
        steps_x = max(3, min(K, 10))
        extra["mixed_precision"] = {n: mixed_leg(args, n, local, stream, sms, steps_x) for n in ("corner8", "osc10")}
        extra["batch"] = batch_leg(args, local)
        extra["serving"] = serve_leg(args, local)

    line = {
        "metric": "integrand evaluations per second", "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": K, "warmup": Wm, "ms_per_step": t_max / K, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": w.name, "d": w.d, "ncall": w.ncall, "g": geom["g"], "m": geom["m"], "p": geom["p"],
                   "samples_per_step": N, "nbins": w.nb, "precision": prec, "adjusting": True,
                   "lanes_per_cube": geom["lanes"], "blocks": geom["blocks"],
                   "parallelism": (f"one integral, cube ranges over {world} GPUs, rank-order all-gather of the "
                                   f"partials per iteration" if sharded else
                                   (f"{world} independent replicas" if world > 1 else "single GPU")),
                   "l2": "flushed between timed steps (256 MB write)",
                   **({"table_bytes": w.meta["table_bytes"], "tables": "resident, uploaded once before timing"}
                      if w.fid == W.F_TABLE else {})},
        "kernel": {"sample_ms_avg": avg_sample_ms, "refine_ms_avg": kt["refine_ms"] / max(kt["refine_launches"], 1),
                   "sample_launches": kt["sample_launches"], "refine_launches": kt["refine_launches"]},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
                "call": "mcubes_integrate (host params/bounds/result), %d iterations" % K},
        # sampling + refinement per iteration; sharded also the range reduction and the rank-order combine
        "gpu_launches": (kt["sample_launches"] + kt["refine_launches"]) * (2 if sharded else 1),
        "clocks": clk,
        "alu_peaks": {"ffma_tflops": 2 * pk["ffma_per_s"] / 1e12, "dfma_tflops": 2 * pk["dfma_per_s"] / 1e12,
                      "fp64_inst_per_clk_per_sm": {k: pk[f"{k}_per_s"] / (sms * sm_mhz * 1e6) if sm_mhz else None
                                                   for k in ("dfma", "dadd", "dmul")},
                      "how": "independent FMA chains on every thread of 8 blocks/SM, CUDA events"},
        "result": {"estimate": res["estimate"], "sigma": res["sigma"], "chi2_dof": res["chi2_dof"],
                   "e2e_estimate": r2["estimate"]},
        **extra,
    }
    print(json.dumps(line))
    if dist.is_initialized():
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# retries with more calls for integrals that end unconverged (the accuracy
# protocol of Sec. 5.1 raises the sample count for tighter tolerances)
# ---------------------------------------------------------------------------
RETRY_MIN, RETRY_MAX = 2.0, 64.0     # retry factor range: ncall x 2 (sigma/tau)^2, clamped
BATCH_NCALL_MAX = 64_000_000
SERVE_NCALL_MAX = 102_400_000
SERVE_LOAD = 0.75                   # the steady stream's rate, as a fraction of the measured capacity
RETRY_RULE = (f"unconverged after itmax: fresh run with ncall x 2 (sigma/tau)^2, the factor clamped to "
              f"[{RETRY_MIN:g}, {RETRY_MAX:g}]")


def _req(w, ncall, tol):
    return dict(fid=w.fid, params=w.params, lo=w.lo, hi=w.hi, ncall=ncall, itmax=w.itmax, rel_tol=tol, seed=w.seed)


def _retry(ncall, r, tol, ncall_max):
    from paper_2202_01753_gb300.retry import retry_ncall
    if r["converged"] or r["status"] != 5 or ncall >= ncall_max:
        return ncall
    return retry_ncall(ncall, r["estimate"], r["sigma"], tol, 0.0, RETRY_MIN, RETRY_MAX, ncall_max)


def batch_escalated(ctx, ws, tol, ncall_max):
    """Batched integration with retries: every round integrates the still
    unconverged integrals in one batch with their calls sized by the retry
    rule (paper_2202_01753_gb300.retry, the server's).  Returns (final
    results, wall seconds, rounds, samples drawn)."""
    out = [None] * len(ws)
    ncall = [w.ncall for w in ws]
    todo = list(range(len(ws)))
    rounds, samples = 0, 0
    t0 = time.perf_counter()
    while todo:
        res = ctx.integrate_batch([_req(ws[i], ncall[i], tol) for i in todo])
        rounds += 1
        nxt = []
        for i, r in zip(todo, res):
            out[i] = r
            samples += r["samples_per_iter"] * r["iterations"]
            more = _retry(ncall[i], r, tol, ncall_max)
            if more > ncall[i]:
                ncall[i] = more
                nxt.append(i)
        todo = nxt
    return out, time.perf_counter() - t0, rounds, samples


def solo_escalated(ctx, w, tol, ncall_max):
    """The same rule for one integral in plain FP64 (one context call per try)."""
    ncall = w.ncall
    while True:
        ctx.set_opts(seed=w.seed)
        r = ctx.integrate(w.fid, w.params, w.lo, w.hi, ncall, w.itmax, tol)
        more = _retry(ncall, r, tol, ncall_max)
        if more <= ncall:
            return r
        ncall = more


def oracle_per_result(ws, results, tols, ncall_max_samples, k):
    """The CPU baseline of a batched or served leg, and each sampled result's
    error against the FP64 oracle: the oracle integrates (one core, timed)
    up to k of the integrals that converged on their first run with at most
    ncall_max_samples calls per iteration x itmax -- the same request, seed
    and samples as the GPU's mixed-precision run -- and the relative
    difference of the estimates, max(|I|, sigma) of the oracle's as scale,
    is reported per result where both ran the same iterations."""
    import oracle
    pick = []
    for i, (w, r) in enumerate(zip(ws, results)):
        if len(pick) >= k:
            break
        if not r["converged"] or w.ncall * w.itmax > ncall_max_samples:
            continue
        g, m, p = oracle.geometry(w.d, w.ncall, 0, w.nb)
        if r["samples_per_iter"] == m * p:            # no retry: the request's own calls
            pick.append(i)
    errs, n_same, samples = [], 0, 0
    t = time.perf_counter()
    outs = [oracle.integrate(ws[i].fid, ws[i].params, ws[i].lo, ws[i].hi, ws[i].ncall, ws[i].itmax, nb=ws[i].nb,
                             seed=ws[i].seed, rel_tol=tols[i]) for i in pick]
    dt = time.perf_counter() - t
    for i, o in zip(pick, outs):
        samples += o["m"] * o["p"] * o["iterations"]
        if o["iterations"] == results[i]["iterations"]:
            n_same += 1
            errs.append(abs(results[i]["estimate"] - o["estimate"]) / max(abs(o["estimate"]), o["sigma"]))
    return {
        "error_vs_fp64_oracle": {
            "per_result": errs, "max": max(errs) if errs else None,
            "median": statistics.median(errs) if errs else None,
            "sample": f"{len(pick)} converged results without retries ({n_same} with the oracle's iteration "
                      f"count; the estimates' difference relative to max(|I|, sigma))"},
        "cpu_baseline": {"value": len(pick) / dt if dt > 0 else None, "unit": "integrals/s", "cores": 1,
                         "kind": "oracle", "evals_per_s": samples / dt if dt > 0 else None,
                         "sample": f"the same {len(pick)} integrals, one process ({dt:.1f} s)"},
    }


# ---------------------------------------------------------------------------
# batched integrals: integrals/s at rel_tol of the batched mixed-precision
# path against the plain per-integral FP64 path on the same GPU
# ---------------------------------------------------------------------------
def batch_leg(args, local):
    import torch

    from paper_2202_01753_gb300 import mcubes

    ws = W.batch4096(n=args.batch_n)
    tol = args.batch_rel_tol
    ctx = mcubes.Context(local, precision="mixed")
    ctx.integrate_batch([_req(w, w.ncall, tol) for w in ws[:64]])   # warm-up (autotune, graph capture)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    out, t_batch, rounds, samples = batch_escalated(ctx, ws, tol, BATCH_NCALL_MAX)
    clk = clocks.stop()
    ctx.close()
    conv = [bool(o["converged"]) for o in out]
    # plain FP64, one integral at a time with the same retry rule, on an evenly spaced sample
    step = max(1, len(ws) // args.seq_sample)
    idx = list(range(0, len(ws), step))[: args.seq_sample]
    solo = mcubes.Context(local, precision="fp64")
    solo.integrate(ws[0].fid, ws[0].params, ws[0].lo, ws[0].hi, ws[0].ncall, 2)
    t_seq, rel, seq_conv = 0.0, [], []
    for i in idx:
        t0 = time.perf_counter()
        r = solo_escalated(solo, ws[i], tol, BATCH_NCALL_MAX)
        t_seq += time.perf_counter() - t0
        seq_conv.append(bool(r["converged"]))
        if r["converged"] and conv[i]:
            rel.append(abs(out[i]["estimate"] - r["estimate"]) / max(abs(r["estimate"]), r["sigma"]))
    solo.close()
    n_conv = sum(conv)
    seq_conv_per_s = sum(seq_conv) / t_seq
    cpu = oracle_per_result(ws, out, [tol] * len(ws), 2_000_000, 12) if not args.no_cpu_baseline else {}
    return {
        "integrals_per_s_at_tol": n_conv / t_batch, "unit": "integrals/s",
        "rel_tol": tol, "integrals": len(ws), "converged": n_conv, "converged_fraction": n_conv / len(ws),
        "unconverged_fraction": 1.0 - n_conv / len(ws), "seconds": t_batch, "rounds": rounds,
        "evals_per_s": samples / t_batch, "precision": "mixed",
        "retry_rule": f"{RETRY_RULE}, calls <= {BATCH_NCALL_MAX:.3g}",
        "sequential_fp64": {"integrals_per_s_at_tol": seq_conv_per_s, "sample": f"{len(idx)} integrals",
                            "converged_fraction": statistics.mean(seq_conv),
                            "batched_converged_fraction_same_sample": statistics.mean([conv[i] for i in idx]),
                            "speedup_of_batched": (n_conv / t_batch) / seq_conv_per_s if seq_conv_per_s else None,
                            "max_rel_diff_of_estimates": max(rel) if rel else None,
                            "median_rel_diff": statistics.median(rel) if rel else None},
        **cpu,
        "clocks": clk,
    }


def batch_arm(args):
    import torch

    from paper_2202_01753_gb300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    leg = batch_leg(args, local)
    line = {
        "metric": "integrals per second at the relative tolerance", "value": leg["integrals_per_s_at_tol"],
        "unit": "integrals/s", "n_gpus": 1, "steps": leg["rounds"], "warmup": 1,
        "ms_per_step": 1e3 * leg["seconds"] / leg["rounds"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"batch{leg['integrals']}", "integrals": leg["integrals"], "itmax": 10,
                   "rel_tol": leg["rel_tol"], "precision": "mixed"},
        **{k: v for k, v in leg.items() if k not in ("clocks",)}, "clocks": leg["clocks"],
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# serving: a Poisson stream of requests through the continuous-batching
# server, latency percentiles and integrals/s at each request's tolerance,
# against plain FP64 one by one
# ---------------------------------------------------------------------------
def serve_leg(args, local):
    """Three runs of the server on requests of the serving distribution, with
    the retry rule: its capacity (a burst offered at once), the configured
    Poisson stream (offered rate args.serve_rate, which can exceed the
    capacity: then its latencies are queueing time), and a Poisson stream at
    SERVE_LOAD of the measured capacity, whose latencies are the server's."""
    import numpy as np

    from paper_2202_01753_gb300 import mcubes

    ctx = mcubes.Context(local, precision="mixed")
    srv = mcubes.Server(ctx, itcap=20)
    srv.set_step_iterations(args.serve_iters)
    srv.set_retry_sized(RETRY_MIN, RETRY_MAX, SERVE_NCALL_MAX)
    pct = lambda a, q: 1e3 * float(np.percentile(a, q)) if len(a) else None  # noqa: E731

    def run(stream, at_once=False):
        ws = [w for _, w in stream]
        arrival = np.zeros(len(ws)) if at_once else np.array([t for t, _ in stream])
        res, lat, wall = srv.run_stream([_req(w, w.ncall, w.rel_tol) for w in ws], arrival)
        conv = np.array([bool(r["converged"]) for r in res])
        lat_c = lat[conv]
        return ws, res, {
            "requests": len(ws), "seconds": wall, "integrals_per_s_at_tol": float(conv.sum()) / wall,
            "converged_fraction": float(conv.mean()), "unconverged_fraction": float(1.0 - conv.mean()),
            "retried_requests": int(sum(r["samples_per_iter"] > w.ncall for w, r in zip(ws, res))),
            "latency_ms_converged": {"p50": pct(lat_c, 50), "p99": pct(lat_c, 99), "p99.9": pct(lat_c, 99.9),
                                     "max": 1e3 * float(lat_c.max()) if len(lat_c) else None},
            "latency_ms_all": {"p50": pct(lat, 50), "p99": pct(lat, 99), "p99.9": pct(lat, 99.9),
                               "max": 1e3 * float(lat.max())}}

    # warm-up on requests of the same distribution, offered at once: every
    # kernel class is loaded and captured and the launch shape tuned (the
    # tuner waits for 32 live integrals) before anything is timed
    run(W.serving_stream(rate=args.serve_rate, duration=0.25, draw_seed=7206), at_once=True)
    clocks = ClockSampler(local)
    clocks.start()
    _, _, cap = run(W.serving_stream(rate=args.serve_rate, duration=args.serve_burst / args.serve_rate,
                                     draw_seed=8206), at_once=True)
    ws_o, res_o, over = run(W.serving_stream(rate=args.serve_rate, duration=args.serve_seconds))
    rate = SERVE_LOAD * cap["integrals_per_s_at_tol"]
    _, _, steady = run(W.serving_stream(rate=rate, duration=args.serve_steady_seconds, draw_seed=9206))
    clk = clocks.stop()
    srv.close()
    ctx.close()
    # plain FP64, one request at a time with the same retry rule, on an evenly
    # spaced sample of the configured stream
    idx = list(range(0, len(ws_o), max(1, len(ws_o) // args.seq_sample)))[: args.seq_sample]
    solo = mcubes.Context(local, precision="fp64")
    t_seq, rel, seq_conv = 0.0, [], []
    for i in idx:
        t0 = time.perf_counter()
        r = solo_escalated(solo, ws_o[i], ws_o[i].rel_tol, SERVE_NCALL_MAX)
        t_seq += time.perf_counter() - t0
        seq_conv.append(bool(r["converged"]))
        if r["converged"] and res_o[i]["converged"]:
            rel.append(abs(res_o[i]["estimate"] - r["estimate"]) / max(abs(r["estimate"]), r["sigma"]))
    solo.close()
    seq_rate = sum(seq_conv) / t_seq
    cpu = (oracle_per_result(ws_o, res_o, [w.rel_tol for w in ws_o], 2_000_000, 6)
           if not args.no_cpu_baseline else {})
    return {
        "capacity": {**cap, "offered": "all at once"},
        "offered_stream": {**over, "offered_per_s": args.serve_rate, "stream_seconds": args.serve_seconds},
        "steady_stream": {**steady, "offered_per_s": rate, "stream_seconds": args.serve_steady_seconds,
                          "load": f"{SERVE_LOAD} x the measured capacity"},
        "precision": "mixed", "iterations_per_step": args.serve_iters,
        "request_mix": "d 3..12, rel_tol log-uniform [1e-5, 1e-3], gauss/corner/osc, 1e5 calls x 20 iterations",
        "retry_rule": f"{RETRY_RULE}, ahead of new arrivals, calls <= {SERVE_NCALL_MAX:.3g}",
        "sequential_fp64": {"integrals_per_s_at_tol": seq_rate, "sample": f"{len(idx)} requests of the offered stream",
                            "converged_fraction": statistics.mean(seq_conv),
                            "speedup_of_served_capacity": cap["integrals_per_s_at_tol"] / seq_rate if seq_rate else None,
                            "max_rel_diff_of_estimates": max(rel) if rel else None,
                            "median_rel_diff": statistics.median(rel) if rel else None},
        **cpu,
        "clocks": clk,
    }


def serve_arm(args):
    import torch

    from paper_2202_01753_gb300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    leg = serve_leg(args, local)
    line = {
        "metric": "integrals per second at tolerance (served)", "value": leg["capacity"]["integrals_per_s_at_tol"],
        "unit": "integrals/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * leg["capacity"]["seconds"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "serving", "offered_per_s": args.serve_rate, "seconds": args.serve_seconds,
                   "precision": "mixed", "iterations_per_step": args.serve_iters},
        **{k: v for k, v in leg.items() if k not in ("clocks",)}, "clocks": leg["clocks"],
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# m-Cubes1D (Sec. 3): speed-up over m-Cubes on the suite's symmetric
# integrands, per iteration and to a relative tolerance
# ---------------------------------------------------------------------------
def onedim_arm(args):
    import math

    import torch

    from paper_2202_01753_gb300 import build, mcubes

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    d = 6
    names = ("f2", "f4", "f5")
    ncall_iter = int(args.ncall or 1e8)
    per_iter, to_tol, speedups = {}, [], []
    ctxs = {v: mcubes.Context(local, precision="fp64", one_dim=v) for v in (0, 1)}
    clocks = ClockSampler(local)
    clocks.start()
    for name in names:
        w = W.suite(name, d, ncall=ncall_iter, itmax=10)
        rates = {}
        for v, ctx in ctxs.items():
            ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, 2)
            ctx.iterate(2)                                   # warm-up
            ctx.result()
            ctx.setup(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax)
            ctx.timing_reset(True)
            ctx.iterate(w.itmax)
            ctx.result()
            kt = ctx.timing()
            ctx.timing_reset(False)
            g = ctx.geometry()
            rates[v] = g["m"] * g["p"] * kt["sample_launches"] / (kt["sample_ms"] / 1e3)
        per_iter[name] = {"mcubes_evals_per_s": rates[0], "mcubes1d_evals_per_s": rates[1],
                          "speedup": rates[1] / rates[0]}
        exact = CF.exact(W.suite(name, d))
        for tau in (1e-3, 2e-4, 4e-5, 8e-6):
            ws = W.suite(name, d, ncall=10 ** 7, itmax=60)
            row = {"integrand": name, "tau": tau}
            for v, ctx in ctxs.items():
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = ctx.integrate(ws.fid, ws.params, ws.lo, ws.hi, ws.ncall, ws.itmax, tau)
                dt = time.perf_counter() - t0
                key = "mcubes1d" if v else "mcubes"
                row[key] = {"ms": 1e3 * dt, "iterations": r["iterations"], "converged": r["converged"],
                            "true_rel_err": abs(r["estimate"] - exact) / abs(exact)}
            if row["mcubes"]["converged"] and row["mcubes1d"]["converged"]:
                row["speedup"] = row["mcubes"]["ms"] / row["mcubes1d"]["ms"]
                speedups.append(row["speedup"])
            to_tol.append(row)
    clk = clocks.stop()
    for ctx in ctxs.values():
        ctx.close()
    gmean = math.exp(sum(math.log(x) for x in speedups) / len(speedups)) if speedups else None
    line = {
        "metric": "m-Cubes1D speed-up over m-Cubes (time to relative tolerance)", "value": gmean, "unit": "x",
        "n_gpus": 1, "steps": len(to_tol), "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "suite f2/f4/f5, d=6, [0,1]^6", "precision": "fp64", "ncall_to_tol": 10 ** 7,
                   "itmax_to_tol": 60, "ncall_per_iter_rate": ncall_iter},
        "per_iteration": per_iter, "to_tolerance": to_tol, "clocks": clk,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# accuracy sweep (Sec. 5.1 protocol): f2..f6, tau_rel from 1e-3 divided by 5
# per successful level down to 1e-9; 100 seeds per level run as one batch;
# true relative error against the closed forms
# ---------------------------------------------------------------------------
ACCURACY_SUITE = (("f1", 3), ("f2", 6), ("f3", 3), ("f4", 5), ("f5", 8), ("f6", 6))


def accuracy_arm(args):
    import numpy as np
    import torch

    from paper_2202_01753_gb300 import build, mcubes

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    runs, itmax, ncall_cap = args.sweep_runs, 20, int(args.sweep_ncall_cap)
    ctx = mcubes.Context(local, precision=args.sweep_precision)
    rows, t_total, n_total = [], 0.0, 0
    t_sweep = time.perf_counter()
    stop_reason = {}
    clocks = ClockSampler(local)
    clocks.start()
    budget = args.sweep_seconds / len(ACCURACY_SUITE)   # per integrand
    for name, d in ACCURACY_SUITE:
        exact = CF.exact(W.suite(name, d))
        ncall, tau = int(args.sweep_ncall0), 1e-3
        t_start = time.perf_counter()
        stop_reason[name] = "reached tau 1e-9"
        while tau >= 1e-9:
            tries = 0
            while True:
                ws = [W.suite(name, d, ncall=ncall, itmax=itmax, seed=1000 + r) for r in range(runs)]
                reqs = [dict(fid=w.fid, params=w.params, lo=w.lo, hi=w.hi, ncall=w.ncall, itmax=itmax,
                             rel_tol=tau, seed=w.seed) for w in ws]
                t0 = time.perf_counter()
                out = ctx.integrate_batch(reqs)
                dt = time.perf_counter() - t0
                tries += 1
                conv = np.array([bool(o["converged"]) for o in out], dtype=bool)
                if conv.mean() >= 0.9 or ncall * 4 > ncall_cap or time.perf_counter() - t_start > budget:
                    break
                ncall *= 4                      # more samples for a tighter tolerance (Sec. 5.1)
            t_total += dt
            n_total += runs
            err = np.array([abs(o["estimate"] - exact) / abs(exact) for o in out])
            chi = np.array([o["chi2_dof"] for o in out])
            ok = conv & (chi < 5.0)                     # boolean mask: the runs the paper's plots keep
            row = {"integrand": f"{name},d={d}", "tau": tau, "ncall": ncall, "runs": runs, "tries": tries,
                   "converged": float(conv.mean()), "converged_chi2_lt5": float(ok.mean()),
                   "within_tau": float(np.mean(err[ok] <= tau)) if ok.any() else None,
                   "median_true_rel_err": float(np.median(err[ok])) if ok.any() else None,
                   "median_err_over_tau": float(np.median(err[ok]) / tau) if ok.any() else None,
                   "p90_true_rel_err": float(np.percentile(err[ok], 90)) if ok.any() else None,
                   "median_iterations": float(np.median([o["iterations"] for o in out])),
                   "seconds": dt, "integrals_per_s": runs / dt}
            rows.append(row)
            print(json.dumps({"level": row}), file=sys.stderr, flush=True)
            if conv.mean() < 0.9:
                why = "cap" if ncall * 4 > ncall_cap else "time budget"
                stop_reason[name] = (f"tau {tau:.3g}: {conv.mean():.2f} converged at {ncall:.3g} calls "
                                     f"({why}: cap {ncall_cap:.3g} calls, {budget:.0f} s per integrand)")
                break                           # the level failed: the sweep of this integrand ends
            if time.perf_counter() - t_start > budget:
                stop_reason[name] = f"time budget ({budget:.0f} s per integrand) spent after tau {tau:.3g}"
                break
            tau /= 5.0
            # sigma falls as ncall^-1/2: a tolerance five times tighter needs
            # about 25 times the calls; start two factors of 4 up
            ncall = min(ncall * 16, ncall_cap)
    clk = clocks.stop()
    ctx.close()
    line = {
        "metric": "accuracy sweep: true relative error vs requested tau_rel", "value": n_total / t_total,
        "unit": "integrals/s", "n_gpus": 1, "steps": len(rows), "warmup": 0, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.sweep_precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": "paper suite f1-f6 (Sec. 5 eqs. 1-6)", "dims": dict(ACCURACY_SUITE), "runs": runs,
                   "itmax": itmax, "nbins": 500, "ncall_start": int(args.sweep_ncall0), "ncall_cap": ncall_cap,
                   "precision": args.sweep_precision, "batched": True,
                   "ncall_rule": "next level starts at 16x the last level's calls; x4 while < 90% converge"},
        "stopped": stop_reason, "levels": rows, "clocks": clk, "seconds": time.perf_counter() - t_sweep,
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.config == "accuracy":
        return accuracy_arm(args)
    if args.config == "serve":
        return serve_arm(args)
    if args.config == "onedim":
        return onedim_arm(args)
    if args.config == "batch4096":
        return batch_arm(args)
    if args.impl == "reference":
        return reference_arm(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
