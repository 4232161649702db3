"""Benchmark: Sinkhorn n*r entry-updates per second on the large two-cloud workload.

Workload (one step = the whole hot path once): n = m = 2^20 points in R^3, X
uniform on the unit cube, Y ~ N(0.5*1, 0.1^2 I), uniform weights, eps = 0.1,
r = 1024 Gaussian positive features (Lemma 1), 200 iterations of Alg. 1 for
each of the three solves of the debiased divergence (Eq. 2). A step runs:
radius, Lemma 1 parameters, anchors, the features of both clouds the variant uses,
the lock-step debiased solve, residuals and the Eq. (6)/(2) reductions.

Three variants are timed: stored features (HBM-bound), features recomputed in
the pass (FP32-pipe-bound) and the hybrid pass (half the feature columns
recomputed, half streamed: both at once); ``value`` is the fastest,
``variants`` has all three.

Updates per step = iters * 3 * (n + m) * r  (each feature entry used once per
half-iteration of each of the three solves).

Output: one JSON line. ``value`` is device-timed with inputs resident in HBM;
``e2e`` times the same workload through one C-ABI call (lsf_pipeline_run) from
pinned host buffers, with the copies of the inputs in and of the result record
out inside the timed region. ``roofline`` reports the dominant kernel of the
reported variant (its fused pass) against the measured HBM copy bandwidth
(stored; the stored half of the hybrid) and the FP32 pipe rate measured by the
library's probe (recompute; the recomputed half of the hybrid).
``cpu_baseline`` times the FP64 oracle on a bounded sample of the same workload
on the host cores (all cores and one thread, median of three). The metric's
batched and served solves/s are measured in the same run and reported as the
``batched`` and ``serving`` sub-objects (``--no-extra`` skips them). Other
workloads: ``--workload tiny|diff|batched|serving|arccos|accel|multi`` print
their own line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Sinkhorn n*r updates/s & %HBM roofline; batched/served solves/s, p99 vs plain"
UNIT = "updates/s"
# FP32 work per feature entry of a pass at d = 3 (the recompute roofline): 4
# operations for the exponent A_k + B_i + x.W_k, then per right-hand side one for
# the row product and one for the transposed product; the debiased lock-step
# schedule averages 1.5 right-hand sides per pass, so 7 per recomputed entry and
# 3 per stored entry (which needs no exponent). One ex2 per recomputed entry goes
# to the special-function unit, whose rate (32 per clock per SM) is above the
# FP32 pipe's 128 / 7.
OPS_RC_ENTRY = 7.0
OPS_ST_ENTRY = 3.0
# DRAM traffic of a hybrid pass launch over its algorithmic bytes, from one ncu
# capture of hybrid_kernel<4, 3, 2, 1024> at n = 2^18 (dram__bytes_read.sum
# 542.28 MB + dram__bytes_write.sum 5.54 MB against 547.36 MB algorithmic;
# profiles/hybrid_kernel_large_two_cloud.md). The full-size launch is too large to
# capture under the profiling size rule; the pass's traffic grows in proportion to
# the rows, so the full-size traffic is this ratio times its algorithmic bytes.
HYBRID_TRAFFIC_RATIO = (542.28 + 5.54) / 547.36
# NVIDIA's HBM3e figure for the part, reported beside the measured-peak fraction
# (the fraction that counts is the one against the measured copy bandwidth)
HBM_SPEC_GBS = 7900.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="all", choices=["all", "both", "stored", "recompute", "hybrid",
                                                      "log"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="large",
                    choices=["large", "batched", "serving", "diff", "tiny", "arccos", "accel", "multi"])
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--slots", type=int, default=32)
    ap.add_argument("--batch-strategy", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--pairs", type=int, default=16, help="weight pairs of --workload multi (1..32)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched and serving sub-objects of the default line")
    ap.add_argument("--serve-count", type=int, default=2000)
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle timing

ORACLE_SNIPPET = """
import json, os, sys, time
sys.path.insert(0, os.environ["LSF_ROOT"])
import synth
from oracle import oracle as o
n, iters, reps = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3])
p = synth.large_problem(seed=0, n=n, iters=iters)
ts = []
for _ in range(reps):
    t0 = time.perf_counter()
    o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True, mode="scaled")
    ts.append(time.perf_counter() - t0)
threads = None
try:
    from threadpoolctl import threadpool_info
    nt = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
    threads = int(max(nt)) if nt else None
except Exception:
    pass
print(json.dumps({"times": ts, "r": p.r, "eps": p.eps, "blas_threads": threads}))
"""


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_times(n_sample: int, iters: int, reps: int, threads: int | None) -> dict:
    """Run the oracle in a child process (so that the BLAS thread count is set
    before numpy loads) and return its per-run times."""
    env = dict(os.environ, LSF_ROOT=ROOT)
    if threads is not None:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    out = subprocess.run([sys.executable, "-c", ORACLE_SNIPPET, str(n_sample), str(iters), str(reps)],
                         capture_output=True, text=True, env=env, timeout=600, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_sample(n_sample: int, iters: int, reps: int = 3) -> dict:
    """Time the FP64 oracle on a bounded sample of the workload on the host cores:
    median of `reps` runs at all cores and at one thread, CPU model recorded."""
    updates = iters * 3 * (2 * n_sample) * 1024
    allc = _oracle_times(n_sample, iters, reps, None)
    one = _oracle_times(n_sample, iters, reps, 1)
    t_all = statistics.median(allc["times"])
    t_one = statistics.median(one["times"])
    cores = allc["blas_threads"] or os.cpu_count()
    return {"value": updates / t_all, "unit": UNIT, "cores": cores, "kind": "oracle", "ms": t_all * 1e3,
            "one_thread": {"value": updates / t_one, "ms": t_one * 1e3, "cores": 1},
            "cpu_model": cpu_model(), "nproc": os.cpu_count(), "runs": reps,
            "sample": f"FP64 oracle (scaling-domain mode, numpy BLAS) on n=m={n_sample} points "
                      f"of the same distributions, r={allc['r']}, eps={allc['eps']}, {iters} "
                      f"iterations, debiased (3 solves); median of {reps} runs: {t_all:.2f} s at "
                      f"{cores} threads, {t_one:.2f} s at 1 thread"}


# ---------------------------------------------------------------- distributed helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: every rank's timed region counts (replicas only)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, world: int, ms: float) -> float:
    """Units all ranks processed per second of the slowest rank's step."""
    return units_per_rank * world / (ms / 1e3)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    iters = 20
    n_sample = 1 << 13
    # each step: one oracle run on the sample at all host cores (warm-up and timed
    # runs in one child process, the warm-up runs discarded), plus a 1-thread record
    allc = _oracle_times(n_sample, iters, args.warmup + args.steps, None)
    updates = iters * 3 * (2 * n_sample) * 1024
    vals = [{"value": updates / t, "ms": t * 1e3} for t in allc["times"][args.warmup:]]
    value = statistics.median(v["value"] for v in vals)
    one = _oracle_times(n_sample, iters, 1, 1)
    cores = allc["blas_threads"] or os.cpu_count()
    cb = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
          "one_thread": {"value": updates / one["times"][0], "cores": 1},
          "cpu_model": cpu_model(), "nproc": os.cpu_count(),
          "sample": f"FP64 oracle (scaling-domain mode, numpy BLAS) on n=m={n_sample} points of "
                    f"the same distributions, r=1024, eps=0.1, {iters} iterations, debiased "
                    f"(3 solves), one run per step at {cores} threads"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.median(v["ms"] for v in vals), "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(args, mode=None):
    mode = mode or (args.mode if args.mode not in ("both", "all") else "stored")
    return {"workload": f"large two-cloud: n=m={args.n}, d=3, X~U[0,1]^3 vs Y~N(0.5,0.1^2 I), "
                        f"uniform weights, eps=0.1, r=1024 Gaussian features, {args.iters} "
                        f"iterations, debiased (Eq. 2), {mode} features",
            "n": args.n, "m": args.n, "d": 3, "r": 1024, "eps": 0.1, "iters": args.iters,
            "debiased": True, "mode": mode,
            "l2": ("inputs larger than L2 (two 4 GiB feature matrices streamed every pass)"
                   if mode in ("stored", "log") else
                   "inputs larger than L2 (two 2 GiB stored half-feature blocks streamed every "
                   "pass); a 256 MiB buffer is also written before every timed step"
                   if mode == "hybrid" else
                   "points and vectors (about 50 MB) fit in L2: a 256 MiB buffer is written "
                   "before every timed step to flush it (its time counted in the step)"),
            "parallelism": f"replicas x{args.gpus} (independent problems, no collective)"}


# ---------------------------------------------------------------- our arm

def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(batched_measure(args, args.count)))
    return 0


def batched_measure(args, count):
    """Batched workload: independent problems of uneven shape, one persistent launch per
    feature width, CUDA-graph captured; against the same problems solved one after
    another with the plain solver on the same stream. Returns the JSON line."""
    import torch
    import paper_2006_07057_gb300 as lsf
    lsf.lsf_set_batch_strategy(args.batch_strategy)
    iters = 100
    probs = synth.batched_problems(seed=0, count=count, iters=iters)
    dev = torch.device("cuda", torch.cuda.current_device())

    class Dev:
        def __init__(self, p):
            self.X, self.Y, self.a, self.b, self.Z = (torch.from_numpy(getattr(p, k)).to(dev)
                                                      for k in ("X", "Y", "a", "b", "Z"))
            self.eps = p.eps

    groups = {}
    for p in probs:
        groups.setdefault(lsf.ldr_for(p.r), []).append(Dev(p))
    solvers = [lsf.BatchedSolver(g, ldr=ldr, mode="auto") for ldr, g in sorted(groups.items())]
    for sv in solvers:
        sv.capture(iters)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def batched_step():
        for sv in solvers:
            sv.replay()

    for _ in range(args.warmup):
        batched_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batched_step()
    e1.record(stream)
    e1.synchronize()
    ms_batched = e0.elapsed_time(e1) / args.steps
    vals = [v for sv in solvers for v in sv.values()]
    nonfinite = sum(1 for v in vals if v["status"] & lsf.LSF_ERR_NONFINITE)

    routed = sum(len(idx) for sv in solvers for b, idx in sv.batches if b.mode == "log")
    # plain: the same problems, one lsf_solve + Eq. (6) after another, same stream, in the
    # mode the batched solver routed them to
    singles = [lsf.SinkhornProblem(pp.X, pp.Y, pp.a, pp.b, pp.Z, pp.eps, ldr=sv.ldr, mode=pp.mode)
               for sv in solvers for pp in sv.problems]
    for sp in singles[: min(8, len(singles))]:
        sp.run(iters, debiased=False)
    torch.cuda.synchronize()
    done = [torch.cuda.Event(enable_timing=True) for _ in singles]
    p0 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for sp, ev in zip(singles, done):
        sp.run(iters, debiased=False)
        ev.record(stream)
    done[-1].synchronize()
    lat_plain = sorted(p0.elapsed_time(ev) for ev in done)
    ms_plain = lat_plain[-1]
    n = len(singles)
    pct = lambda xs, q: xs[min(len(xs) - 1, int(q * len(xs)))]  # noqa: E731
    line = {
        "metric": METRIC, "value": n / (ms_batched / 1e3), "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batched,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batched: {n} problems, n,m log-uniform [2^10, 2^16], d in {{2,3,16}}, "
                               f"r in {{128,256}}, eps log-uniform [0.05,1], mixture clouds, Dirichlet(1) "
                               f"weights, {iters} iterations, CUDA-graph captured, one launch per feature "
                               f"width and domain (one cluster per problem or one persistent kernel), "
                               f"stored features resident",
                   "groups": {str(sv.ldr): [{"mode": b.mode, "problems": len(idx),
                                             "strategy": ("clusters" if b.info.strategy == 1
                                                          else "persistent"),
                                             "tile_bytes": b.tile_bytes, "tile_rows": b.info.tile_rows,
                                             "stages": b.info.stages} for b, idx in sv.batches]
                              for sv in solvers}},
        "batched": {"solves_per_s": n / (ms_batched / 1e3), "ms_per_batch": ms_batched,
                    "latency_ms_p50": ms_batched, "latency_ms_p99": ms_batched,
                    "nonfinite_problems": nonfinite, "log_domain_problems": routed},
        "plain_sequential": {"solves_per_s": n / (ms_plain / 1e3), "ms_total": ms_plain,
                             "latency_ms_p50": pct(lat_plain, 0.5), "latency_ms_p99": pct(lat_plain, 0.99)},
        "speedup_vs_plain": ms_plain / ms_batched,
    }
    return line


def run_serving(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(serving_measure(args, args.count, args.rate)))
    return 0


def extra_legs(args) -> dict:
    """The batched and served solves/s of the metric, measured in the default run
    (with the GPU clocks sampled during each), as sub-objects of its JSON line."""
    out = {}
    sampler = ClockSampler(0)
    sampler.start()
    b = batched_measure(args, 512)
    out["batched"] = {"solves_per_s": b["value"], "ms_per_batch": b["ms_per_step"],
                      "config": b["config"]["workload"], **b["batched"],
                      "plain_sequential": b["plain_sequential"],
                      "speedup_vs_plain": b["speedup_vs_plain"], "clocks": sampler.stop()}
    sampler = ClockSampler(0)
    sampler.start()
    v = serving_measure(args, args.serve_count, 2000.0)
    out["serving"] = {"solves_per_s": v["value"], "config": v["config"]["workload"],
                      "served": v["served"], "servers": v["servers"],
                      "plain_sequential": v["plain_sequential"],
                      "p99_ratio_plain_over_served": v["p99_ratio_plain_over_served"],
                      "max_rel_diff_served_vs_alone": v["max_rel_diff_served_vs_alone"],
                      "note": f"{args.serve_count} requests of the 10k-request stream's distribution "
                              "(a reduced count keeps the default run within minutes)",
                      "clocks": sampler.stop()}
    return out


def serving_measure(args, count, rate):
    """Serving workload: a Poisson stream of debiased-divergence requests of uneven
    shape served by the continuous-batching server (40 GB admission budget), against
    the same stream served one request at a time. Returns the JSON line."""
    import dataclasses
    import torch
    import paper_2006_07057_gb300 as lsf
    from paper_2006_07057_gb300 import serve
    lsf.lib()
    iters = 100
    base = []
    for i, rq in enumerate(synth.serving_stream(seed=0, count=count, rate_per_s=rate, iters=iters)):
        p = rq.problem
        base.append(serve.Request(i, p.X, p.Y, p.a, p.b, p.Z, p.eps, iters, rq.arrival_s).pin())
    fresh = lambda: [dataclasses.replace(r, result={}) for r in base]  # noqa: E731
    # two continuous-batching servers: per-request streams (each request one
    # lsf_pipeline_run) and groups of requests solved by the persistent batched
    # kernel; the better one is reported as `served`
    arms = {}
    for name, make in (("streams", lambda: serve.Server(budget_bytes=40e9, slots=args.slots)),
                       ("batched_groups", lambda: serve.BatchingServer(budget_bytes=40e9))):
        srv_ = make()
        srv_.serve(fresh()[: min(16, count)], realtime=False)   # warm-up (kernels loaded)
        torch.cuda.synchronize()
        out_ = srv_.serve(fresh(), realtime=True)
        arms[name] = (srv_, out_, serve.latency_stats(out_))
        srv_.pool.buf = None   # the 40 GB pool goes back before the next arm
        del srv_
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    best_name = max(arms, key=lambda k: arms[k][2]["throughput_per_s"])
    srv, mixed, st_mixed = arms[best_name]
    seq = serve.serve_sequential(fresh(), realtime=True)
    st_seq = serve.latency_stats(seq)
    nonfinite = sum(1 for r in mixed if r.status & lsf.LSF_ERR_NONFINITE)
    # where the GPU time goes: the sequential arm serves one request at a time,
    # so each request's start-to-done time is its whole service time
    service = {}
    for r in seq:
        key = r.result.get("mode", "?")
        service.setdefault(key, [0, 0.0])
        service[key][0] += 1
        service[key][1] += r.done_s - r.start_s
    st_seq["service_s_by_domain"] = {k: {"requests": v[0], "seconds": v[1]} for k, v in service.items()}
    by_id = {r.rid: r for r in seq}
    worst = max(abs(r.W_bar - by_id[r.rid].W_bar) /
                max(abs(r.result["W_xy"]) + 0.5 * abs(r.result["W_xx"]) + 0.5 * abs(r.result["W_yy"]), 1e-30)
                for r in mixed)
    line = {
        "metric": METRIC, "value": st_mixed["throughput_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": 1e3 * st_mixed["span_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serving: Poisson stream of {count} debiased-divergence requests at "
                               f"{rate:g}/s, n,m log-uniform [2^8, 2^18], d in {{2,3,16}}, "
                               f"r in {{128,512}}, eps in {{0.05,0.2,1.0}}, mixture clouds, uniform "
                               f"weights, {iters} iterations, 40 GB admission budget, {args.slots} slots"},
        "served": {**st_mixed, "server": best_name, "peak_inflight": srv.peak_inflight,
                   "peak_bytes": srv.peak_bytes, "nonfinite_requests": nonfinite,
                   "relaunched_in_log_domain": srv.relaunched},
        "servers": {k: {**v[2], "relaunched_in_log_domain": v[0].relaunched,
                        "peak_inflight": v[0].peak_inflight} for k, v in arms.items()},
        "plain_sequential": st_seq,
        "p99_ratio_plain_over_served": st_seq["latency_ms_p99"] / st_mixed["latency_ms_p99"],
        "max_rel_diff_served_vs_alone": worst,
    }
    return line


def _profile_roofline(lsf, cls, kernel, peak, peak_kind, ms_total):
    """Roofline entry for one kernel class from the library's CUDA-event records."""
    k_ms, k_n, k_bytes = lsf.lsf_profile_read(cls)
    achieved = (k_bytes / 1e9) / (k_ms / 1e3) if k_ms > 0 else None
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
            "traffic": None, "launches": k_n, "avg_launch_ms": k_ms / max(k_n, 1),
            "bytes_per_launch": k_bytes / max(k_n, 1),
            "share_of_step": k_ms / ms_total if ms_total > 0 else None}


def _timed(fn, steps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def run_diff(args):
    """Differentiation workload: features, the debiased forward solve and the adjoint
    w.r.t. X, Y, a, b (and the anchors) for n = m = 8192 points in R^128."""
    import torch
    import paper_2006_07057_gb300 as lsf
    torch.cuda.set_device(0)
    lsf.lib()
    p = synth.diff_problem(seed=0)
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(getattr(p, k)).to(dev) for k in ("X", "Y", "a", "b", "Z")}
    stream = torch.cuda.current_stream()
    holder = {}

    def forward():
        prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps)
        prob.run(p.iters, debiased=True)
        holder["prob"] = prob

    def step():
        forward()
        holder["g"] = holder["prob"].gradient()
        holder["gU"] = holder["prob"].anchor_gradient()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    vals = holder["prob"].values()
    ms_fwd = _timed(forward, args.steps, stream)
    prob = holder["prob"]
    ms_adj = _timed(lambda: (prob.gradient(), prob.anchor_gradient()), args.steps, stream)
    lsf.lsf_profile_enable(True)
    lsf.lsf_launch_count_reset()
    sampler = ClockSampler(0)
    sampler.start()
    ms = _timed(step, args.steps, stream)
    clocks = sampler.stop()
    launches = lsf.lsf_launch_count()
    peak, peak_kind = load_peaks()
    roof = _profile_roofline(lsf, lsf.LSF_KERNEL_PASS, "pass_kernel (32 MiB features: L2-resident)",
                             peak, peak_kind, ms * args.steps)
    adj_ms, adj_n, _ = lsf.lsf_profile_read(lsf.LSF_KERNEL_ADJOINT)
    feat_ms, feat_n, _ = lsf.lsf_profile_read(lsf.LSF_KERNEL_FEATURES)
    lsf.lsf_profile_enable(False)
    updates = p.iters * 3 * (p.n + p.m) * p.r
    line = {
        "metric": METRIC, "value": updates / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"differentiation: n=m={p.n} points in R^{p.d} (N(0,I) vs N(mu,I), "
                               f"|mu|=1), uniform weights, eps={p.eps}, r={p.r}, {p.iters} iterations, "
                               f"debiased forward + adjoint w.r.t. X, Y, a, b and the anchors",
                   "l2": "features (2 x 32 MiB) stay L2-resident; step counted with features rebuilt"},
        "gpu_launches": int(launches), "roofline": roof, "clocks": clocks,
        "forward_ms": ms_fwd, "adjoint_ms": ms_adj,
        "adjoint_kernels_ms_per_step": adj_ms / args.steps, "adjoint_launches": adj_n,
        "features_ms_per_step": feat_ms / args.steps,
        "result": {"W_bar": vals["W_bar"], "status": vals["status"]},
    }
    print(json.dumps(line))
    return 0


def run_tiny(args):
    """Tiny workload: latency of one whole solve (parameters, features, 100 iterations,
    Eq. (6)) for n = m = 1000 points in R^2, r = 100: launch-bound, reported per solve,
    plain stream launches and one CUDA-graph replay of the same solve."""
    import torch
    import paper_2006_07057_gb300 as lsf
    torch.cuda.set_device(0)
    lsf.lib()
    p = synth.tiny_problem()
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(getattr(p, k)).to(dev) for k in ("X", "Y", "a", "b", "Z")}
    stream = torch.cuda.current_stream()
    steps = max(args.steps, 20)

    def solve():
        prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps)
        prob.run(p.iters, debiased=False)
        return prob

    for _ in range(args.warmup):
        prob = solve()
    torch.cuda.synchronize()
    vals = prob.values()
    lsf.lsf_launch_count_reset()
    ms_full = _timed(solve, steps, stream)
    launches = lsf.lsf_launch_count() / steps
    # the iterations alone, resident problem, captured once in a CUDA graph
    prob = solve()
    torch.cuda.synchronize()
    ms_solve = _timed(lambda: prob.run(p.iters, debiased=False), steps, stream)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(stream)
    with torch.cuda.stream(s):
        prob.stream = s
        prob.run(p.iters, debiased=False)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            prob.run(p.iters, debiased=False)
    prob.stream = None
    torch.cuda.synchronize()
    ms_graph = _timed(g.replay, steps, stream)
    updates = p.iters * (p.n + p.m) * p.r
    line = {
        "metric": METRIC, "value": updates / (ms_full / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms_full, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"tiny: n=m={p.n} points in R^2 (3-component mixture vs the same "
                               f"mixture + 1), uniform weights, eps={p.eps}, r={p.r}, {p.iters} "
                               f"iterations, W(a,b) (Eq. 6)",
                   "l2": "inputs L2-resident (latency-bound workload)"},
        "gpu_launches_per_solve": launches,
        "latency_us": {"whole_path": 1e3 * ms_full, "iterations_resident": 1e3 * ms_solve,
                       "iterations_graph_replay": 1e3 * ms_graph},
        "result": {"W": vals["W_xy"], "res": vals["res_xy"], "status": vals["status"]},
    }
    print(json.dumps(line))
    return 0


def run_arccos(args):
    """Arc-cosine features (Sec. 3.2 and its appendix lemma) on the large two-cloud
    shape: n = m = 2^20 points in R^3, r = 1023 anchors (1024 features with the
    merged constant), s = 1, sigma = 1.5, kappa = 0.1, 200 iterations, debiased,
    stored features. The solve is the same fused pass as for the Gaussian map."""
    import torch
    import paper_2006_07057_gb300 as lsf
    torch.cuda.set_device(0)
    lsf.lib()
    p = synth.large_problem(seed=0, n=args.n, iters=args.iters)
    r = 1023
    Z = p.Z[:r]
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(getattr(p, k)).to(dev) for k in ("X", "Y", "a", "b")}
    tZ = torch.from_numpy(np.ascontiguousarray(Z)).to(dev)
    stream = torch.cuda.current_stream()
    holder = {}

    def step():
        prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], tZ, 1.0, kernel="arccos", s=1,
                                   sigma=1.5, kappa=0.1)
        prob.run(args.iters, debiased=True)
        holder["prob"] = prob

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    vals = holder["prob"].values()
    if vals["status"] != 0:
        raise SystemExit(f"arc-cosine solve reported status {vals['status']}")
    sampler = ClockSampler(0)
    sampler.start()
    lsf.lsf_profile_enable(True)
    lsf.lsf_launch_count_reset()
    ms = _timed(step, args.steps, stream)
    clocks = sampler.stop()
    launches = lsf.lsf_launch_count()
    peak, peak_kind = load_peaks()
    roof = _profile_roofline(lsf, lsf.LSF_KERNEL_PASS, "pass_kernel (fused Sinkhorn half-iteration)",
                             peak, peak_kind, ms * args.steps)
    feat_ms, feat_n, feat_bytes = lsf.lsf_profile_read(lsf.LSF_KERNEL_FEATURES)
    lsf.lsf_profile_enable(False)
    ldr = 1024
    updates = args.iters * 3 * (p.n + p.m) * ldr
    line = {
        "metric": METRIC, "value": updates / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"arc-cosine features (s=1, sigma=1.5, kappa=0.1) on the large "
                               f"two-cloud shape: n=m={p.n}, d=3, r={r} anchors + 1 constant "
                               f"feature, eps=1, {args.iters} iterations, debiased, stored features",
                   "l2": "inputs larger than L2 (two 4 GiB feature matrices streamed every pass)"},
        "gpu_launches": int(launches), "roofline": roof, "clocks": clocks,
        "features_ms_per_step": feat_ms / args.steps,
        "features_GBps": (feat_bytes / 1e9) / (feat_ms / 1e3) if feat_ms > 0 else None,
        "result": {"W_bar": vals["W_bar"], "W_xy": vals["W_xy"], "res_xy": vals["res_xy"],
                   "status": vals["status"]},
    }
    print(json.dumps(line))
    return 0


def run_accel(args):
    """Accelerated Sinkhorn (App. A.2) against plain Alg. 1, both in the log domain,
    measured as time to the same residual: the accelerated solver runs K iterations
    (three log-domain passes and a host decision per line-search attempt); the
    plain solver is run for 100, 200, 400, ... iterations until its residual
    ||P 1 - a||_1 is at most the accelerated one's ||P 1 - a||_1 + ||P^T 1 - b||_1,
    then bisected to the fewest iterations that reach it.
    Workload: the tiny workload's mixtures at n = m = 2^16, r = 512, eps = 0.01."""
    import torch
    import paper_2006_07057_gb300 as lsf
    torch.cuda.set_device(0)
    lsf.lib()
    n = min(args.n, 1 << 16)
    K = 300
    p = synth.tiny_problem(seed=0, n=n, m=n, r=512, eps=0.01, iters=K)
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(getattr(p, k)).to(dev) for k in ("X", "Y", "a", "b", "Z")}
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode="log")

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3, out

    for _ in range(max(args.warmup, 1)):
        prob.run_accelerated(20, debiased=False)
        prob.run(20, debiased=False)
    sampler = ClockSampler(0)
    sampler.start()
    lsf.lsf_launch_count_reset()
    ms_acc, stats = wall(lambda: prob.run_accelerated(K, debiased=False))
    acc_launches = lsf.lsf_launch_count()
    va = prob.values()
    target = va["res_xy"]
    plain = []

    def plain_run(its):
        ms_p, _ = wall(lambda: prob.run(its, debiased=False))
        vp = prob.values()
        rec = {"iters": its, "ms": ms_p, "residual": vp["res_xy"], "W": vp["W_xy"]}
        plain.append(rec)
        return rec

    # doubling until the target residual is reached, then bisection between the
    # last two counts for the fewest iterations that reach it
    it, lo_it, reached = 100, 0, None
    while it <= 12800:
        rec = plain_run(it)
        if rec["residual"] <= target:
            reached = rec
            break
        lo_it, it = it, it * 2
    if reached is not None:
        hi_it = reached["iters"]
        while hi_it - lo_it > max(2, hi_it // 64):
            mid = (lo_it + hi_it) // 2
            rec = plain_run(mid)
            if rec["residual"] <= target:
                hi_it, reached = mid, rec
            else:
                lo_it = mid
    clocks = sampler.stop()
    attempts = stats[0]["attempts"]
    # entry updates: per attempt an X column pass, a Y row+column pass and an X row pass
    acc_updates = attempts * (2 * n + n) * p.r
    line = {
        "metric": METRIC, "value": acc_updates / (ms_acc / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": args.warmup, "ms_per_step": ms_acc, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"accelerated Sinkhorn (App. A.2) vs plain Alg. 1, log domain: "
                               f"n=m={n} points in R^2 (3-component mixture vs the same mixture + 1), "
                               f"uniform weights, eps={p.eps}, r={p.r}, {K} accelerated iterations",
                   "l2": "features (2 x 128 MiB) exceed L2"},
        "gpu_launches": int(acc_launches), "clocks": clocks,
        "accelerated": {"iters": stats[0]["iters"], "attempts": attempts, "ms": ms_acc,
                        "residual": target, "W": va["W_xy"], "L": stats[0]["L"],
                        "plain_iteration_equivalents": attempts * 1.5},
        "plain_to_same_residual": reached, "plain_runs": plain,
        "time_ratio_plain_over_accelerated": (reached["ms"] / ms_acc) if reached else None,
    }
    print(json.dumps(line))
    return 0


def run_multi(args):
    """Many weight vectors on one support (the tensor-core pass): k = 16 pairs of
    Dirichlet(1) weights on the large two-cloud shape (n = m = 2^20 in R^3, eps = 0.1,
    r = 1024), 200 iterations of Alg. 1 for each of the three terms of Eq. (2) per
    pair. A step = features, their bf16 pair split, three multi-right-hand-side
    solves ((X, Y), (X, X), (Y, Y)) and Eq. (6)/(2). Compared with the same 16 pairs'
    debiased divergences computed one after another by the stored-feature single
    solve (its lock-step schedule)."""
    import torch
    import paper_2006_07057_gb300 as lsf
    torch.cuda.set_device(0)
    lsf.lib()
    n = args.n
    k = args.pairs
    p = synth.large_problem(seed=0, n=n, iters=args.iters)
    rng = np.random.default_rng(7)
    A = rng.exponential(size=(k, n))
    B = rng.exponential(size=(k, n))
    A = (A / A.sum(axis=1, keepdims=True)).astype(np.float32)
    B = (B / B.sum(axis=1, keepdims=True)).astype(np.float32)
    dev = torch.device("cuda", 0)
    t = {q: torch.from_numpy(getattr(p, q)).to(dev) for q in ("X", "Y", "Z")}
    tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    stream = torch.cuda.current_stream()
    holder = {}

    def step():
        prob = lsf.MultiSinkhornProblem(t["X"], t["Y"], tA, tB, t["Z"], p.eps)
        prob.run(args.iters, debiased=True)
        holder["prob"] = prob

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    vals = holder["prob"].values()
    if any(v["status"] != 0 for v in vals):
        raise SystemExit(f"multi solve reported status {[v['status'] for v in vals]}")
    sampler = ClockSampler(0)
    sampler.start()
    lsf.lsf_profile_enable(True)
    lsf.lsf_launch_count_reset()
    ms = _timed(step, args.steps, stream)
    launches = lsf.lsf_launch_count()
    peak, peak_kind = load_peaks()
    roof = _profile_roofline(lsf, lsf.LSF_KERNEL_PASS_MULTI,
                             f"multi_pass_kernel (tcgen05 bf16-pair passes, {k} right-hand sides)",
                             peak, peak_kind, ms * args.steps)
    feat_ms, _, _ = lsf.lsf_profile_read(lsf.LSF_KERNEL_FEATURES)
    lsf.lsf_profile_enable(False)
    clocks = sampler.stop()

    # the same pairs one after another through the single solve (stored features)
    def sequential():
        out = []
        single = lsf.SinkhornProblem(t["X"], t["Y"], tA[0].contiguous(), tB[0].contiguous(),
                                     t["Z"], p.eps, mode="stored")
        for q in range(k):
            single.x.w = tA[q].contiguous()
            single.y.w = tB[q].contiguous()
            single.run(args.iters, debiased=True)
            out.append(single.values()["W_bar"])
        return out

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_W = sequential()
    torch.cuda.synchronize()
    ms_seq = (time.perf_counter() - t0) * 1e3
    worst = max(abs(v["W_bar"] - w) / (abs(v["W"]) + 0.5 * abs(v["W_xx"]) + 0.5 * abs(v["W_yy"]))
                for v, w in zip(vals, seq_W))
    updates = 3 * k * args.iters * (p.n + p.m) * p.r
    line = {
        "metric": METRIC, "value": updates / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x2/f32", "data": "synthetic",
        "config": {"workload": f"{k} weight pairs (Dirichlet(1)) on one support: the large two-cloud "
                               f"shape n=m={p.n}, d=3, eps={p.eps}, r={p.r}, {args.iters} iterations "
                               f"per term, debiased divergence (Eq. 2) per pair; tensor-core "
                               f"multi-right-hand-side passes",
                   "l2": "inputs larger than L2 (two 4 GiB bf16-pair feature matrices per pass)"},
        "gpu_launches": int(launches), "roofline": roof, "clocks": clocks,
        "features_ms_per_step": feat_ms / args.steps,
        "sequential_single_solves_ms": ms_seq,
        "speedup_vs_sequential": ms_seq / ms,
        "max_rel_W_bar_diff_vs_single": worst,
        "result": {"W_bar": [v["W_bar"] for v in vals[:4]], "W": [v["W"] for v in vals[:4]],
                   "residual": [v["residual"] for v in vals[:4]]},
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "diff":
        return run_diff(args)
    if args.workload == "tiny":
        return run_tiny(args)
    if args.workload == "accel":
        return run_accel(args)
    if args.workload == "multi":
        return run_multi(args)
    if args.workload == "arccos":
        return run_arccos(args)
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2006_07057_gb300 as lsf
    lsf.lib()

    p = synth.large_problem(seed=rank, n=args.n, iters=args.iters)
    updates = args.iters * 3 * (p.n + p.m) * p.r
    dev = torch.device("cuda", local)
    host = {k: torch.from_numpy(getattr(p, k)).pin_memory() for k in ("X", "Y", "a", "b", "Z")}
    devt = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
    stream = torch.cuda.current_stream()
    peak, peak_kind = load_peaks()
    peak_kind_hbm = peak_kind

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def slowest(ms):
        return max_over_ranks(ms, world, dev)

    # the recompute variant's inputs fit in L2: flush it between timed steps
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    rates = lsf.lsf_probe_pipe_rates()

    def measure(mode):
        """Warm-up, then K timed steps of one variant with inputs resident."""
        def step_resident():
            prob = lsf.SinkhornProblem(devt["X"], devt["Y"], devt["a"], devt["b"], devt["Z"], p.eps,
                                       mode=mode)
            prob.run(args.iters, debiased=True)
            return prob

        for _ in range(args.warmup):
            prob = step_resident()
        torch.cuda.synchronize()
        check = prob.values()
        if check["status"] != 0 or not np.isfinite(check["W_bar"]):
            raise SystemExit(f"{mode}: solver reported status {check['status']}, W_bar {check['W_bar']}")
        sampler = ClockSampler(local)
        sampler.start()
        lsf.lsf_profile_enable(True)
        lsf.lsf_launch_count_reset()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        e0.record(stream)
        marks[0].record(stream)
        for i in range(args.steps):
            if mode in ("recompute", "hybrid"):
                l2_flush.zero_()
            prob = step_resident()
            marks[i + 1].record(stream)
        e1.record(stream)
        barrier()
        launches = lsf.lsf_launch_count()
        clocks = sampler.stop()
        ms = slowest(e0.elapsed_time(e1) / args.steps)
        per_step = sorted(marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps))
        ms_median = per_step[len(per_step) // 2]
        cls = {"stored": lsf.LSF_KERNEL_PASS, "recompute": lsf.LSF_KERNEL_PASS_RECOMPUTE,
               "log": lsf.LSF_KERNEL_PASS_LOG, "hybrid": lsf.LSF_KERNEL_PASS_HYBRID}[mode]
        k_ms, k_n, k_bytes = lsf.lsf_profile_read(cls)
        feat_ms, _, _ = lsf.lsf_profile_read(lsf.LSF_KERNEL_FEATURES)
        lsf.lsf_profile_enable(False)
        vals = prob.values()
        share = k_ms / (ms * args.steps) if ms > 0 else None
        if mode in ("stored", "log"):
            achieved = (k_bytes / 1e9) / (k_ms / 1e3) if k_ms > 0 else None
            kname = ("pass_kernel (fused Sinkhorn half-iteration)" if mode == "stored" else
                     "logpass_kernel (log-domain fused half-iteration; ex2-bound)")
            roof = {"bound": "hbm", "kernel": kname,
                    "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                    "frac_of_spec": (achieved / HBM_SPEC_GBS) if achieved else None,
                    "traffic": None, "launches": k_n, "avg_launch_ms": k_ms / max(k_n, 1),
                    "bytes_per_launch": k_bytes / max(k_n, 1), "share_of_step": share}
        else:
            # passes per step: 2 per iteration over each cloud, plus the start and residual
            # passes (one each per cloud); every pass uses each entry of its cloud once.
            # FP32 pipe peak: lanes per clock per SM measured by the packed-FMA probe,
            # times the SMs and the SM clock sampled during the timed region.
            entries = (2 * args.iters + 2) * (p.n + p.m) * p.r * args.steps
            launches_n = max(k_n, 1)
            sm_mhz = clocks.get("sm_mhz") or 2070.0
            lanes = rates["ffma2_lane_ops_per_clk_sm"]
            alu_peak = lanes * sms * sm_mhz * 1e6 / 1e12            # T FP32 ops/s
            alu_kind = (f"measured: {lanes:.1f} FP32 lane-ops/clk/SM (packed FMA probe) x {sms} "
                        f"SMs x {sm_mhz:.0f} MHz")
            if mode == "recompute":
                ops = entries * OPS_RC_ENTRY
                achieved = ops / (k_ms / 1e3) / 1e12 if k_ms > 0 else None
                roof = {"bound": "alu", "kernel": "recompute_kernel (fused pass, features rebuilt with ex2)",
                        "achieved": achieved, "peak": alu_peak, "unit": "T FP32 ops/s",
                        "frac": (achieved / alu_peak) if achieved else None, "peak_kind": alu_kind,
                        "ops_per_entry": OPS_RC_ENTRY, "entries_per_launch": entries / launches_n,
                        "traffic": None, "launches": k_n, "avg_launch_ms": k_ms / launches_n,
                        "share_of_step": share}
            else:
                # half the columns recomputed (ALU), half streamed (HBM): the kernel's
                # bound is the larger of the two times; both fractions are reported
                c0 = lsf.lsf_hybrid_columns(1024)
                frac_rc = min(c0, p.r) / p.r
                ops = entries * (frac_rc * OPS_RC_ENTRY + (1 - frac_rc) * OPS_ST_ENTRY)
                t_alu = ops / (alu_peak * 1e12)
                t_hbm = (k_bytes / 1e9) / peak
                t_meas = k_ms / 1e3
                hbm_ach = (k_bytes / 1e9) / t_meas if k_ms > 0 else None
                alu_ach = ops / t_meas / 1e12 if k_ms > 0 else None
                hbm_bound = t_hbm >= t_alu
                roof = {"bound": "hbm" if hbm_bound else "alu",
                        "kernel": "hybrid_kernel (fused pass: half the feature columns rebuilt, half streamed)",
                        "achieved": hbm_ach if hbm_bound else alu_ach,
                        "peak": peak if hbm_bound else alu_peak,
                        "unit": "GB/s" if hbm_bound else "T FP32 ops/s",
                        "frac": (max(t_hbm, t_alu) / t_meas) if k_ms > 0 else None,
                        "peak_kind": peak_kind_hbm if hbm_bound else alu_kind,
                        "hbm": {"achieved": hbm_ach, "peak": peak, "unit": "GB/s",
                                "frac": hbm_ach / peak if hbm_ach else None, "peak_kind": peak_kind_hbm,
                                "frac_of_spec": hbm_ach / HBM_SPEC_GBS if hbm_ach else None},
                        "alu": {"achieved": alu_ach, "peak": alu_peak, "unit": "T FP32 ops/s",
                                "frac": alu_ach / alu_peak if alu_ach else None, "peak_kind": alu_kind},
                        "traffic": HYBRID_TRAFFIC_RATIO * k_bytes / launches_n,
                        "traffic_note": "scaled from the n = 2^18 ncu capture (DRAM bytes / algorithmic "
                                        "bytes = %.4f)" % HYBRID_TRAFFIC_RATIO,
                        "launches": k_n, "avg_launch_ms": k_ms / launches_n,
                        "bytes_per_launch": k_bytes / launches_n, "share_of_step": share}
        return {"mode": mode, "ms": ms, "value": whole_job_value(updates, world, ms), "launches": launches,
                "clocks": clocks, "roofline": roof, "vals": vals,
                "features_ms_per_step": feat_ms / args.steps, "ms_median": ms_median}

    modes = (["stored", "recompute", "hybrid"] if args.mode == "all" else
             ["stored", "recompute"] if args.mode == "both" else [args.mode])
    runs = [measure(m) for m in modes]
    best = max(runs, key=lambda r: r["value"])

    # ---- end to end from pinned host buffers through one C-ABI call
    # (lsf_pipeline_run: inputs copied in, the whole path, the result record copied
    # out, all on the stream), best variant
    e2e = None
    if not args.no_e2e:
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        hp = lsf.HostPipeline(dev)
        hargs = [host[k] for k in ("X", "Y", "a", "b", "Z")]

        def step_e2e():
            if best["mode"] in ("recompute", "hybrid"):
                l2_flush.zero_()
            hp.run(*hargs, p.eps, args.iters, debiased=True, mode=best["mode"])

        step_e2e()
        chk = hp.result()
        if chk["status"] != 0 or abs(chk["W"] - best["vals"]["W_bar"]) > 1e-5 * abs(best["vals"]["W_xy"]):
            raise SystemExit(f"e2e path disagrees: {chk['W']} vs {best['vals']['W_bar']}")
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            step_e2e()
        f1.record(stream)
        barrier()
        ms_e2e = slowest(f0.elapsed_time(f1) / args.steps)
        e2e = {"value": whole_job_value(updates, world, ms_e2e), "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(ctypes.sizeof(lsf.LsfPipelineOut)),
               "api": "lsf_pipeline_run (host inputs, host result record)",
               "W_bar": hp.result()["W"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_sample(1 << 13, 20)
    rates["sms"] = sms

    if rank == 0:
        vals = best["vals"]
        line = {
            "metric": METRIC, "value": best["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(args, best["mode"]), "e2e": e2e,
            "gpu_launches": int(best["launches"]), "roofline": best["roofline"],
            "cpu_baseline": cpu, "clocks": best["clocks"],
            "ms_per_step_median": best["ms_median"],
            "variants": {r["mode"]: {"value": r["value"], "ms_per_step": r["ms"],
                                     "ms_per_step_median": r["ms_median"],
                                     "gpu_launches": int(r["launches"]), "roofline": r["roofline"],
                                     "W_bar": r["vals"]["W_bar"], "clocks": r["clocks"],
                                     "features_ms_per_step": r["features_ms_per_step"]}
                         for r in runs},
            "result": {"W_bar": vals["W_bar"], "W_xy": vals["W_xy"], "res_xy": vals["res_xy"],
                       "status": vals["status"]},
            "features_ms_per_step": best["features_ms_per_step"],
            "pipe_rates": rates,
        }
        if world == 1 and not args.no_extra:
            line.update(extra_legs(args))
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
