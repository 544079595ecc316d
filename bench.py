"""Benchmark: time-to-rank-k and pivots/s of accelerated RPCholesky on GB300.

One step = one complete factorisation of the workload's kernel matrix to
rank k (every round of Algorithm 2: proposals, H, Algorithm 1, fused column
step, diagonal update) with a fresh seed, inputs resident in HBM.  The
default workload is the largest single-GPU configuration, unif64_n1e6
(N = 1e6 points uniform on [0,1]^64 with 1% outliers scaled by 10,
l2-Laplace kernel with the median bandwidth, k = 4000, T = 200, FP32 factor
of 16 GB).  The same line carries simple RPCholesky (Algorithm 6) on the
same GPU and workload, the column step's roofline, the oracle on the host
cores, the end-to-end time through the public API with host buffers, the
N = 1e5 Gaussian-mixture workload (with the FP64 mode, block RPCholesky and
the low-memory and QR variants), the batched workload and the serving
stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision mixed|fp64]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores, on the first N' points of the same workload (N' sized so
that the whole run takes a few minutes; the line reports the time it
measured).  With N > 1 (one process per GPU under torch.distributed.run)
every rank factorises its own seeds independently (weak scaling, no
data-path collective).
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

import workloads  # noqa: E402

METRIC = "time-to-rank-k & pivots/s vs plain RPCholesky, 1 GB300, equal trace error; p99"
UNIT = "pivots/s"


_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line is the only stdout)."""
    print("[bench %7.1fs] %s" % (time.perf_counter() - _T0, msg), file=sys.stderr, flush=True)


def _pct(v, q):
    v = sorted(v)
    if not v:
        return None
    i = min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))
    return v[i]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return j, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# DRAM traffic of the tensor-core column step per launch (dram__bytes_read.sum +
# dram__bytes_write.sum of the k_colstep_tc launches of one ncu capture of
# `bench.py --quick --no-graph --steps 1 --warmup 1` on the workload, averaged over
# the launches that ran a round), with the SHA-256 of the sources the capture ran.
# The N = 10^6 workload (16 GB of F) is captured at N = 10^5 (`--n-points 100000`,
# same k, T and rank sequence) and scaled by the rows, 10x: every row of F and X is
# read once per round, so the traffic grows in proportion to N.  When the sources
# have changed since, the figure no longer describes the kernel and the bench
# reports null.  Summaries: profiles/colstep_tc_unif64_n1e6.md (and
# profiles/colstep_tc_mixture20_n1e5.md for the earlier kernel).
_COLSTEP_SOURCES = ("k_colstep_tc.cu", "colstep_body.cuh", "tc_ptx.cuh", "common.cuh",
                    "internal.h")
_COLSTEP_TRAFFIC = {
    ("mixture20_n1e5", "mixed"): (
        162153888.0, "04fcd24dcced58aeb93d85712943709620fd5bdf030f42de1d6c007425f931cb"),
    ("unif64_n1e6", "mixed"): (
        9929326649.0, "5a3d05fb369c24f6a46e133306ec26fed88b42aeef509c009ebb5b267d901afb"),
}


def _colstep_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in _COLSTEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2410_03969_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _colstep_traffic(workload: str, precision: str):
    e = _COLSTEP_TRAFFIC.get((workload, precision))
    if e is None:
        return None
    try:
        return e[0] if _colstep_sources_sha() == e[1] else None
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def job_throughput(local_ms, steps, k, world, device):
    """Whole-job pivots/s: every rank factorises `steps` problems to rank k;
    the job takes as long as its slowest rank (max over ranks of the timed
    region).  Returns (max_ms, pivots per second over all ranks)."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps * k / (total_ms / 1e3)


def batched_measure(args):
    """Batched workload (uneven Matern-5/2 instances, N log-uniform in
    [2000, 50000], d in {8, 16, 32}, k uniform in [100, 1000]): T per shape
    class from the autotuner, then all instances in one batch launch, timed
    with CUDA events, against the same instances run one after another."""
    import torch
    import paper_2410_03969_gb300 as rp
    from paper_2410_03969_gb300 import autotune
    probs = workloads.batched_matern(0, count=args.batched)
    tuner = autotune.Autotuner(precision="mixed", repeats=1)
    t0 = time.perf_counter()
    Ts = []
    for i, p in enumerate(probs):
        Ts.append(tuner.choose(p.X, p.kernel, p.sigma, p.k))
        if i % 32 == 31:
            log("  autotuned %d/%d instances (%d classes)" % (i + 1, len(probs), len(tuner.cache)))
    tune_s = time.perf_counter() - t0
    fs = [rp.Factorizer(p.X, p.kernel, p.sigma, k_max=p.k, T_max=T, precision="mixed",
                        instance=i) for i, (p, T) in enumerate(zip(probs, Ts))]
    ks = [p.k for p in probs]
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def one_by_one(seed):
        for i, (f, T) in enumerate(zip(fs, Ts)):
            f.run(ks[i], T, seed + i)

    log("  %d contexts created" % len(fs))
    one_by_one(7)  # record each context's graph
    log("  one by one done")
    seq_ms = min(timed(lambda: one_by_one(100 + 1000 * r)) for r in range(2))
    execs = {}
    with rp.Batch(fs, Ts) as b:
        log("  batch set up")
        for name, mode in (("graph", rp.BATCH_GRAPH), ("engine", rp.BATCH_ENGINE)):
            b.mode = mode
            b.run(ks, [7 + i for i in range(len(fs))])
            ms = [timed(lambda: b.run(ks, [200 + 1000 * r + i for i in range(len(fs))]))
                  for r in range(10)]
            execs[name] = {"ms_p50": _pct(ms, 50), "ms_p99": _pct(ms, 99), "launches_timed": len(ms),
                           "pivots_per_s": sum(ks) / (statistics.median(ms) / 1e3)}
            log("  %s executor: p50 %.2f ms" % (name, execs[name]["ms_p50"]))
        b.mode = rp.BATCH_GRAPH
        terr = [f.stats()["trace_error"] for f in fs[:16]]
    for f in fs:
        f.close()
    piv = sum(ks)
    classes = {}
    for p, T in zip(probs, Ts):
        classes[autotune.shape_class(p.N, p.d, p.k, p.kernel)] = T
    best = execs["graph"]
    return {"instances": len(probs), "pivots": piv, "batch_ms": best["ms_p50"],
            "batch_ms_p50": best["ms_p50"], "batch_ms_p99": best["ms_p99"],
            "pivots_per_s": best["pivots_per_s"], "one_by_one_ms": seq_ms,
            "speedup_vs_one_by_one": seq_ms / best["ms_p50"], "autotune_s": tune_s,
            "shape_classes": len(classes), "T_chosen": sorted(set(Ts)),
            "trace_error_mean_first16": statistics.mean(terr),
            "executor": "graph (the default): one CUDA graph, one conditional round loop per "
                        "instance",
            "executors": {
                "graph": dict(execs["graph"], launch="one CUDA graph launch"),
                "engine": dict(execs["engine"], launch=(
                    "one persistent kernel launch: clusters of 8 CTAs run the rounds' control "
                    "phases, any CTA the column-step tile parts, instances from a device queue "
                    "largest N k^2 first"))}}


def serving_measure(args):
    """Serving workload: Poisson arrivals (20 jobs/s) of jobs with N
    log-uniform in [1e3, 2e5], d = 32 mixture points, Gaussian or l2-Laplace,
    k uniform in [200, 2000], FP32 factors admitted by memory; p50/p99 of the
    end-to-end latency (arrival -> factor ready on the device) and the
    throughput, for the whole stream as it arrives and for the same jobs in
    one burst.  The points of each job are generated by a thread pool ahead of
    its arrival (the server copies them at submission)."""
    import queue
    from concurrent.futures import ThreadPoolExecutor
    import paper_2410_03969_gb300 as rp
    jobs = workloads.serving_stream(0, jobs=args.serving, materialize=False)
    budget, slots = 64 << 30, 16
    pool = ThreadPoolExecutor(max(2, min(16, (os.cpu_count() or 4) - 2)))

    def drive(arrivals):
        ahead = 64  # jobs generated ahead of the submitting thread
        futs = {}

        def fut(i):
            if i < len(jobs) and i not in futs:
                futs[i] = pool.submit(workloads.materialize_job, jobs[i])
            return futs.get(i)

        for i in range(ahead):
            fut(i)
        late = 0
        with rp.Server(budget, slots) as srv:
            pending, res = queue.Queue(), []

            def collect():  # oldest first: it is admitted before any later job
                for _ in range(len(arrivals)):
                    t = pending.get()
                    res.append(srv.poll(t, wait_ms=-1))
                    srv.release(t)  # the client has its result; free the memory

            th = threading.Thread(target=collect)
            th.start()
            t0 = time.perf_counter()
            for i, t_arr in enumerate(arrivals):
                p = fut(i).result()
                del futs[i]
                fut(i + ahead)
                dt = t_arr - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                elif dt < -0.005:
                    late += 1
                pending.put(srv.submit(p.X, p.kernel, p.sigma, p.k, seed=i))
            th.join()
            wall = time.perf_counter() - t0
        lat = [r["latency_ms"] for r in res]
        ok = sum(1 for r in res if r["state"] == "finished")
        return {"jobs": len(res), "finished": ok, "p50_ms": _pct(lat, 50),
                "p99_ms": _pct(lat, 99), "max_ms": max(lat),
                "mean_queue_ms": statistics.mean(r["queue_ms"] for r in res),
                "wall_s": wall, "jobs_per_s": len(res) / wall,
                "pivots_per_s": sum(r["rank"] for r in res) / wall,
                "trace_error_mean": statistics.mean(r["trace_error"] for r in res),
                "submissions_late_over_5ms": late}

    log("  %d jobs in the stream" % len(jobs))
    stream = drive([j.arrival_s for j in jobs])
    log("  stream done (%.1f s)" % stream["wall_s"])
    burst = drive([0.0] * len(jobs))
    log("  burst done (%.1f s)" % burst["wall_s"])
    pool.shutdown()
    return {"arrival": "Poisson 20 jobs/s", "jobs": len(jobs), "budget_bytes": budget,
            "slots": slots, "latency": "host time from submit to the observed completion",
            "stream": stream, "burst": burst}


def _problem(args, name=None):
    """The workload; --n-points shrinks N (small cases for profiling only)."""
    make = workloads.WORKLOADS[name or args.workload]
    return make(0, N=args.n_points) if (args.n_points and name is None) else make(0)


def _time_oracle(prob, Np, seed, threads):
    import oracle
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    out = oracle.rpc_accel(prob.k, prob.T, seed, X=prob.X[:Np], kernel=prob.kernel,
                           sigma=prob.sigma)
    return time.perf_counter() - t0, used, out["rank"]


def cpu_baseline(prob, budget_s=10.0):
    """The FP64 C oracle (accelerated RPCholesky, as it stands) on the host
    cores: with every core (OpenMP over the N-loops) on the first N' points of
    the workload, N' sized to about budget_s, and on one thread on the
    smallest sample that still reaches rank k (N1 = k + T points).  `value` is
    what the all-core run measured (k pivots over its time on N' points); the
    estimate for all N points (the time scales linearly in N at fixed k) is a
    separate key."""
    import oracle
    oracle.build()
    nproc = os.cpu_count() or 1
    N, k = prob.N, prob.k
    N1 = min(N, k + prob.T)
    t_cal, used, _ = _time_oracle(prob, N1, 0, nproc)
    Np = int(min(N, max(N1, N1 * budget_s / max(t_cal, 1e-3))))
    t_all, used, rank = _time_oracle(prob, Np, 1, nproc) if Np > N1 else (t_cal, used, k)
    t_one, used1, _ = _time_oracle(prob, N1, 2, 1)
    return {"value": k / t_all, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "FP64 C oracle, accelerated RPCholesky (Algorithm 2) to rank %d on the "
                      "first %d of %d points, %d threads: %.2f s" % (k, Np, N, used, t_all),
            "seconds": t_all, "sample_N": Np, "rank": rank,
            "single_thread": {"value": k / t_one, "unit": UNIT, "cores": used1,
                              "sample_N": N1, "seconds": t_one},
            "all_cores_on_single_thread_sample": {"sample_N": N1, "seconds": t_cal,
                                                  "cores": used},
            "estimate_full_N": {"value": k / (t_all * N / Np), "unit": UNIT,
                                "how": "measured time x N / N' (linear in N at fixed k)"}}


def reference_arm(args):
    """The oracle on the host cores as the reference implementation: the same
    workload and metric, each step one factorisation to rank k of the first N'
    points (N' sized so that W + K steps take about two minutes); the line
    reports the times it measured, on N' points."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob = _problem(args)
    import oracle
    oracle.build()
    nproc = os.cpu_count() or 1
    N, k = prob.N, prob.k
    N1 = min(N, k + prob.T)
    t_cal, used, _ = _time_oracle(prob, N1, 999, nproc)
    per_step = min(6.0, 120.0 / max(1, args.warmup + args.steps))
    Np = int(min(N, max(N1, N1 * per_step / max(t_cal, 1e-3))))
    times = []
    t_wall = time.perf_counter()
    for i in range(args.warmup + args.steps):
        t, used, _ = _time_oracle(prob, Np, 1000 + i, nproc)
        if i >= args.warmup:
            times.append(t)
    t_wall = time.perf_counter() - t_wall
    mean = sum(times) / len(times)
    value = k / mean
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": prob.name, "N": N, "d": prob.d, "k": k, "T": prob.T,
                   "kernel": prob.kernel, "sigma": prob.sigma, "precision": "fp64",
                   "l2": "n/a (host)", "parallelism": "%d host threads" % used,
                   "sample_N": Np},
        "time_to_rank_k_ms": {"p50": _pct(times, 50) * 1e3, "p99": _pct(times, 99) * 1e3},
        "wall_s": t_wall,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": "each step: FP64 C oracle, accelerated RPCholesky to rank "
                                   "%d on the first %d of %d points (the time measured)"
                                   % (k, Np, N)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "estimate_full_N": {"value": k / (mean * N / Np), "unit": UNIT,
                            "how": "measured time x N / N' (an estimate, not a measurement)"},
    }
    print(json.dumps(line))
    return 0


def _ev_time(stream, fn, flush=None):
    """CUDA-event time (ms) of fn() on `stream`, L2 flushed before (outside
    the events)."""
    import torch
    if flush is not None:
        flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def _peak_tf(peaks, dtype, sustained):
    """Dense tensor peak (TFLOP/s) for `dtype`: the measured bf16 figure (burst
    or sustained) times the nominal dtype ratio (fp16 1, tf32 1.1/2.25)."""
    bf16 = peaks.get("bf16_tflops_sustained" if sustained else "bf16_tflops", 1700.0)
    return bf16 * (1.0 if dtype == "f16" else 1.1 / 2.25)


def roofline_measure(rp, Xd, prob, prec, seed, workload, fp64_peak=None):
    """Roofline of the column step (the dominant kernel): one profiled
    factorisation (host loop, CUDA events around every phase on the launch
    stream).  The attainable time of the column-step launches is the larger
    of their algorithmic bytes at the measured HBM bandwidth and their
    executed tensor-core flops (split terms and padding included) at the
    dense peak of their dtypes; the bound is whichever is larger and
    `achieved` is that quantity over the measured time."""
    peaks, src = _peaks()
    with rp.Factorizer(Xd, prob.kernel, prob.sigma, k_max=prob.k, T_max=prob.T, precision=prec,
                       profile=True) as g:
        g.run(prob.k, prob.T, seed)
        sp = g.stats()
    col_ms = sp["phase_ms"]["colstep"]
    nl = max(1, sp["phase_launches"]["colstep"])
    phase_total = sum(sp["phase_ms"].values())
    t = col_ms / 1e3
    base = {"kernel": "column step", "launches": nl, "avg_launch_ms": col_ms / nl,
            "alg_bytes_per_launch": sp["col_bytes"] / nl,
            "alg_flops_per_launch": sp["col_flops"] / nl,
            "share_of_profiled_step": col_ms / max(phase_total, 1e-9),
            "phase_ms": sp["phase_ms"]}
    if prec == "fp64":
        achieved = sp["col_flops"] / t / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": None,
                "peak_source": "FP64 rate of a cuBLAS DGEMM (4096^3) timed in this run"}
        roof.update(base)
        return roof
    hbm = peaks["hbm_gbs"]
    t_hbm = sp["col_bytes"] / (hbm * 1e9)
    p32, p16 = _peak_tf(peaks, "tf32", True), _peak_tf(peaks, "f16", True)
    t_tc = sp["mma_flops_tf32"] / (p32 * 1e12) + sp["mma_flops_f16"] / (p16 * 1e12)
    mma = sp["mma_flops_tf32"] + sp["mma_flops_f16"]
    if t_tc > t_hbm:
        roof = {"bound": "tensor", "achieved": mma / t / 1e12, "peak": mma / t_tc / 1e12,
                "unit": "TFLOP/s", "frac": t_tc / t,
                "peak_source": "bf16_tflops_sustained of MEASURED_PEAKS.json (%s) x the nominal "
                               "ratio of each MMA kind (tf32 1.1/2.25, f16 1), weighted by the "
                               "flops of each kind" % src}
    else:
        roof = {"bound": "hbm", "achieved": sp["col_bytes"] / t / 1e9, "peak": hbm,
                "unit": "GB/s", "frac": t_hbm / t,
                "peak_source": "hbm_gbs of MEASURED_PEAKS.json (%s)" % src}
    roof["traffic"] = _colstep_traffic(workload, prec)
    roof.update(base)
    roof.update({"mma_flops_tf32_per_launch": sp["mma_flops_tf32"] / nl,
                 "mma_flops_f16_per_launch": sp["mma_flops_f16"] / nl,
                 "hbm_floor_ms": t_hbm * 1e3, "tensor_floor_ms": t_tc * 1e3,
                 "hbm_fraction": t_hbm / t, "tensor_fraction": t_tc / t})
    return roof


def plain_measure(f, k, seeds, stream, flush):
    """Simple RPCholesky (Algorithm 6) on the same context: CUDA-event time to
    rank k and trace error per seed."""
    ms, terr = [], []
    for sd in seeds:
        ms.append(_ev_time(stream, lambda: f.run_plain(k, sd), flush))
        terr.append(f.stats()["trace_error"])
    return ms, terr


def fp64_dgemm_peak():
    """FP64 rate (TFLOP/s) of cuBLAS DGEMM, 4096^3, best of 3 (the FP64 mode's
    ALU roofline; this GPU's FP64 rate is far below its tensor rates)."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e9
    for _ in range(3):
        best = min(best, _ev_time(torch.cuda.current_stream(), lambda: torch.matmul(a, b)))
    return 2.0 * 4096 ** 3 / (best / 1e3) / 1e12


def context_measure(args, rp, name, stream, flush, seed_base):
    """A second workload on the same GPU (default: mixture20_n1e5, N = 1e5):
    accelerated RPCholesky in the bench precision (p50/p99), simple
    RPCholesky, the FP64 mode (with its ALU roofline), block RPCholesky
    (Algorithm 7), the low-memory variant (Algorithm 3, FP64) and randomly
    pivoted QR (Algorithm 5, FP64 on a dense 2000 x 20000 matrix)."""
    import torch
    prob = _problem(args, name)
    k, T, prec = prob.k, prob.T, args.precision
    Xd = torch.from_numpy(prob.X).cuda()
    out = {"config": {"workload": prob.name, "N": prob.N, "d": prob.d, "k": k, "T": T,
                      "kernel": prob.kernel, "sigma": prob.sigma, "precision": prec}}
    with rp.Factorizer(Xd, prob.kernel, prob.sigma, k_max=k, T_max=T, precision=prec) as f:
        for i in range(3):
            f.run(k, T, seed_base + 900 + i)
        ms = [_ev_time(stream, lambda: f.run(k, T, seed_base + i), flush)
              for i in range(args.context_steps)]
        terr = []
        for i in range(min(5, args.context_steps)):
            f.run(k, T, seed_base + i)
            terr.append(f.stats()["trace_error"])
        out["accelerated"] = {
            "ms_p50": _pct(ms, 50), "ms_p99": _pct(ms, 99), "steps": len(ms),
            "pivots_per_s": k / (statistics.median(ms) / 1e3),
            "trace_error_mean": statistics.mean(terr),
            "trace_error_sd": statistics.pstdev(terr)}
        pm, pt = plain_measure(f, k, [seed_base + i for i in range(args.plain_steps)], stream,
                               flush)
        out["plain_gpu"] = {"ms_p50": _pct(pm, 50), "pivots_per_s": k / (statistics.median(pm) / 1e3),
                            "trace_error_mean": statistics.mean(pt), "steps": len(pm)}
        out["speedup_vs_plain_gpu"] = statistics.median(pm) / statistics.median(ms)
        out["trace_error_ratio_vs_plain_gpu"] = statistics.mean(terr) / statistics.mean(pt)
        bm, bt = [], []
        for i in range(3):
            bm.append(_ev_time(stream, lambda: f.run_block(k, T, seed_base + i), flush))
            bt.append(f.stats()["trace_error"])
        out["block_rpc_gpu"] = {"ms_p50": _pct(bm, 50), "b": T,
                                "pivots_per_s": k / (statistics.median(bm) / 1e3),
                                "trace_error_mean": statistics.mean(bt), "steps": len(bm)}
        out["trace_error_ratio_block_vs_accelerated"] = statistics.mean(bt) / statistics.mean(terr)
    out["roofline"] = roofline_measure(rp, Xd, prob, prec, seed_base, prob.name)
    log("  FP64 mode")
    fp64_peak = fp64_dgemm_peak()
    with rp.Factorizer(Xd, prob.kernel, prob.sigma, k_max=k, T_max=T, precision="fp64") as g:
        g.run(k, T, seed_base + 950)
        om, ot = [], []
        for i in range(2):
            om.append(_ev_time(stream, lambda: g.run(k, T, seed_base + i), flush))
            ot.append(g.stats()["trace_error"])
    out["fp64_mode"] = {"ms_p50": _pct(om, 50), "trace_error_mean": statistics.mean(ot),
                        "roofline": roofline_measure(rp, Xd, prob, "fp64", seed_base, prob.name,
                                                     fp64_peak=fp64_peak)}
    log("  low-memory accelerated RPCholesky (Algorithm 3, FP64)")
    free0 = torch.cuda.mem_get_info()[0]
    with rp.LowMemFactorizer(prob.X, prob.kernel, prob.sigma, k_max=k, T_max=T) as lm:
        held = free0 - torch.cuda.mem_get_info()[0]
        lms, lterr = [], []
        for i in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lm.run(k, T, seed_base + i)  # synchronous
            lms.append((time.perf_counter() - t0) * 1e3)
            lterr.append(float(lm.copy()["d"].sum()) / prob.N)
    out["lowmem_fp64"] = {
        "ms_p50": _pct(lms, 50), "pivots_per_s": k / (statistics.median(lms) / 1e3),
        "trace_error_mean": statistics.mean(lterr), "steps": len(lms),
        "device_bytes_held": held, "timing": "host wall clock (synchronous call)"}
    log("  accelerated randomly pivoted QR (Algorithm 5, FP64)")
    rng = np.random.default_rng(5)
    Mq, Nq, kq, Tq = 2000, 20000, 500, 128
    Bq = (rng.standard_normal((Mq, 400)) @ rng.standard_normal((400, Nq))
          + 0.01 * rng.standard_normal((Mq, Nq)))
    with rp.RPQR(Bq, k_max=kq, T_max=Tq) as qr:
        qms = []
        for i in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            qr.run(kq, Tq, seed_base + i)  # synchronous
            qms.append((time.perf_counter() - t0) * 1e3)
        qo = qr.copy()
    out["rpqr_fp64"] = {
        "M": Mq, "N": Nq, "k": kq, "T": Tq, "ms_p50": _pct(qms, 50),
        "pivots_per_s": kq / (statistics.median(qms) / 1e3), "rounds": qo["rounds"],
        "residual_frobenius_rel": float(np.sqrt(qo["u"].sum() / np.sum(Bq * Bq))),
        "timing": "host wall clock (synchronous call)"}
    del Xd
    return out


def small_measure(rp, stream, seeds=100):
    """The small configuration (N = 2000, d = 8, Gaussian, k = 100, T = 20) in
    FP64 mode over 100 seeds: p50/p99 of time-to-rank-k for accelerated and
    simple RPCholesky (CUDA events around each graph launch; the problem is
    far smaller than L2, so this is a latency measurement)."""
    prob = workloads.gauss8_n2000(0)
    out = {"config": {"workload": prob.name, "N": prob.N, "d": prob.d, "k": prob.k, "T": prob.T,
                      "kernel": prob.kernel, "sigma": prob.sigma, "precision": "fp64",
                      "seeds": seeds}}
    with rp.Factorizer(prob.X, prob.kernel, prob.sigma, k_max=prob.k, T_max=prob.T,
                       precision="fp64") as f:
        for name, fn in (("accelerated", lambda sd: f.run(prob.k, prob.T, sd)),
                         ("plain", lambda sd: f.run_plain(prob.k, sd))):
            for sd in range(3):
                fn(10_000 + sd)
            ms, terr = [], []
            for sd in range(seeds):
                ms.append(_ev_time(stream, lambda: fn(sd)))
                terr.append(f.stats()["trace_error"])
            out[name] = {"ms_p50": _pct(ms, 50), "ms_p99": _pct(ms, 99),
                         "pivots_per_s": prob.k / (statistics.median(ms) / 1e3),
                         "trace_error_mean": statistics.mean(terr),
                         "trace_error_sd": statistics.pstdev(terr)}
    out["speedup_vs_plain_gpu"] = out["plain"]["ms_p50"] / out["accelerated"]["ms_p50"]
    return out


def e2e_measure(rp, prob, prec, steps, seed_base):
    """End to end through the public API: create a context from pinned host X
    (copied to the device by rpchol_create), run to rank k with F streamed to
    pinned host memory round by round (rpchol_run_to_host: the copy engine
    moves each round's columns while later rounds compute), destroy; host
    wall clock per step, every copy inside."""
    import torch
    Xh = torch.from_numpy(prob.X).pin_memory()
    es = 4 if prec == "mixed" else 8
    Fh = torch.empty((prob.N, prob.k), dtype=torch.float32 if es == 4 else torch.float64,
                     pin_memory=True)
    Ph = torch.empty(prob.k, dtype=torch.int64, pin_memory=True)
    em = []
    for i in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with rp.Factorizer(Xh, prob.kernel, prob.sigma, k_max=prob.k, T_max=prob.T,
                           precision=prec) as g:
            g.run_to_host(prob.k, prob.T, seed_base + i, Fh.data_ptr(), prob.k, Ph.data_ptr())
        em.append(time.perf_counter() - t0)
    e2e_t = statistics.median(em)
    return {"value": prob.k / e2e_t, "unit": UNIT, "ms_p50": e2e_t * 1e3, "steps": steps,
            "h2d_bytes_per_step": int(prob.X.nbytes),
            "d2h_bytes_per_step": int(prob.N * prob.k * es + prob.k * 8),
            "path": "rpchol_create from pinned host X, rpchol_run_to_host to pinned host F and "
                    "pivots (columns copied round by round during the run), destroy"}


def ours_arm(args):
    import torch
    import torch.distributed as dist
    import paper_2410_03969_gb300 as rp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    rp.lib()
    prob = _problem(args)
    k, T = prob.k, prob.T
    prec = args.precision
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(prob.X).cuda()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    f = rp.Factorizer(Xd, prob.kernel, prob.sigma, k_max=k, T_max=T, precision=prec,
                      use_graph=not args.no_graph)
    seed_base = 1000 * (rank + 1)
    for i in range(args.warmup):
        f.run(k, T, seed_base + 900 + i)
    torch.cuda.synchronize()

    log("timed region")
    # ---- timed region: K factorisations, per-step CUDA events, L2 flushed between steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            f.run(k, T, seed_base + i)
            evs[i][1].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    # per-step trace error and round counts (re-run the same seeds, outside timing)
    terr, rounds, kl, accepted_rate = [], [], [], []
    for i in range(min(args.steps, 5)):
        f.run(k, T, seed_base + i)
        st = f.stats()
        terr.append(st["trace_error"])
        rounds.append(st["rounds"])
        kl.append(st["kernel_launches"])
        accepted_rate.append(st["accepted"] / max(1, st["proposals"]))
    st_last = f.stats()
    launches = int(round(args.steps * sum(kl) / len(kl)))
    total_ms, value = job_throughput(total_ms, args.steps, k, world, "cuda")
    ms_per_step = total_ms / args.steps

    extra = {}
    if rank == 0 and not args.quick:
        if args.plain_steps > 0:
            log("simple RPCholesky on the same GPU and workload")
            pm, pterr = plain_measure(f, k, [seed_base + i for i in range(args.plain_steps)],
                                      stream, flush)
            extra["plain_gpu"] = {
                "ms_p50": _pct(pm, 50), "ms": pm,
                "pivots_per_s": k / (statistics.median(pm) / 1e3),
                "trace_error_mean": statistics.mean(pterr), "steps": len(pm), "precision": prec,
                "alg_bytes": f.stats()["col_bytes"]}
            extra["plain_gpu"]["hbm_fraction"] = (
                extra["plain_gpu"]["alg_bytes"] / (statistics.median(pm) / 1e3)
                / (_peaks()[0]["hbm_gbs"] * 1e9))
            extra["speedup_vs_plain_gpu"] = statistics.median(pm) / statistics.median(step_ms)
            extra["trace_error_ratio_vs_plain_gpu"] = statistics.mean(terr) / statistics.mean(pterr)
        f.close()
        log("roofline of the dominant kernel")
        extra["roofline"] = roofline_measure(rp, Xd, prob, prec, seed_base, args.workload)
        del Xd
        log("end to end through the public API with host buffers")
        extra["e2e"] = e2e_measure(rp, prob, prec, args.e2e_steps, seed_base)
        if not args.no_cpu_baseline:
            log("cpu baseline (oracle)")
            extra["cpu_baseline"] = cpu_baseline(prob, budget_s=args.cpu_budget)
        log("small configuration, 100 seeds")
        extra["gauss8_n2000"] = small_measure(rp, stream)
        if args.context_workload and args.context_workload != args.workload:
            log("second workload: %s" % args.context_workload)
            extra[args.context_workload] = context_measure(args, rp, args.context_workload,
                                                           stream, flush, seed_base)
        if args.batched:
            log("batched workload")
            extra["batched"] = batched_measure(args)
        if args.serving:
            log("serving workload")
            extra["serving"] = serving_measure(args)
    else:
        f.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32x3/f32+f64" if prec == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": prob.name, "N": prob.N, "d": prob.d, "k": k, "T": T,
                       "kernel": prob.kernel, "sigma": prob.sigma, "precision": prec,
                       "l2": "flushed between steps (256 MiB write, outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_rank_k_ms": {"p50": _pct(step_ms, 50), "p99": _pct(step_ms, 99),
                                  "mean": statistics.mean(step_ms),
                                  "min": min(step_ms), "max": max(step_ms)},
            "trace_error": {"mean": statistics.mean(terr),
                            "sd": statistics.pstdev(terr) if len(terr) > 1 else 0.0},
            "rounds_mean": statistics.mean(rounds),
            "acceptance_rate": statistics.mean(accepted_rate),
            "wall_s_timed_region": t_wall,
            "clocks": clk.summary(),
            "gpu_launches": launches,
            "status": st_last["status"],
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def colgen_measure(args):
    """Columns of F formed per second by one block step of size b (block
    RPCholesky to rank b: draws, H, Cholesky, fused column step), against b,
    on N standard Gaussian points with sigma = 1 (the setting of the paper's
    Fig. 1, which times the generation of b kernel columns)."""
    import torch
    import paper_2410_03969_gb300 as rp
    rp.lib()
    N = args.n_points or 100_000
    rows = []
    for kern in ("gaussian", "laplace_l1"):
        for d in (10, 100, 1000):
            X = torch.from_numpy(workloads.gaussian_cloud(N, d, 0)).cuda()
            with rp.Factorizer(X, kern, 1.0, k_max=256, T_max=256,
                               precision=args.precision) as f:
                for b in (1, 2, 4, 8, 16, 32, 64, 128, 256):
                    ms, cols = [], []
                    for i in range(8):
                        e0, e1 = (torch.cuda.Event(enable_timing=True),
                                  torch.cuda.Event(enable_timing=True))
                        e0.record()
                        f.run_block(b, b, 77 + i)
                        e1.record()
                        torch.cuda.synchronize()
                        st = f.stats()
                        if i >= 3:
                            ms.append(e0.elapsed_time(e1))
                            cols.append(st["rank"])
                    med = statistics.median(ms)
                    rows.append({"kernel": kern, "d": d, "b": b, "ms_p50": med,
                                 "columns_per_s": statistics.mean(cols) / (med / 1e3),
                                 "status": st["status"]})
            del X
    print(json.dumps({"metric": "columns_per_s_vs_block_size", "N": N,
                      "precision": args.precision, "rows": rows}))
    return 0


def profile_case(args):
    """One run of Algorithm 3 or Algorithm 5 on a fixed case, for ncu captures
    (no bench line): lowmem = the bench workload to rank k; rpqr = a dense
    2000 x 20000 matrix to rank 500 with T = 128."""
    import torch
    import paper_2410_03969_gb300 as rp
    rp.lib()
    if args.profile_case == "lowmem":
        prob = _problem(args)
        with rp.LowMemFactorizer(prob.X, prob.kernel, prob.sigma, k_max=prob.k,
                                 T_max=prob.T) as lm:
            out = lm.run(prob.k, prob.T, 1).copy()
        print(json.dumps({"case": "lowmem", "rank": out["rank"], "rounds": out["rounds"]}))
    else:
        rng = np.random.default_rng(5)
        B = (rng.standard_normal((2000, 400)) @ rng.standard_normal((400, 20000))
             + 0.01 * rng.standard_normal((2000, 20000)))
        with rp.RPQR(B, k_max=500, T_max=128) as qr:
            out = qr.run(500, 128, 1).copy()
        print(json.dumps({"case": "rpqr", "rank": out["rank"], "rounds": out["rounds"]}))
    torch.cuda.synchronize()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="unif64_n1e6", choices=list(workloads.WORKLOADS))
    ap.add_argument("--context-workload", default="mixture20_n1e5",
                    help="second workload reported under its own key ('' = skip)")
    ap.add_argument("--context-steps", type=int, default=10)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", type=int, default=256,
                    help="instances of the batched workload to time (0 = skip)")
    ap.add_argument("--serving", type=int, default=2000,
                    help="jobs of the serving workload to time (0 = skip)")
    ap.add_argument("--quick", action="store_true", help="timed region only")
    ap.add_argument("--n-points", type=int, default=0,
                    help="override N of the workload (small profiling cases; not a bench line)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven round loop (one launch per kernel), e.g. for ncu")
    ap.add_argument("--colgen", action="store_true",
                    help="columns per second against the block size (no bench line)")
    ap.add_argument("--profile-case", choices=["lowmem", "rpqr"], default=None,
                    help="one run of Algorithm 3 or 5 for profiling (no bench line)")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args)
    if args.colgen:
        return colgen_measure(args)
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
