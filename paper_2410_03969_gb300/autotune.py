"""Block-size autotuner for accelerated RPCholesky runs.

The block size T (Algorithm 2's b) trades the number of rounds (fewer with a
larger T, as long as most proposals are accepted) against the work that
grows with T: H and Algorithm 1 are O(T^2) and O(T^3) per round and are
latency-bound on the GPU, and rejected proposals are wasted.  Where the
balance lies depends on N, d, k, the kernel and the spectrum, so the tuner
measures: for each shape class (kernel, d, log2 N, k in steps of 250) it
times complete factorisations of the first instance of that class at every
candidate T on the device (CUDA events, after one untimed run) and keeps
the fastest.  Results are cached per class, in memory and optionally in a
JSON file.  The tile shape of the column step is fixed (128-row tiles, one
per TMEM lane), so T is the tuned parameter of a factorisation.

For a batch, `choose_executor` times both executors (one CUDA graph with a
conditional round loop per instance, or one persistent kernel over a device
instance queue) on the batch itself and keeps the faster one: which wins
depends on the mix of instance sizes.
"""
from __future__ import annotations

import json
import math
import os

from . import BATCH_ENGINE, BATCH_GRAPH, Factorizer

CANDIDATES = (32, 64, 96, 120, 128, 160, 200, 256)


def shape_class(N: int, d: int, k: int, kernel: str) -> str:
    return "%s/d%d/n2^%d/k%d" % (kernel, d, int(round(math.log2(max(N, 2)))),
                                 250 * ((k + 249) // 250))


class Autotuner:
    def __init__(self, candidates=CANDIDATES, precision: str = "mixed", repeats: int = 2,
                 cache_path: str | None = None, seed: int = 12345):
        self.candidates = tuple(int(t) for t in candidates)
        self.precision = precision
        self.repeats = int(repeats)
        self.cache_path = cache_path
        self.seed = int(seed)
        self.cache: dict[str, int] = {}
        self.timings: dict[str, dict[int, float]] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = {k: int(v) for k, v in json.load(f).items()}

    def choose(self, X, kernel: str, sigma: float, k: int) -> int:
        import torch
        N, d = X.shape
        key = shape_class(N, d, k, kernel)
        if key in self.cache:
            return self.cache[key]
        cands = [t for t in self.candidates if t <= N] or [1]
        times = {}
        stream = torch.cuda.current_stream()
        with Factorizer(X, kernel, sigma, k_max=k, T_max=max(cands),
                        precision=self.precision) as f:
            for T in cands:
                f.run(k, T, self.seed)  # untimed: graph recording, caches
                ms = []
                for r in range(self.repeats):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    f.run(k, T, self.seed + 1 + r)
                    b.record(stream)
                    b.synchronize()
                    ms.append(a.elapsed_time(b))
                times[T] = sorted(ms)[len(ms) // 2]
        best = min(times, key=times.get)
        self.cache[key] = best
        self.timings[key] = times
        if self.cache_path:
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
        return best


def choose_executor(batch, k, seeds, repeats: int = 3):
    """Time the batch on each executor it supports (after one untimed run
    each), leave it on the faster one and return (mode, {mode: ms})."""
    import torch
    from . import RpcholError
    stream = torch.cuda.current_stream()
    times = {}
    for mode in (BATCH_GRAPH, BATCH_ENGINE):
        try:
            batch.mode = mode
        except RpcholError:
            continue  # a member the engine cannot run
        batch.run(k, seeds)
        ms = []
        for r in range(repeats):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.run(k, [int(s) + 1 + r for s in seeds])
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        times[mode] = sorted(ms)[len(ms) // 2]
    best = min(times, key=times.get)
    batch.mode = best
    return best, times
