"""Seeded synthetic inputs for randomly pivoted Cholesky.

This module holds input generation only, none of the method's arithmetic.
Both the FP64 oracle (through the tests) and the CUDA path (through the
tests and the benchmark) take their points from here, so that both sides
see identical inputs.

The paper's real data sets (LIBSVM / OpenML / UCI, sGDML molecules) are not
available; these generators stand in for the paper's random point-cloud
testbed (Sec. 3.1: standard Gaussian clouds, N up to 1e5, Gaussian /
Matern / Laplace kernels with the median-distance bandwidth).

Recipe shared by every workload:
  * points are drawn in FP64 with numpy's PCG64 generator seeded by the
    workload seed, then rounded once to FP32; that FP32 set is what every
    mode (oracle FP64, GPU FP64, GPU mixed) factorises;
  * the bandwidth sigma, where it is the median heuristic, is computed here
    in FP64 from the FP32 points and passed to both sides as a number.

Workloads (sizes named by what they are):
  gauss8_n2000       N=2000, d=8, x ~ N(0, I); Gaussian kernel, sigma = 1;
                     k = 100, T = 20.
  mixture20_n1e5     N=1e5, d=20, 10-component Gaussian mixture (means
                     ~ N(0, 9 I), unit covariance, equal weights); Gaussian
                     kernel, sigma = median distance of 1000 sampled pairs;
                     k = 1000, T = 120.
  unif64_n1e6        N=1e6, d=64, x ~ U[0,1]^64 with 1% of the points (drawn
                     without replacement) scaled by 10; l2-Laplace kernel
                     exp(-||x-y||/sigma), sigma = median heuristic over 1000
                     distinct points; k = 4000, T = 200.
  batched_matern     256 instances; N log-uniform in [2000, 50000],
                     d uniform in {8,16,32}, x ~ N(0, I); Matern-5/2 kernel,
                     sigma = median heuristic; k uniform in [100, 1000].
  serving_stream     jobs with Poisson arrivals at 20/s; N log-uniform in
                     [1000, 200000]; d = 32 mixture points; Gaussian or
                     l2-Laplace (probability 1/2 each); k uniform in
                     [200, 2000] (capped at N); sigma = median heuristic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KERNEL_NAMES = ("gaussian", "laplace_l2", "matern52")


@dataclass
class Problem:
    """One factorisation problem: points X (N x d, float32) and a kernel."""
    name: str
    X: np.ndarray
    kernel: str
    sigma: float
    k: int
    T: int
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _to_f32(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))


def gaussian_cloud(N: int, d: int, seed: int) -> np.ndarray:
    return _to_f32(_rng(seed, 1).standard_normal((N, d)))


def gaussian_mixture(N: int, d: int, seed: int, components: int = 10,
                     mean_std: float = 3.0) -> np.ndarray:
    g = _rng(seed, 2)
    means = mean_std * g.standard_normal((components, d))
    comp = g.integers(0, components, size=N)
    return _to_f32(means[comp] + g.standard_normal((N, d)))


def uniform_with_outliers(N: int, d: int, seed: int, frac: float = 0.01,
                          scale: float = 10.0) -> np.ndarray:
    g = _rng(seed, 3)
    x = g.random((N, d))
    n_out = int(round(frac * N))
    if n_out > 0:
        idx = g.choice(N, size=n_out, replace=False)
        x[idx] *= scale
    return _to_f32(x)


def _middle(v: np.ndarray) -> float:
    v = np.sort(np.asarray(v, dtype=np.float64))
    n = len(v)
    if n % 2:
        return float(v[n // 2])
    return float(0.5 * (v[n // 2 - 1] + v[n // 2]))


def median_pairs_bandwidth(X: np.ndarray, seed: int, pairs: int = 1000) -> float:
    """Median l2 distance of `pairs` random pairs (i != j), FP64."""
    g = _rng(seed, 4)
    N = X.shape[0]
    i = g.integers(0, N, size=pairs)
    j = g.integers(0, N - 1, size=pairs)
    j = j + (j >= i)
    diff = X[i].astype(np.float64) - X[j].astype(np.float64)
    return _middle(np.sqrt((diff * diff).sum(axis=1)))


def median_subsample_bandwidth(X: np.ndarray, seed: int, m: int = 1000) -> float:
    """Median pairwise l2 distance among m distinct random points, FP64."""
    from scipy.spatial.distance import pdist
    g = _rng(seed, 5)
    N = X.shape[0]
    m = min(m, N)
    idx = g.choice(N, size=m, replace=False)
    Y = X[idx].astype(np.float64)
    # all m (m - 1) / 2 distances by direct differences (scipy's C loop)
    return _middle(pdist(Y, "euclidean"))


def gauss8_n2000(seed: int = 0, N: int = 2000) -> Problem:
    X = gaussian_cloud(N, 8, seed)
    return Problem("gauss8_n2000", X, "gaussian", 1.0, k=min(100, N), T=20)


def mixture20_n1e5(seed: int = 0, N: int = 100_000) -> Problem:
    X = gaussian_mixture(N, 20, seed)
    sigma = median_pairs_bandwidth(X, seed, 1000)
    return Problem("mixture20_n1e5", X, "gaussian", sigma, k=min(1000, N), T=120)


def unif64_n1e6(seed: int = 0, N: int = 1_000_000) -> Problem:
    X = uniform_with_outliers(N, 64, seed)
    sigma = median_subsample_bandwidth(X, seed, 1000)
    return Problem("unif64_n1e6", X, "laplace_l2", sigma, k=min(4000, N), T=200)


def batched_matern(seed: int = 0, count: int = 256, n_lo: int = 2000, n_hi: int = 50000,
                   k_lo: int = 100, k_hi: int = 1000) -> list[Problem]:
    g = _rng(seed, 6)
    out = []
    for i in range(count):
        N = int(math.floor(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(g.choice([8, 16, 32]))
        k = int(min(g.integers(k_lo, k_hi + 1), N))
        sub = int(g.integers(0, 2**31 - 1))
        X = gaussian_cloud(N, d, sub)
        sigma = median_subsample_bandwidth(X, sub, 1000)
        out.append(Problem("batched_matern[%d]" % i, X, "matern52", sigma, k=k, T=0,
                           meta={"seed": sub}))
    return out


@dataclass
class Job:
    arrival_s: float
    problem: Problem


def serving_stream(seed: int = 0, jobs: int = 2000, rate_per_s: float = 20.0,
                   n_lo: int = 1000, n_hi: int = 200000, k_lo: int = 200, k_hi: int = 2000,
                   d: int = 32, materialize: bool = True) -> list[Job]:
    """Job list of the serving workload; with materialize=False the points are
    left as None (their seed is in meta) so that long streams stay cheap."""
    g = _rng(seed, 7)
    t = 0.0
    out = []
    for i in range(jobs):
        t += float(g.exponential(1.0 / rate_per_s))
        N = int(math.floor(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        k = int(min(g.integers(k_lo, k_hi + 1), N))
        kernel = "gaussian" if g.random() < 0.5 else "laplace_l2"
        sub = int(g.integers(0, 2**31 - 1))
        X = gaussian_mixture(N, d, sub) if materialize else None
        sigma = median_subsample_bandwidth(X, sub, 1000) if materialize else float("nan")
        out.append(Job(t, Problem("serving[%d]" % i, X, kernel, sigma, k=k, T=0,
                                  meta={"seed": sub, "N": N, "d": d})))
    return out


def materialize_job(job: Job) -> Problem:
    p = job.problem
    if p.X is not None:
        return p
    sub = p.meta["seed"]
    X = gaussian_mixture(p.meta["N"], p.meta["d"], sub)
    sigma = median_subsample_bandwidth(X, sub, 1000)
    return Problem(p.name, X, p.kernel, sigma, k=p.k, T=p.T, meta=p.meta)


WORKLOADS = {
    "gauss8_n2000": gauss8_n2000,
    "mixture20_n1e5": mixture20_n1e5,
    "unif64_n1e6": unif64_n1e6,
}
