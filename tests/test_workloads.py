"""The seeded synthetic inputs follow their stated recipes (CPU only)."""
import numpy as np
import pytest

import workloads


def test_gaussian_cloud_is_seeded_fp32():
    a = workloads.gaussian_cloud(500, 7, 3)
    b = workloads.gaussian_cloud(500, 7, 3)
    c = workloads.gaussian_cloud(500, 7, 4)
    assert a.dtype == np.float32 and a.shape == (500, 7) and a.flags["C_CONTIGUOUS"]
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    big = workloads.gaussian_cloud(200_000, 2, 0).astype(np.float64)
    assert abs(big.mean()) < 0.01 and abs(big.std() - 1.0) < 0.01


def test_mixture_recipe():
    X = workloads.gaussian_mixture(40_000, 20, 1).astype(np.float64)
    # means ~ N(0, 9 I), unit noise: per-coordinate variance about 10 in total,
    # and within-component variance 1 (10 well separated clusters)
    assert 6.0 < X.var(axis=0).mean() < 14.0
    g = np.random.Generator(np.random.PCG64([1, 2]))
    means = 3.0 * g.standard_normal((10, 20))
    comp = g.integers(0, 10, size=40_000)
    resid = X - means[comp]
    assert abs(resid.std() - 1.0) < 0.01
    assert np.bincount(comp, minlength=10).min() > 3500


def test_uniform_with_outliers_recipe():
    X = workloads.uniform_with_outliers(50_000, 64, 2).astype(np.float64)
    scaled = np.max(X, axis=1) >= 1.0
    assert scaled.sum() == 500  # 1% of the rows, scaled by 10
    assert X.min() >= 0.0 and X[~scaled].max() < 1.0 and X.max() < 10.0


def test_bandwidth_heuristics():
    X = np.array([[0.0, 0.0], [3.0, 4.0]], dtype=np.float32)
    assert workloads.median_pairs_bandwidth(X, 0, pairs=11) == 5.0  # never i == j
    Y = workloads.gaussian_cloud(300, 3, 5)
    D = np.sqrt(((Y[:, None, :].astype(np.float64) - Y[None, :, :]) ** 2).sum(-1))
    iu = np.triu_indices(300, 1)
    assert workloads.median_subsample_bandwidth(Y, 0, m=300) == pytest.approx(
        np.median(D[iu]), rel=1e-12)


def test_named_workloads_sizes():
    p = workloads.mixture20_n1e5(0, N=5000)
    assert (p.N, p.d, p.kernel, p.k, p.T) == (5000, 20, "gaussian", 1000, 120)
    assert p.sigma == workloads.median_pairs_bandwidth(p.X, 0, 1000)
    q = workloads.gauss8_n2000(0)
    assert (q.N, q.d, q.sigma, q.k, q.T) == (2000, 8, 1.0, 100, 20)
    u = workloads.unif64_n1e6(0, N=4000)
    assert (u.d, u.kernel, u.k, u.T) == (64, "laplace_l2", 4000, 200)


def test_batched_and_serving_recipes():
    probs = workloads.batched_matern(0, count=12)
    assert len(probs) == 12
    for p in probs:
        assert 2000 <= p.N <= 50000 and p.d in (8, 16, 32) and 100 <= p.k <= 1000
        assert p.kernel == "matern52" and p.sigma > 0
    jobs = workloads.serving_stream(0, jobs=2000, materialize=False)
    t = np.array([j.arrival_s for j in jobs])
    assert np.all(np.diff(t) > 0)
    assert np.mean(np.diff(t)) == pytest.approx(1 / 20.0, rel=0.1)  # Poisson, 20 jobs/s
    frac = np.mean([j.problem.kernel == "gaussian" for j in jobs])
    assert 0.45 < frac < 0.55
    assert all(1000 <= j.problem.meta["N"] <= 200000 for j in jobs)
