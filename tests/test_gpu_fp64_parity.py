"""GPU FP64 mode against the FP64 oracle, element by element.

Both sides draw from the same Philox stream, so the pivot sequences must be
identical; a divergence is tolerated only at a decision whose margin lies
within 1e-12 (the proposal map's running sum within 1e-12 W of U W, or the
acceptance ratio h/u within 1e-12 of its uniform).  F must agree to 1e-10
relative Frobenius error and d to 1e-12 (absolute, A_jj = 1).
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from divergence import accel_divergence, plain_divergence

pytestmark = pytest.mark.gpu

F_TOL = 1e-10
D_TOL = 1e-12


@pytest.fixture(scope="module")
def rp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_03969_gb300 as rp
    rp.lib()
    return rp


def compare(rp_mod, prob, seed, T, plain=False, precision="fp64"):
    X, kern, sg = prob.X, prob.kernel, prob.sigma
    k = prob.k
    with rp_mod.Factorizer(X, kern, sg, k_max=k, T_max=max(T, 1), precision=precision) as f:
        (f.run_plain(k, seed) if plain else f.run(k, T, seed)).sync()
        g = f.copy_factor()
        st = f.stats()
    o = (oracle.rpc_plain(k, seed, X=X, kernel=kern, sigma=sg) if plain
         else oracle.rpc_accel(k, T, seed, X=X, kernel=kern, sigma=sg))
    return g, o, st


def assert_parity(g, o, prob, seed, T, plain=False):
    """'identical' when the pivot sequences agree (then F to 1e-10 and d to
    1e-12); otherwise the divergence must be an allowed near-tie, named by
    the analyser, and the columns of F formed before the round of the
    divergence must still agree to 1e-10.  Returns the description."""
    if plain:
        div = plain_divergence(prob.X, prob.kernel, prob.sigma, prob.k, seed, g["S"], o["S"])
    else:
        div = accel_divergence(prob.X, prob.kernel, prob.sigma, prob.k, T, seed, g["S"], o["S"])
    if div is None:
        assert g["rank"] == o["rank"]
        Fo, Fg = o["F"], g["F"]
        err = np.linalg.norm(Fg - Fo) / max(np.linalg.norm(Fo), 1e-300)
        assert err <= F_TOL, err
        assert np.max(np.abs(g["d"] - o["d"])) <= D_TOL
        return "identical"
    assert div["allowed"], "pivot divergence without a near-tie: %r" % (div,)
    r0 = div["rank0"]
    if r0 > 0:
        Fo, Fg = o["F"][:, :r0], g["F"][:, :r0]
        err = np.linalg.norm(Fg - Fo) / max(np.linalg.norm(Fo), 1e-300)
        assert err <= F_TOL, err
    return "allowed near-tie: %r" % (div,)


def small_problem(N, d, kernel, sigma, k, seed=0):
    X = workloads.gaussian_cloud(N, d, seed)
    return workloads.Problem("gauss%d_n%d" % (d, N), X, kernel, sigma, k=k, T=0)


def test_gauss8_n2000_accelerated_100_seeds(rp):
    """The small configuration (N = 2000, d = 8, Gaussian, k = 100, T = 20) on
    100 seeds: the same points, a fresh Philox stream per seed."""
    prob = workloads.gauss8_n2000(0)
    res = []
    with rp.Factorizer(prob.X, prob.kernel, prob.sigma, k_max=prob.k, T_max=prob.T,
                       precision="fp64") as f:
        for seed in range(100):
            f.run(prob.k, prob.T, seed).sync()
            g = f.copy_factor()
            st = f.stats()
            assert st["rank"] == prob.k and st["status"] == 0
            o = oracle.rpc_accel(prob.k, prob.T, seed, X=prob.X, kernel=prob.kernel,
                                 sigma=prob.sigma)
            res.append(assert_parity(g, o, prob, seed, prob.T))
    assert sum(r == "identical" for r in res) >= 99, res


def test_gauss8_n2000_plain_100_seeds(rp):
    prob = workloads.gauss8_n2000(0)
    res = []
    with rp.Factorizer(prob.X, prob.kernel, prob.sigma, k_max=prob.k, T_max=1,
                       precision="fp64") as f:
        for seed in range(100):
            f.run_plain(prob.k, seed).sync()
            g = f.copy_factor()
            o = oracle.rpc_plain(prob.k, seed, X=prob.X, kernel=prob.kernel, sigma=prob.sigma)
            res.append(assert_parity(g, o, prob, seed, 1, plain=True))
    assert sum(r == "identical" for r in res) >= 99, res


@pytest.mark.parametrize("seed", range(3))
def test_gauss8_other_point_sets(rp, seed):
    prob = workloads.gauss8_n2000(seed + 1)
    g, o, st = compare(rp, prob, seed, prob.T)
    assert assert_parity(g, o, prob, seed, prob.T) == "identical"
    assert st["rank"] == prob.k and st["status"] == 0


@pytest.mark.parametrize("N,d,kernel,sigma,k,T", [
    (1000, 3, "gaussian", 0.7, 60, 7),      # several tiles, ragged tail (1000 = 7*128 + 104)
    (1000, 3, "laplace_l2", 1.5, 90, 33),   # block of G spans two 32-column blocks
    (1300, 5, "matern52", 2.0, 150, 120),
    (640, 2, "gaussian", 0.3, 200, 256),    # T beyond the shared-memory triangle (global path)
    (257, 4, "laplace_l2", 1.0, 40, 1),     # T = 1: accelerated == simple
    (129, 6, "matern52", 1.0, 129, 16),     # k = N
    (1000, 4, "matern32", 1.2, 80, 24),     # Matern-3/2
    (900, 5, "laplace_l1", 5.0, 70, 20),    # l1-Laplace: direct l1 distances everywhere
])
def test_shapes_and_kernels(rp, N, d, kernel, sigma, k, T):
    prob = small_problem(N, d, kernel, sigma, k)
    res = []
    for seed in (1, 2):
        g, o, st = compare(rp, prob, seed, T)
        res.append(assert_parity(g, o, prob, seed, T))
        assert st["status"] == 0
    assert res.count("identical") >= 1, res


def test_rank_stops_at_exhaustion(rp):
    # duplicated points: rank(A) = 5, so sum(d) reaches (numerically) zero or the
    # residual is at rounding level; GPU and oracle agree
    base = workloads.gaussian_cloud(5, 3, 4)
    X = np.repeat(base, 8, axis=0)
    prob = workloads.Problem("dup", X, "gaussian", 1.0, k=5, T=0)
    g, o, st = compare(rp, prob, 3, 4)
    assert g["rank"] == 5
    assert sorted(X[g["S"]].tolist()) == sorted(base.tolist())


@pytest.mark.parametrize("seed", [77, 78, 79])
def test_numerically_rank_deficient_stops_like_the_oracle(rp, seed):
    """1-D points under a Gaussian kernel (numerical rank about 20): with the
    residual floor (weights at the rounding level are exhausted) both sides stop with every weight at zero,
    long before the round limit, with the oracle's pivots (or an allowed
    near-tie) and status 0; asked for rank 130, the rank reached is small."""
    X = np.random.default_rng(11).standard_normal((1000, 1)).astype(np.float32)
    prob = workloads.Problem("gauss1_n1000", X, "gaussian", 1.0, k=130, T=0)
    g, o, st = compare(rp, prob, seed, 16)
    assert st["status"] == 0
    assert g["rank"] < 40 and o["rank"] < 40
    assert float(np.sum(g["d"])) == 0.0 and float(np.sum(o["d"])) == 0.0
    div = accel_divergence(prob.X, prob.kernel, prob.sigma, prob.k, 16, seed, g["S"], o["S"])
    assert div is None or div["allowed"], div
    if div is None:
        # the last pivots have residuals near the floor, so rounding
        # differences in their columns are amplified; the approximations
        # F F^* agree to the floor's level
        Ag, Ao = g["F"] @ g["F"].T, o["F"] @ o["F"].T
        assert np.max(np.abs(Ag - Ao)) < 1e-10


def test_tiny_edge_cases(rp):
    X = np.array([[0.5, -1.0]], dtype=np.float32)
    with rp.Factorizer(X, "gaussian", 1.0, k_max=1, T_max=4) as f:
        f.run(1, 4, 0).sync()
        g = f.copy_factor()
    assert g["rank"] == 1 and g["S"][0] == 0 and g["F"][0, 0] == 1.0
    with pytest.raises(rp.RpcholError):
        rp.Factorizer(X, "gaussian", 1.0, k_max=2, T_max=4)


def test_host_loop_equals_graph(rp):
    prob = workloads.gauss8_n2000(9)
    outs = []
    for use_graph in (True, False):
        with rp.Factorizer(prob.X, prob.kernel, prob.sigma, k_max=prob.k, T_max=prob.T,
                           use_graph=use_graph) as f:
            f.run(prob.k, prob.T, 9).sync()
            outs.append(f.copy_factor())
    assert np.array_equal(outs[0]["S"], outs[1]["S"])
    assert np.array_equal(outs[0]["F"], outs[1]["F"])


def test_repeat_runs_are_deterministic(rp):
    prob = workloads.gauss8_n2000(1)
    with rp.Factorizer(prob.X, prob.kernel, prob.sigma, k_max=prob.k, T_max=prob.T) as f:
        a = f.run(prob.k, prob.T, 5).sync().copy_factor()
        b = f.run(prob.k, prob.T, 5).sync().copy_factor()
        c = f.run(prob.k, prob.T, 6).sync().copy_factor()
    assert np.array_equal(a["S"], b["S"]) and np.array_equal(a["F"], b["F"])
    assert not np.array_equal(a["S"], c["S"])


def test_mixture20_n1e5_full_size_matches_oracle(rp):
    """The N = 1e5 configuration at full size (d = 20 mixture, Gaussian with
    the median bandwidth, k = 1000, T = 120) in FP64 mode against the oracle
    (Algorithm 2 with Algorithm 1, all N rows): identical pivots, F to 1e-10
    relative Frobenius error and d to 1e-12, or an allowed near-tie."""
    import torch
    import oracle as orc
    orc.set_threads(os.cpu_count() or 1)
    prob = workloads.mixture20_n1e5(0)
    Xd = torch.from_numpy(prob.X).cuda()
    res = []
    for seed in (0, 1):
        with rp.Factorizer(Xd, prob.kernel, prob.sigma, k_max=prob.k, T_max=prob.T,
                           precision="fp64") as f:
            f.run(prob.k, prob.T, seed).sync()
            g = f.copy_factor()
            st = f.stats()
        assert st["rank"] == prob.k and st["status"] == 0
        o = orc.rpc_accel(prob.k, prob.T, seed, X=prob.X, kernel=prob.kernel, sigma=prob.sigma)
        res.append(assert_parity(g, o, prob, seed, prob.T))
        del g, o
    assert res.count("identical") >= 1, res


def test_mixture20_full_size_sampled_rows(rp):
    """mixture20_n1e5 at its full size (N=1e5, k=1000, T=120) in FP64 mode:
    rows of F sampled at random are recomputed from the GPU's pivots as
    F(r,:) = A(r,S) L_S^{-*} with A(S,S) = L_S L_S^* (textbook Cholesky of
    oracle kernel entries); the trace error equals the exact Nystrom error."""
    prob = workloads.mixture20_n1e5(0)
    with rp.Factorizer(prob.X, prob.kernel, prob.sigma, k_max=prob.k, T_max=prob.T) as f:
        f.run(prob.k, prob.T, 0).sync()
        g = f.copy_factor()
        st = f.stats()
    S = g["S"]
    assert g["rank"] == prob.k and len(set(S.tolist())) == prob.k
    ASS = oracle.kernel_matrix(prob.X, prob.kernel, prob.sigma, rows=S, cols=S)
    Ls = np.linalg.cholesky(ASS)
    rng = np.random.default_rng(0)
    rows = np.concatenate([rng.choice(prob.N, 48, replace=False), S[:8]])
    ArS = oracle.kernel_matrix(prob.X, prob.kernel, prob.sigma, rows=rows, cols=S)
    Fr = np.linalg.solve(Ls, ArS.T).T
    err = np.linalg.norm(g["F"][rows] - Fr) / np.linalg.norm(Fr)
    assert err <= 1e-8, err
    # d equals the residual diagonal of the sampled rows
    dres = 1.0 - np.sum(Fr * Fr, axis=1)
    assert np.max(np.abs(g["d"][rows] - np.maximum(dres, 0))) <= 1e-9
    assert st["trace_error"] == pytest.approx(np.sum(g["d"]) / prob.N, rel=1e-6, abs=1e-12)
