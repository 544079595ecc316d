"""Batched launch: many uneven instances in one launch (the persistent
engine, or one CUDA graph) give exactly the results each instance gives alone
(same RNG contract, same block decomposition of every phase), and the
autotuner picks a candidate block size per shape class."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2410_03969_gb300 as rp
    rp.lib()
    return rp


def _instances(count, seed=3):
    probs = workloads.batched_matern(seed, count=count, n_lo=1500, n_hi=9000, k_lo=40,
                                     k_hi=260)
    Ts = [32, 64, 120, 20, 96, 128, 48, 200][:count]
    return probs, Ts


@pytest.mark.parametrize("precision,mode", [("mixed", "engine"), ("mixed", "graph"),
                                            ("fp64", "graph")])
def test_batch_equals_each_instance_alone(rp, precision, mode):
    probs, Ts = _instances(8)
    fs = [rp.Factorizer(p.X, p.kernel, p.sigma, k_max=p.k, T_max=max(Ts), precision=precision,
                        instance=i) for i, p in enumerate(probs)]
    seeds = [1000 + 17 * i for i in range(len(fs))]
    alone = []
    for f, p, T, s in zip(fs, probs, Ts, seeds):
        f.run(p.k, T, s)
        alone.append(f.copy_factor())
    with rp.Batch(fs, Ts) as b:
        assert b.mode == rp.BATCH_GRAPH  # the default executor
        b.mode = rp.BATCH_ENGINE if mode == "engine" else rp.BATCH_GRAPH
        assert b.mode == (rp.BATCH_ENGINE if mode == "engine" else rp.BATCH_GRAPH)
        for rep in range(2):  # the same set-up serves repeated runs
            b.run([p.k for p in probs], seeds)
            for i, f in enumerate(fs):
                got = f.copy_factor()
                assert got["rank"] == alone[i]["rank"] == probs[i].k
                assert np.array_equal(got["S"], alone[i]["S"]), i
                assert np.array_equal(got["F"], alone[i]["F"]), i
                assert np.array_equal(got["d"], alone[i]["d"]), i
                st = f.stats()
                assert st["status"] == 0 and st["rank"] == probs[i].k
    for f in fs:
        f.close()


def test_engine_queue_longer_than_grid(rp):
    """More instances than resident clusters, N from 128 (one tile) to ragged
    multi-tile sizes, ranks from 1 to a few hundred: the queue hands every
    instance out once and each result is the one it gives alone; a second
    run with other k and seeds reuses the set-up."""
    rng = np.random.default_rng(11)
    count = 48
    probs = []
    for i in range(count):
        N = int(rng.choice([128, 129, 300, 1000, 2500, 6000]))
        d = int(rng.choice([1, 3, 8, 20]))
        X = rng.standard_normal((N, d))
        k = int(min(N, rng.choice([1, 7, 40, 130, 300])))
        probs.append((X, ["gaussian", "laplace_l2", "matern32", "matern52"][i % 4], k))
    T = [int(rng.choice([16, 32, 64, 128, 256])) for _ in range(count)]
    fs = [rp.Factorizer(X, kern, 1.0, k_max=k, T_max=256, precision="mixed", instance=i)
          for i, (X, kern, k) in enumerate(probs)]
    with rp.Batch(fs, T) as b:
        b.mode = rp.BATCH_ENGINE
        for rep in range(2):
            ks = [max(1, k - 3 * rep) for (_, _, k) in probs]
            seeds = [77 + 5 * i + 1000 * rep for i in range(count)]
            alone, alone_st = [], []
            for f, k, t, s in zip(fs, ks, T, seeds):
                f.run(k, t, s)
                alone.append(f.copy_factor())
                alone_st.append(f.stats())
            b.run(ks, seeds)
            for i, f in enumerate(fs):
                got = f.copy_factor()
                st = f.stats()
                # a low-dimensional cloud can exhaust the FP32 residual before
                # rank k (every d_i rounds to 0): the run then stops early, in
                # the batch as alone
                assert got["rank"] == alone[i]["rank"] <= ks[i], i
                assert np.array_equal(got["S"], alone[i]["S"]), i
                assert np.array_equal(got["F"], alone[i]["F"]), i
                assert np.array_equal(got["d"], alone[i]["d"]), i
                assert st["status"] == alone_st[i]["status"], i
                assert st["rounds"] == alone_st[i]["rounds"], i
            full = sum(int(alone[i]["rank"] == ks[i]) for i in range(count))
            assert full >= count // 2
    for f in fs:
        f.close()


@pytest.mark.parametrize("case", ["fp64", "l1_laplace", "small_N"])
def test_engine_mode_needs_support(rp, case):
    """The engine runs only the mixed-precision tensor-core path: a batch with
    an FP64 member, an l1-Laplace member (CUDA-core column step) or a member
    below one 128-row tile stays on the graph executor."""
    probs, Ts = _instances(2)
    prec = "fp64" if case == "fp64" else "mixed"
    fs = [rp.Factorizer(p.X, p.kernel, p.sigma, k_max=p.k, T_max=64, precision=prec)
          for p in probs]
    if case == "l1_laplace":
        fs.append(rp.Factorizer(probs[0].X, "laplace_l1", probs[0].sigma, k_max=20, T_max=64,
                                precision="mixed"))
    elif case == "small_N":
        fs.append(rp.Factorizer(probs[0].X[:100], "gaussian", probs[0].sigma, k_max=20,
                                T_max=64, precision="mixed"))
    with rp.Batch(fs, [32] * len(fs)) as b:
        assert b.mode == rp.BATCH_GRAPH
        with pytest.raises(rp.RpcholError):
            b.mode = rp.BATCH_ENGINE
        with pytest.raises(rp.RpcholError):
            b.mode = 7
        b.run([20] * len(fs), list(range(len(fs))))
        for f in fs:
            assert f.stats()["status"] == 0 and f.stats()["rank"] == 20
    for f in fs:
        f.close()


def test_batch_rejects_bad_arguments(rp):
    probs, Ts = _instances(2)
    fs = [rp.Factorizer(p.X, p.kernel, p.sigma, k_max=p.k, T_max=64, precision="mixed")
          for p in probs]
    with pytest.raises(rp.RpcholError):
        rp.Batch(fs, [65, 32])  # T above T_max
    with pytest.raises(rp.RpcholError):
        rp.Batch([fs[0], fs[0]], [32, 32])  # a context twice
    with rp.Batch(fs, [32, 64]) as b:
        with pytest.raises(rp.RpcholError):
            b.run([probs[0].k + 1, probs[1].k], [1, 2])  # k above k_max
    for f in fs:
        f.close()


def test_autotuner_picks_a_candidate_and_caches(rp, tmp_path):
    from paper_2410_03969_gb300 import autotune
    probs, _ = _instances(1)
    p = probs[0]
    tuner = autotune.Autotuner(candidates=(32, 64, 128), repeats=1,
                               cache_path=str(tmp_path / "tune.json"))
    T = tuner.choose(p.X, p.kernel, p.sigma, p.k)
    assert T in (32, 64, 128)
    key = autotune.shape_class(p.N, p.d, p.k, p.kernel)
    assert tuner.timings[key][T] == min(tuner.timings[key].values())
    again = autotune.Autotuner(candidates=(32, 64, 128), cache_path=str(tmp_path / "tune.json"))
    assert again.choose(p.X, p.kernel, p.sigma, p.k) == T


def test_autotuner_picks_the_faster_executor(rp):
    from paper_2410_03969_gb300 import autotune
    probs, Ts = _instances(6)
    fs = [rp.Factorizer(p.X, p.kernel, p.sigma, k_max=p.k, T_max=max(Ts), precision="mixed",
                        instance=i) for i, p in enumerate(probs)]
    ks = [p.k for p in probs]
    seeds = [500 + i for i in range(len(fs))]
    with rp.Batch(fs, Ts[:len(fs)]) as b:
        mode, times = autotune.choose_executor(b, ks, seeds, repeats=1)
        assert set(times) == {rp.BATCH_GRAPH, rp.BATCH_ENGINE}
        assert mode == min(times, key=times.get) and b.mode == mode
        b.run(ks, seeds)
        assert all(f.stats()["status"] == 0 for f in fs)
    for f in fs:
        f.close()
    # FP64 members: the engine is not offered, the graph is kept
    fs = [rp.Factorizer(p.X, p.kernel, p.sigma, k_max=p.k, T_max=64, precision="fp64")
          for p in probs[:2]]
    with rp.Batch(fs, [32, 64]) as b:
        mode, times = autotune.choose_executor(b, [p.k for p in probs[:2]], [1, 2], repeats=1)
        assert mode == rp.BATCH_GRAPH and set(times) == {rp.BATCH_GRAPH}
    for f in fs:
        f.close()
