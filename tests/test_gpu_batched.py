"""Batched launch: many uneven instances in one CUDA graph give exactly the
results each instance gives alone (same RNG contract, same kernels), and the
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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_equals_each_instance_alone(rp, precision):
    probs, Ts = _instances(8)
    fs = [rp.Factorizer(p.X, p.kernel, p.sigma, k_max=p.k, T_max=max(Ts), precision=precision,
                        instance=i) for i, p in enumerate(probs)]
    seeds = [1000 + 17 * i for i in range(len(fs))]
    alone = []
    for f, p, T, s in zip(fs, probs, Ts, seeds):
        f.run(p.k, T, s)
        alone.append(f.copy_factor())
    with rp.Batch(fs, Ts) as b:
        for rep in range(2):  # the recorded graph serves repeated runs
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
