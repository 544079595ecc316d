"""Checkpoints (rpchol_save / rpchol_restore) and continuation
(rpchol_resume): a restored context describes the saved run exactly, a
resumed run continues bit for bit as the original context would, and resuming
at a round boundary reproduces the uninterrupted run (same random stream)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_03969_gb300 as rp
    rp.lib()
    return rp


def same(a, b):
    return (a["rank"] == b["rank"] and np.array_equal(a["S"], b["S"])
            and np.array_equal(a["F"], b["F"]) and np.array_equal(a["d"], b["d"]))


@pytest.mark.parametrize("precision,algo", [("fp64", "accel"), ("mixed", "accel"),
                                            ("mixed", "block"), ("fp64", "plain")])
def test_save_restore_resume_is_exact(rp, precision, algo):
    X = workloads.gaussian_cloud(3000, 8, 50)
    k1, k2, T, seed = 150, 260, 24, 9
    kw = dict(k_max=k2, T_max=T, precision=precision)
    with rp.Factorizer(X, "gaussian", 3.0, **kw) as a, \
            rp.Factorizer(X, "gaussian", 3.0, **kw) as b:
        if algo == "accel":
            a.run(k1, T, seed)
        elif algo == "block":
            a.run_block(k1, T, seed)
        else:
            a.run_plain(k1, seed)
        a.sync()
        blob = a.save()
        ga, sa = a.copy_factor(), a.stats()
        b.restore(blob)
        gb, sb = b.copy_factor(), b.stats()
        assert same(ga, gb)
        assert (sa["rank"], sa["rounds"], sa["proposals"], sa["plain"]) == \
            (sb["rank"], sb["rounds"], sb["proposals"], sb["plain"])
        a.resume(k2).sync()
        b.resume(k2).sync()
        ra, rb = a.copy_factor(), b.copy_factor()
        assert ra["rank"] == k2 and same(ra, rb)
        assert np.array_equal(ra["S"][:k1], ga["S"])


def test_resume_at_a_round_boundary_is_the_uninterrupted_run(rp):
    X = workloads.gaussian_cloud(2500, 6, 51)
    k2, T, seed = 220, 32, 4
    o = oracle.rpc_accel(k2, T, seed, X=X, kernel="matern52", sigma=2.0)
    k1 = int(np.cumsum(o["round_sizes"])[2])  # rank after three full rounds
    with rp.Factorizer(X, "matern52", 2.0, k_max=k2, T_max=T) as f:
        f.run(k2, T, seed).sync()
        full = f.copy_factor()
        f.run(k1, T, seed).sync()
        assert f.stats()["rounds"] == 3
        f.resume(k2).sync()
        res = f.copy_factor()
    assert same(full, res)
    assert np.array_equal(full["S"], o["S"])


def test_checkpoint_errors(rp):
    X = workloads.gaussian_cloud(800, 4, 52)
    with rp.Factorizer(X, "gaussian", 2.0, k_max=60, T_max=16) as a, \
            rp.Factorizer(X, "gaussian", 2.5, k_max=60, T_max=16) as other:
        with pytest.raises(rp.RpcholError):
            a.save()  # nothing to save yet
        a.run(40, 16, 1).sync()
        blob = a.save()
        with pytest.raises(rp.RpcholError):
            other.restore(blob)  # different sigma
        with pytest.raises(rp.RpcholError):
            a.restore(blob[:-8])  # truncated
        with pytest.raises(rp.RpcholError):
            a.resume(40)  # not beyond the current rank
        with pytest.raises(rp.RpcholError):
            a.resume(61)  # beyond k_max
