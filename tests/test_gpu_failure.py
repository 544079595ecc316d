"""Failure detection on the GPU without a fault: the bounded waits of the
column step (CTA scope) and of Algorithm 1 (cluster scope) are made to run
out on a barrier that nothing completes; each must give up after its limit,
report it to the host, and leave the CUDA context usable."""
import ctypes

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


def test_bounded_waits_expire_and_report(rp):
    waited = (ctypes.c_double * 2)()
    rc = rp.lib().rpchol_selftest_wait(100, waited)
    assert rc == 4, rp.lib().rpchol_last_error()  # RPCHOL_ETIMEOUT: both waits gave up
    for w in waited:
        assert 100.0 <= w < 1000.0, list(waited)
    # the context is still usable: a factorisation afterwards matches the oracle
    X = workloads.gaussian_cloud(600, 8, 0)
    with rp.Factorizer(X, "gaussian", 1.0, k_max=48, T_max=16, precision="fp64") as f:
        f.run(48, 16, 3).sync()
        g = f.copy_factor()
    o = oracle.rpc_accel(48, 16, 3, X=X, kernel="gaussian", sigma=1.0)
    assert np.array_equal(g["S"], o["S"])


def test_selftest_rejects_bad_limits(rp):
    assert rp.lib().rpchol_selftest_wait(0, None) == 1
    assert rp.lib().rpchol_selftest_wait(5000, None) == 1
