"""rpchol_run_to_host streams F to caller memory round by round while later
rounds compute; its result is bit-identical to rpchol_run followed by
rpchol_copy_factor_raw, including runs that stop below k, a padded leading
dimension and runs long enough that several rounds' columns go in one
copy, and it leaves entries beyond the final rank unwritten."""
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


def _points(case):
    if case == "rank_deficient":
        # 60 distinct points, each repeated: numerical rank at most 60
        base = workloads.gaussian_cloud(60, 3, 21)
        return np.ascontiguousarray(np.repeat(base, 40, axis=0))
    return workloads.gaussian_cloud(3000, 8, 5)


def _host(shape, np_dtype, fill, pinned):
    if pinned:
        import torch
        t = torch.from_numpy(np.full(shape, fill, np_dtype)).pin_memory()
        return t, t.numpy()
    a = np.full(shape, fill, np_dtype)
    return a, a


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("case,pinned", [("full", True), ("ld_pad", False),
                                         ("rank_deficient", True), ("grouped", True)])
def test_run_to_host_equals_run_then_copy(rp, precision, case, pinned):
    X = _points(case)
    N = X.shape[0]
    k, T, seed = 300, 64, 1234  # k not a multiple of T: the last round stops at k
    if case == "grouped":
        # rank far enough from k that several rounds' columns go in one copy
        k, T = 1500, 100
    ld_out = k + 17 if case == "ld_pad" else k
    dt = np.float32 if precision == "mixed" else np.float64
    with rp.Factorizer(X, "gaussian", 1.0, k_max=k, T_max=T, precision=precision) as f:
        f.run(k, T, seed)
        Fa = np.full((N, ld_out), np.nan, dt)
        Pa = np.zeros(k, np.int64)
        f.copy_factor_raw(Fa.ctypes.data, ld_out, Pa.ctypes.data)
        sa = f.stats()
        keepF, Fb = _host((N, ld_out), dt, np.nan, pinned)
        keepP, Pb = _host((k,), np.int64, -1, pinned)
        f.run_to_host(k, T, seed, Fb.ctypes.data, ld_out, Pb.ctypes.data)
        sb = f.stats()
    r = sa["rank"]
    assert sb["rank"] == r and sb["rounds"] == sa["rounds"] and sb["status"] == sa["status"] == 0
    if case == "rank_deficient":
        assert r < k
    else:
        assert r == k
    assert np.array_equal(Pa[:r], Pb[:r])
    assert np.array_equal(Fa[:, :r], Fb[:, :r])
    assert np.isnan(Fb[:, r:]).all()  # beyond the rank: not written
    assert (Pb[r:] == -1).all()
    assert sb["trace_error"] == sa["trace_error"]
    del keepF, keepP
