"""rpchol_trace_error_noalloc: the relative trace error of a factor computed
without any device allocation (its scratch is a static device array), for
callers that cannot allocate device memory, e.g. code inside a runtime that
owns all device memory in its own pool.  It must agree with rpchol_stats,
which computes the same quantity with a context-allocated buffer.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_03969_gb300 as rp
    fn = rp.lib().rpchol_trace_error_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return torch, rp, fn


@pytest.mark.parametrize("N,d,k,T", [(2000, 8, 100, 20), (10000, 5, 150, 40)])
def test_noalloc_trace_error_matches_stats_on_consecutive_calls(env, N, d, k, T):
    torch, rp, fn = env
    X = workloads.gaussian_cloud(N, d, 3)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with rp.Factorizer(X, "gaussian", 1.0, k_max=k, T_max=T, precision="fp64") as f:
        values = []
        for seed in (1, 2):  # two calls in a row, on two different factors
            f.run(k, T, seed).sync()
            Fp, ld, dt, rank, _ = f.factor_view()
            assert rank == k
            rc = fn(Fp, dt, N, ld, rank, out.data_ptr(), stream)
            assert rc == 0, rp.lib().rpchol_last_error()
            torch.cuda.synchronize()
            got = float(out.item())
            want = f.stats()["trace_error"]
            assert got == pytest.approx(want, rel=1e-12, abs=1e-15)
            # a repeated call on the same factor gives the same value
            rc = fn(Fp, dt, N, ld, rank, out.data_ptr(), stream)
            assert rc == 0
            torch.cuda.synchronize()
            assert float(out.item()) == got
            values.append(got)
        assert values[0] != values[1]


@pytest.mark.parametrize("N,d,k,T", [(6000, 6, 200, 40)])
def test_noalloc_fp32_factor_matches_numpy(env, N, d, k, T):
    """The FP32 factor of mixed mode (the float instantiation of the kernel),
    on two calls in a row: the value equals 1 - sum of squares of each row of
    the copied factor, summed in FP64 by numpy (diag A = 1), and rpchol_stats."""
    torch, rp, fn = env
    X = workloads.gaussian_cloud(N, d, 4)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with rp.Factorizer(X, "gaussian", 1.0, k_max=k, T_max=T, precision="mixed") as f:
        values = []
        for seed in (3, 4):
            f.run(k, T, seed).sync()
            Fp, ld, dt, rank, _ = f.factor_view()
            assert rank == k and dt == 0  # RPCHOL_DT_F32
            rc = fn(Fp, dt, N, ld, rank, out.data_ptr(), stream)
            assert rc == 0, rp.lib().rpchol_last_error()
            torch.cuda.synchronize()
            got = float(out.item())
            Fh = np.empty((N, rank), dtype=np.float32)
            f.copy_factor_raw(Fh.ctypes.data, rank)
            rows = 1.0 - np.einsum("ij,ij->i", Fh.astype(np.float64), Fh.astype(np.float64))
            want = float(np.sum(rows)) / N
            # both sides sum the same FP32 entries in FP64, in different orders
            assert got == pytest.approx(want, rel=1e-10, abs=1e-14)
            assert got == pytest.approx(f.stats()["trace_error"], rel=1e-10, abs=1e-14)
            values.append(got)
        assert values[0] != values[1]


def test_noalloc_rejects_sizes_beyond_the_static_scratch(env):
    torch, rp, fn = env
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = fn(buf.data_ptr(), 1, 8388608 + 1, 1, 1, buf.data_ptr(), None)
    assert rc == 1
    assert b"static scratch" in rp.lib().rpchol_last_error()
    rc = fn(buf.data_ptr(), 1, 4, 1, 2, buf.data_ptr(), None)  # ldF < rank
    assert rc == 1
