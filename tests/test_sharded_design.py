"""The row-sharded form of accelerated RPCholesky (one exchange per round),
checked on CPU ranks (gloo, world size 2) against the single-process oracle.

Each rank owns a contiguous row range of X, F and d.  Per round: the ranks
exchange their totals of d (global offsets of the proposal map); every rank
knows every proposal's uniform, so the owner of each draw resolves it in its
rows; the proposed rows [x | F(s,:) | d_s] are exchanged; every rank forms the
same H and runs Algorithm 1 redundantly (shared random stream); the column
step and the d update are rank-local.  The pivot sequence must equal the
oracle's (the proposal map sums per rank, so in general a divergence is
allowed at a near-tie, as for the GPU; these seeds have none), and the
rank-local rows of F must equal the oracle's factor.  Only host arithmetic runs here: the GPU build is one process
per GPU with replicas (no collective on the data path)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _kappa(oracle, A, B, kernel, sigma):
    Z = np.vstack([A, B]).astype(np.float32)
    na = A.shape[0]
    return oracle.kernel_matrix(Z, kernel, sigma, rows=np.arange(na),
                                cols=np.arange(na, na + B.shape[0]))


def _sum_all(v):
    t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _rank_main(rank, world, port, N, d, kernel, sigma, k, T, seed, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import workloads
    X = workloads.gaussian_cloud(N, d, 7)          # every rank draws the same points,
    lo, hi = rank * N // world, (rank + 1) * N // world
    Xl = X[lo:hi]                                   # and keeps only its rows
    dl = np.ones(hi - lo)
    Fl = np.zeros((hi - lo, k))
    S = []
    rank_now, rnd = 0, 0
    while rank_now < k:
        Wr = np.zeros(world)
        Wr[rank] = np.cumsum(dl)[-1]                # in index order, like the oracle
        Wr = _sum_all(Wr)
        W = float(np.sum(Wr))
        if not W > 0.0:
            break
        offs = np.concatenate([[0.0], np.cumsum(Wr)[:-1]])
        prop = np.zeros(T)
        rows = np.zeros((T, d + k + 1))
        ua = np.zeros(T)
        Cl = np.cumsum(np.concatenate([[offs[rank]], dl]))[1:]
        for j in range(T):
            up, ua[j] = oracle.uniform_pair(seed, j, rnd)
            t = up * W
            owner = int(np.searchsorted(np.cumsum(Wr), t, side="right"))
            owner = min(owner, world - 1)
            while Wr[owner] <= 0.0:                 # rounding past the last weight
                owner -= 1
            if owner == rank:
                hit = np.nonzero((Cl > t) & (dl > 0.0))[0]
                i = int(hit[0]) if len(hit) else int(np.nonzero(dl > 0.0)[0][-1])
                prop[j] = lo + i + 1               # +1 so that the sum of zeros marks "not mine"
                rows[j, :d] = Xl[i]
                rows[j, d:d + k] = Fl[i]
                rows[j, d + k] = dl[i]
        prop = _sum_all(prop).astype(np.int64) - 1
        rows = _sum_all(rows)
        XS, FS, u = rows[:, :d], rows[:, d:d + rank_now], rows[:, d + k]
        H = _kappa(oracle, XS, XS, kernel, sigma) - FS @ FS.T
        acc, L = oracle.reject_chol(H, u, ua, max_accept=k - rank_now)
        n = len(acc)
        if n:
            R = _kappa(oracle, Xl, XS[acc], kernel, sigma) - Fl[:, :rank_now] @ FS[acc].T
            G = np.linalg.solve(L, R.T).T          # G L^* = R
            Fl[:, rank_now:rank_now + n] = G
            dl = np.maximum(dl - np.sum(G * G, axis=1), 0.0)
            S.extend(prop[acc].tolist())
        rank_now += n
        rnd += 1
    out[rank] = (lo, hi, S, Fl[:, :rank_now].copy(), dl.copy(), rnd)
    dist.destroy_process_group()


@pytest.mark.parametrize("kernel,sigma,T", [("gaussian", 3.0, 16), ("matern52", 2.0, 40)])
def test_sharded_rounds_match_the_oracle(kernel, sigma, T):
    import oracle
    import workloads
    world, N, d, k, seed = 2, 900, 6, 120, 11
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), N, d, kernel, sigma, k, T, seed,
                                         out), nprocs=world, start_method="spawn")
    X = workloads.gaussian_cloud(N, d, 7)
    o = oracle.rpc_accel(k, T, seed, X=X, kernel=kernel, sigma=sigma)
    S0 = out[0][2]
    assert all(out[r][2] == S0 for r in range(world))  # every rank holds the same pivots
    assert S0 == o["S"].tolist()
    for r in range(world):
        lo, hi, _, Fl, dl, rounds = out[r]
        assert rounds == o["rounds"]
        assert np.linalg.norm(Fl - o["F"][lo:hi]) <= 1e-10 * np.linalg.norm(o["F"][lo:hi])
        assert np.max(np.abs(dl - o["d"][lo:hi])) <= 1e-12
