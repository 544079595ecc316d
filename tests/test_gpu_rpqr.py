"""Accelerated randomly pivoted QR (Algorithm 5) on the GPU against the FP64
oracle: identical pivots (same random stream; a divergence is allowed only at
a near-tie of the proposal map), Q and F to 1e-9 relative Frobenius error,
u to 1e-10 of the largest squared column norm, Q orthonormal to 1e-12.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_03969_gb300 as rp
    rp.lib()
    return rp


def make_B(M, N, r, noise, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((M, r)) @ rng.standard_normal((r, N))
    B *= np.exp(rng.standard_normal(N))  # uneven column norms
    return B + noise * rng.standard_normal((M, N))


def near_tie(B, k, T, seed, S_gpu, S_orc):
    p = next(i for i in range(min(len(S_gpu), len(S_orc))) if S_gpu[i] != S_orc[i])
    # replay rounds until the one holding position p
    rnd, u = 0, np.sum(B * B, axis=0)
    while True:
        o = oracle.rpqr_accel(B, k, T, seed, max_rounds=rnd + 1)
        if o["rank"] > p or o["rounds"] <= rnd:
            break
        u = o["u"]
        rnd += 1
    C = np.cumsum(u)
    W = float(np.sum(u))
    return any(np.min(np.abs(C - oracle.uniform_pair(seed, j, rnd)[0] * W)) <= 1e-12 * W
               for j in range(T))


CASES = [
    # M, N, latent rank, noise, k, T, seed
    (200, 500, 20, 0.05, 60, 16, 0),
    (64, 1000, 64, 0.0, 64, 32, 1),      # k = M: the factorisation is exact
    (300, 257, 40, 0.01, 100, 1, 2),     # T = 1: randomly pivoted QR (Algorithm 4)
    (1000, 2000, 400, 0.01, 300, 128, 3),
]


@pytest.mark.parametrize("M,N,r,noise,k,T,seed", CASES)
def test_rpqr_matches_oracle(rp, M, N, r, noise, k, T, seed):
    B = make_B(M, N, r, noise, seed)
    with rp.RPQR(B, k_max=k, T_max=T) as f:
        g = f.run(k, T, seed).copy()
    o = oracle.rpqr_accel(B, k, T, seed)
    assert np.max(np.abs(g["Q"].T @ g["Q"] - np.eye(g["rank"]))) <= 1e-12
    if g["rank"] != o["rank"] or not np.array_equal(g["S"], o["S"]):
        assert near_tie(B, k, T, seed, g["S"], o["S"]), "pivot divergence outside the margin"
        print("pivot sequences diverge at a near-tie of the proposal map")
        return
    assert g["rounds"] == o["rounds"]
    for key in ("Q", "F"):
        err = np.linalg.norm(g[key] - o[key]) / np.linalg.norm(o[key])
        assert err <= 1e-9, (key, err)
    u0 = np.max(np.sum(B * B, axis=0))
    assert np.max(np.abs(g["u"] - o["u"])) <= 1e-10 * u0
    if k == M:
        assert np.linalg.norm(g["Q"] @ g["F"].T - B) <= 1e-10 * np.linalg.norm(B)


def test_rpqr_full_size_properties(rp):
    """The benchmarked case (dense 2000 x 20000, numerical rank about 400, k =
    500, T = 128), checked through properties that hold at any size: Q has
    orthonormal columns, sampled rows of F equal B^* Q, sampled u equal the
    squared column norms of B - Q Q^* B, the pivots are distinct, and the
    pivot columns are reproduced."""
    rng = np.random.default_rng(5)
    M, N, k, T = 2000, 20000, 500, 128
    B = rng.standard_normal((M, 400)) @ rng.standard_normal((400, N)) \
        + 0.01 * rng.standard_normal((M, N))
    with rp.RPQR(B, k_max=k, T_max=T) as f:
        g = f.run(k, T, 1).copy()
    Q, F, S, u = g["Q"], g["F"], g["S"], g["u"]
    assert g["rank"] == k and len(set(S.tolist())) == k
    assert np.max(np.abs(Q.T @ Q - np.eye(k))) <= 1e-11
    cols = np.concatenate([rng.choice(N, 64, replace=False), S[:4], S[-4:]])
    Fx = B[:, cols].T @ Q
    assert np.max(np.abs(F[cols] - Fx)) <= 1e-10 * np.max(np.abs(Fx))
    R = B[:, cols] - Q @ Fx.T
    ux = np.sum(R * R, axis=0)
    scale = np.max(np.sum(B[:, cols] ** 2, axis=0))
    assert np.max(np.abs(u[cols] - np.maximum(ux, 0.0))) <= 1e-9 * scale
    assert np.max(np.abs(R[:, -8:])) <= 1e-9 * np.sqrt(scale)
