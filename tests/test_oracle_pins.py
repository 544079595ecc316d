"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: the
published Philox known-answer vectors, closed-form kernel values, textbook
library routines on special cases, brute-force enumeration of the exact
pivot law on tiny matrices, closed-form expectations and one-sided bounds
from the paper's analysis.  Paper: arXiv 2410.03969.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from conftest import read_golden

# ---------------------------------------------------------------- helpers


def gauss_matrix(N, d, sigma, seed):
    X = np.random.default_rng(seed).standard_normal((N, d)).astype(np.float32)
    return X, oracle.kernel_matrix(X, "gaussian", sigma)


def exact_pivot_law(A, m):
    """P{(s_1..s_m)} for simple RPCholesky by enumeration (Eq. 1.3):
    each pivot is drawn with probability R(j,j)/tr R from the current
    residual R, which is then updated by one Schur-complement step."""
    N = A.shape[0]
    law = {}

    def rec(R, prefix, p):
        if len(prefix) == m:
            law[tuple(prefix)] = law.get(tuple(prefix), 0.0) + p
            return
        dg = np.clip(np.diag(R), 0.0, None)
        tr = dg.sum()
        if tr <= 1e-14 * np.trace(A):
            return
        for j in range(N):
            if dg[j] <= 1e-14 * np.trace(A):
                continue
            Rn = R - np.outer(R[:, j], R[j, :]) / R[j, j]
            rec(Rn, prefix + [j], p * dg[j] / tr)

    rec(np.array(A, dtype=np.float64), [], 1.0)
    return law


def chi2_against_law(samples, law, min_expected=5.0):
    n = len(samples)
    keys = list(law.keys())
    counts = {}
    for s in samples:
        counts[tuple(s)] = counts.get(tuple(s), 0) + 1
    unknown = sum(c for t, c in counts.items() if t not in law)
    assert unknown == 0, "pivot tuples of probability zero were produced"
    obs, exp = [], []
    small_o, small_e = 0.0, 0.0
    for t in keys:
        e = law[t] * n
        o = counts.get(t, 0)
        if e < min_expected:
            small_o += o
            small_e += e
        else:
            obs.append(o)
            exp.append(e)
    if small_e > 0:
        obs.append(small_o)
        exp.append(small_e)
    obs = np.array(obs, dtype=np.float64)
    exp = np.array(exp, dtype=np.float64)
    exp *= obs.sum() / exp.sum()
    return stats.chisquare(obs, exp).pvalue


# ---------------------------------------------------------------- random source


def test_philox_known_answers():
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        ctr = [int(v, 16) for v in r[0:4]]
        key = [int(v, 16) for v in r[4:6]]
        want = [int(v, 16) for v in r[6:10]]
        got = [int(v) for v in oracle.philox4x32_10(ctr, key)]
        assert got == want


def test_u53_closed_forms():
    assert oracle.u53(0, 0) == 0.0
    assert oracle.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.u53(1 << 31, 0) == 0.5
    assert oracle.u53(0, 1 << 6) == 2.0 ** -53
    assert oracle.u53(1 << 5, 0) == 2.0 ** -27


def test_uniform_pair_stream_contract():
    # key = (seed low word, seed high word); counter = (slot, round, 0, instance)
    seed = 0x0123456789ABCDEF
    w = oracle.philox4x32_10([7, 3, 0, 5], [seed & 0xFFFFFFFF, seed >> 32])
    up, ua = oracle.uniform_pair(seed, 7, 3, 5)
    assert up == oracle.u53(int(w[0]), int(w[1]))
    assert ua == oracle.u53(int(w[2]), int(w[3]))


def test_uniforms_are_uniform():
    us = np.array([oracle.uniform_pair(11, j, r)[i] for j in range(100) for r in range(50)
                   for i in range(2)])
    assert stats.kstest(us, "uniform").pvalue > 1e-3


# ---------------------------------------------------------------- kernels


def test_kernel_closed_forms():
    rows = read_golden("kernel_closed_forms.txt")
    assert len(rows) >= 10
    for kernel, sigma, r2, value in rows:
        got = oracle.phi(kernel, float(sigma), float(r2))
        assert got == pytest.approx(float(value), rel=2e-15, abs=0), (kernel, sigma, r2)


def test_kernel_entries_direct_differences():
    X = np.zeros((3, 4), dtype=np.float32)
    X[0, 0] = 3.0
    X[1, 1] = 4.0
    X[2] = X[0]
    # ||x0 - x1|| = 5 (3-4-5 triangle); x2 duplicates x0
    K = oracle.kernel_matrix(X, "gaussian", 5.0)
    assert K[0, 1] == pytest.approx(math.exp(-0.5), rel=1e-15)
    assert K[0, 0] == 1.0 and K[1, 1] == 1.0
    assert K[0, 2] == 1.0
    Kl = oracle.kernel_matrix(X, "laplace_l2", 5.0)
    assert Kl[0, 1] == pytest.approx(math.exp(-1.0), rel=1e-15)
    Km = oracle.kernel_matrix(X, "matern52", 5.0 * math.sqrt(5.0))
    assert Km[1, 0] == pytest.approx(7.0 / (3.0 * math.e), rel=1e-15)
    Km3 = oracle.kernel_matrix(X, "matern32", 5.0 * math.sqrt(3.0))
    assert Km3[1, 0] == pytest.approx(2.0 / math.e, rel=1e-15)
    # l1 distance |3 - 0| + |0 - 4| = 7
    K1 = oracle.kernel_matrix(X, "laplace_l1", 7.0)
    assert K1[0, 1] == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert K1[0, 2] == 1.0
    # the l1-Laplace is the product of one-dimensional Laplace kernels
    Y = np.random.default_rng(3).standard_normal((6, 4)).astype(np.float32)
    K1 = oracle.kernel_matrix(Y, "laplace_l1", 1.7)
    prod = np.ones((6, 6))
    for l in range(4):
        prod *= np.exp(-np.abs(Y[:, None, l].astype(np.float64) - Y[None, :, l]) / 1.7)
    assert np.allclose(K1, prod, rtol=1e-13, atol=0)


def test_kernel_matrices_are_psd():
    X = np.random.default_rng(0).standard_normal((40, 3)).astype(np.float32)
    for kern in ("gaussian", "laplace_l2", "matern52", "matern32", "laplace_l1"):
        K = oracle.kernel_matrix(X, kern, 1.3)
        assert np.allclose(K, K.T)
        assert np.linalg.eigvalsh(K).min() > -1e-12


# ---------------------------------------------------------------- proposal map


def test_sample_matches_searchsorted():
    rng = np.random.default_rng(1)
    for _ in range(200):
        n = int(rng.integers(1, 50))
        w = rng.random(n) * (rng.random(n) < 0.7)
        if w.sum() == 0:
            w[0] = 1.0
        U = float(rng.random())
        W = float(np.sum(w))
        want = int(np.searchsorted(np.cumsum(w), U * W, side="right"))
        got = oracle.sample(w, U)
        if want < n:
            assert got == want
            assert w[got] > 0
        else:  # rounding left none: largest positive weight
            assert got == int(np.nonzero(w)[0].max())


def test_sample_edges():
    w = np.array([0.0, 0.0, 2.0, 0.0, 1.0, 0.0])
    assert oracle.sample(w, 0.0) == 2
    assert oracle.sample(w, 1.0 - 2.0 ** -53) == 4
    assert oracle.sample(w, 2.0 / 3.0 - 1e-12) == 2
    assert oracle.sample(w, 2.0 / 3.0 + 1e-12) == 4


def test_sample_frequencies():
    w = np.array([0.5, 0.0, 2.0, 1.0, 0.25])
    counts = np.zeros(len(w))
    for j in range(20000):
        counts[oracle.sample(w, oracle.uniform_pair(5, j % 1000, j // 1000)[0])] += 1
    assert counts[1] == 0
    p = w[w > 0] / w.sum()
    assert stats.chisquare(counts[w > 0], p * counts.sum()).pvalue > 1e-3


# ---------------------------------------------------------------- Algorithm 1


def test_reject_chol_all_accept_is_cholesky():
    _, A = gauss_matrix(12, 3, 2.0, 3)
    acc, L = oracle.reject_chol(A, np.diag(A), np.zeros(12))
    assert list(acc) == list(range(12))
    assert np.allclose(L, np.linalg.cholesky(A), rtol=0, atol=1e-12)


def test_reject_chol_rejects_duplicates_and_follows_rule():
    X = np.random.default_rng(4).standard_normal((5, 2)).astype(np.float32)
    idx = [0, 1, 0, 2, 1]
    A = oracle.kernel_matrix(X, "gaussian", 1.0, rows=idx, cols=idx)
    acc, L = oracle.reject_chol(A, np.diag(A), np.full(5, 0.0))
    # duplicates of accepted points have zero residual and are rejected
    assert list(acc) == [0, 1, 3]
    sub = A[np.ix_(acc, acc)]
    assert np.allclose(L @ L.T, sub, atol=1e-14)
    assert np.allclose(np.triu(L, 1), 0.0)


def test_reject_chol_acceptance_threshold():
    a, b, c = 1.0, 0.8, 0.6
    H = np.array([[a, c], [c, b]])
    thresh = (b - c * c / a) / b  # residual / proposal weight (Sec. 2.1 box)
    for eps, accept in ((-1e-9, True), (1e-9, False)):
        acc, _ = oracle.reject_chol(H, np.array([a, b]), np.array([0.3, thresh + eps]))
        assert (1 in acc) == accept
    # max_accept stops Algorithm 1 early
    acc, L = oracle.reject_chol(H, np.array([a, b]), np.zeros(2), max_accept=1)
    assert list(acc) == [0] and L.shape == (1, 1)


# ---------------------------------------------------------------- Algorithms 2 and 6


@pytest.mark.parametrize("algo", ["plain", "accel"])
def test_full_reconstruction_at_k_equals_N(algo):
    X, A = gauss_matrix(10, 3, 0.6, 5)
    assert np.linalg.cond(A) < 1e6
    if algo == "plain":
        out = oracle.rpc_plain(10, 17, A=A)
    else:
        out = oracle.rpc_accel(10, 4, 17, A=A)
    F = out["F"]
    assert out["rank"] == 10
    assert np.linalg.norm(A - F @ F.T) / np.linalg.norm(A) <= 1e-12
    assert sorted(out["S"]) == list(range(10))


@pytest.mark.parametrize("algo,T", [("plain", 1), ("accel", 1), ("accel", 3), ("accel", 8)])
def test_nystrom_identity_and_invariants(algo, T):
    X = np.random.default_rng(6).standard_normal((60, 4)).astype(np.float32)
    A = oracle.kernel_matrix(X, "matern52", 2.0)
    k = 25
    out = (oracle.rpc_plain(k, 99, X=X, kernel="matern52", sigma=2.0) if algo == "plain"
           else oracle.rpc_accel(k, T, 99, X=X, kernel="matern52", sigma=2.0))
    F, S = out["F"], out["S"]
    assert out["rank"] == k and len(set(S.tolist())) == k
    # Nystrom identity: F F^* = A(:,S) A(S,S)^{-1} A(S,:) (Sec. 2.1)
    C = A[:, S]
    nys = C @ np.linalg.solve(A[np.ix_(S, S)], C.T)
    assert np.linalg.norm(F @ F.T - nys) / np.linalg.norm(nys) <= 1e-10
    # residual diagonal equals d; residual psd; F(S,:) lower triangular in pivot order
    R = A - F @ F.T
    assert np.max(np.abs(np.diag(R) - out["d"])) <= 1e-12
    assert np.linalg.eigvalsh(R).min() >= -1e-12 * np.trace(A)
    FS = F[S, :]
    assert np.max(np.abs(np.triu(FS, 1))) <= 1e-12
    assert np.all(np.diag(FS) > 0)
    # the oracle's fixed-pivot re-evaluation gives the same factor
    F2, d2, te = oracle.fixed_pivot_factor(S, A=A)
    assert np.max(np.abs(F2 - F)) <= 1e-12
    assert te == pytest.approx(np.trace(R), rel=1e-9, abs=1e-13)


def test_residual_diagonal_nonincreasing_and_prefix():
    X = np.random.default_rng(7).standard_normal((80, 3)).astype(np.float32)
    outs = [oracle.rpc_accel(k, 6, 5, X=X, kernel="gaussian", sigma=1.5) for k in (5, 12, 30)]
    for a, b in zip(outs, outs[1:]):
        assert np.all(b["d"] <= a["d"] + 1e-15)
        assert list(b["S"][:a["rank"]]) == list(a["S"])  # stopping at k truncates, not reorders
        assert np.max(np.abs(b["F"][:, :a["rank"]] - a["F"])) <= 1e-13


def test_rank_bounds_and_first_proposal_accepted():
    X = np.random.default_rng(8).standard_normal((200, 2)).astype(np.float32)
    T, t = 16, 6
    out = oracle.rpc_accel(200, T, 3, X=X, kernel="gaussian", sigma=0.7, max_rounds=t)
    assert out["rounds"] == t
    assert t <= out["rank"] <= T * t
    assert np.all(out["round_sizes"] >= 1) and np.all(out["round_sizes"] <= T)
    # Algorithm 1's literal acceptance denominator agrees on the first round
    a = oracle.rpc_accel(200, T, 3, X=X, kernel="gaussian", sigma=0.7, max_rounds=1)
    b = oracle.rpc_accel(200, T, 3, X=X, kernel="gaussian", sigma=0.7, max_rounds=1,
                         accept_rule=1)
    assert list(a["S"]) == list(b["S"])


def test_block_size_one_equals_simple_rpcholesky():
    X = np.random.default_rng(9).standard_normal((300, 5)).astype(np.float32)
    for seed in range(5):
        p = oracle.rpc_plain(40, seed, X=X, kernel="laplace_l2", sigma=2.0)
        a = oracle.rpc_accel(40, 1, seed, X=X, kernel="laplace_l2", sigma=2.0)
        assert list(p["S"]) == list(a["S"])
        assert np.max(np.abs(p["F"] - a["F"])) <= 1e-13


# ---------------------------------------------------------------- Algorithm 7


def _draws_by_searchsorted(d, seed, b, rnd):
    """The b proposals of one round, by numpy's searchsorted on the cumulative
    weights (an independent restatement of the proposal map)."""
    C = np.cumsum(d)
    out = []
    for j in range(b):
        up, _ = oracle.uniform_pair(seed, j, rnd)
        out.append(int(np.searchsorted(C, up * C[-1], side="right")))
    return out


def test_block_rpc_block_one_equals_simple_rpcholesky():
    X = np.random.default_rng(19).standard_normal((300, 5)).astype(np.float32)
    for seed in range(5):
        p = oracle.rpc_plain(40, seed, X=X, kernel="gaussian", sigma=1.5)
        b = oracle.rpc_block(40, 1, seed, X=X, kernel="gaussian", sigma=1.5)
        assert list(p["S"]) == list(b["S"])
        assert np.max(np.abs(p["F"] - b["F"])) <= 1e-13
        assert np.max(np.abs(p["d"] - b["d"])) <= 1e-13


@pytest.mark.parametrize("b", [3, 8, 20])
def test_block_rpc_nystrom_identity_and_unique(b):
    X = np.random.default_rng(20).standard_normal((70, 3)).astype(np.float32)
    A = oracle.kernel_matrix(X, "laplace_l2", 1.5)
    k, seed = 30, 4
    out = oracle.rpc_block(k, b, seed, X=X, kernel="laplace_l2", sigma=1.5)
    F, S = out["F"], out["S"]
    assert out["rank"] == k and len(set(S.tolist())) == k
    # Nystrom identity: F F^* = A(:,S) A(S,S)^{-1} A(S,:) (Sec. 2.1)
    C = A[:, S]
    nys = C @ np.linalg.solve(A[np.ix_(S, S)], C.T)
    assert np.linalg.norm(F @ F.T - nys) / np.linalg.norm(nys) <= 1e-10
    R = A - F @ F.T
    assert np.max(np.abs(np.diag(R) - out["d"])) <= 1e-12
    # round by round: the accepted pivots are the distinct draws in draw order
    # (all residuals positive on this well-conditioned matrix), cut at rank k
    d = np.ones(70)
    pos = 0
    for rnd, n in enumerate(out["round_sizes"]):
        draws = _draws_by_searchsorted(d, seed, b, rnd)
        uniq = list(dict.fromkeys(draws))[:k - pos]
        assert list(S[pos:pos + n]) == uniq
        pos += n
        Fp = F[:, :pos]
        d = np.maximum(1.0 - np.sum(Fp * Fp, axis=1), 0.0)


def test_block_rpc_exact_rank_and_semidefinite_chol():
    # rank-4 psd matrix: one round of 6 draws reaches rank 4 (any 4 distinct
    # rows of a generic B are independent) and the factor reproduces A
    B = np.random.default_rng(21).standard_normal((40, 4))
    A = B @ B.T
    out = oracle.rpc_block(4, 6, 2, A=A)
    assert out["rank"] == 4 and out["rounds"] == 1
    F = out["F"]
    assert np.linalg.norm(A - F @ F.T) / np.linalg.norm(A) <= 1e-10
    # a diagonal matrix: duplicates and zero-weight rows are never pivots
    D = np.diag([4.0, 0.0, 1.0, 0.0, 2.0])
    o = oracle.rpc_block(5, 8, 1, A=D)
    assert sorted(o["S"]) == [0, 2, 4]
    assert np.allclose(o["F"] @ o["F"].T, D, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- Algorithm 3


@pytest.mark.parametrize("T", [1, 6, 16])
def test_lowmem_meets_algorithm_2(T):
    # Algorithm 3 draws the same pivots as Algorithm 2 and keeps L = F(S,:),
    # the Cholesky factor of A(S,S) (Sec. 2.4)
    X = np.random.default_rng(22).standard_normal((90, 3)).astype(np.float32)
    A = oracle.kernel_matrix(X, "matern52", 1.5)
    k, seed = 40, 8
    lo = oracle.rpc_lowmem(k, T, seed, X=X, kernel="matern52", sigma=1.5)
    ac = oracle.rpc_accel(k, T, seed, X=X, kernel="matern52", sigma=1.5)
    assert lo["rank"] == ac["rank"] == k and lo["rounds"] == ac["rounds"]
    assert list(lo["S"]) == list(ac["S"])
    L, S = lo["L"], lo["S"]
    assert np.max(np.abs(np.triu(L, 1))) == 0.0 and np.all(np.diag(L) > 0)
    assert np.max(np.abs(L @ L.T - A[np.ix_(S, S)])) <= 1e-12
    assert np.max(np.abs(L - ac["F"][S, :])) <= 1e-12
    # the implicit approximation A(:,S) L^{-*} L^{-1} A(S,:) and its diagonal
    Z = np.linalg.solve(L, A[S, :])
    assert np.max(np.abs(np.diag(A) - np.sum(Z * Z, axis=0) - lo["d"])) <= 1e-12
    assert np.max(np.abs(lo["d"] - ac["d"])) <= 1e-12


def test_lowmem_exhaustion_and_k_equals_N():
    X, A = gauss_matrix(12, 3, 0.6, 23)
    lo = oracle.rpc_lowmem(12, 5, 3, A=A)
    assert lo["rank"] == 12 and sorted(lo["S"]) == list(range(12))
    S = lo["S"]
    assert np.linalg.norm(lo["L"] @ lo["L"].T - A[np.ix_(S, S)]) <= 1e-12 * np.linalg.norm(A)
    D = np.diag([4.0, 0.0, 1.0, 0.0, 0.0])
    lo = oracle.rpc_lowmem(4, 3, 1, A=D)
    assert lo["rank"] == 2 and sorted(lo["S"]) == [0, 2]


# ---------------------------------------------------------------- Algorithm 5


@pytest.mark.parametrize("T", [1, 5, 12])
def test_rpqr_meets_rpcholesky_on_the_gram_matrix(T):
    # QR-Cholesky correspondence (appendix proposition): with the same pivots,
    # RPQR of B gives the Cholesky factor of A = B^* B; the same random stream
    # then draws the same pivots
    rng = np.random.default_rng(24)
    M, N = 40, 70
    B = rng.standard_normal((M, 6)) @ rng.standard_normal((6, N)) + 0.05 * rng.standard_normal((M, N))
    A = B.T @ B
    k, seed = 25, 5
    qr = oracle.rpqr_accel(B, k, T, seed)
    ch = oracle.rpc_accel(k, T, seed, A=A)
    assert qr["rank"] == ch["rank"] == k and list(qr["S"]) == list(ch["S"])
    assert np.linalg.norm(qr["F"] - ch["F"]) <= 1e-10 * np.linalg.norm(ch["F"])
    assert np.max(np.abs(qr["u"] - ch["d"])) <= 1e-10 * np.max(np.diag(A))
    # Q orthonormal, F = B^* Q, u = squared column norms of (I - QQ^*) B
    Q = qr["Q"]
    assert np.max(np.abs(Q.T @ Q - np.eye(k))) <= 1e-12
    assert np.max(np.abs(qr["F"] - B.T @ Q)) <= 1e-12 * np.max(np.abs(B))
    R = B - Q @ (Q.T @ B)
    assert np.max(np.abs(np.sum(R * R, axis=0) - qr["u"])) <= 1e-10 * np.max(np.diag(A))
    # the pivot columns are reproduced exactly
    S = qr["S"]
    assert np.max(np.abs(R[:, S])) <= 1e-10 * np.max(np.abs(B))


def _rpqr_algorithm4_numpy(B, k, seed):
    """Algorithm 4 (randomly pivoted QR, one pivot per step) restated with
    numpy: draw s from u / sum(u) (searchsorted on the cumulative sums, the
    same Philox uniforms), q = normalised residual column, F(:,i) = B^* q,
    u -= F(:,i)^2 clamped at 0."""
    M, N = B.shape
    u = np.sum(B * B, axis=0)
    Q = np.zeros((M, k))
    F = np.zeros((N, k))
    S = []
    for i in range(k):
        up, _ = oracle.uniform_pair(seed, 0, i)
        C = np.cumsum(u)
        s = int(np.searchsorted(C, up * C[-1], side="right"))
        g = B[:, s] - Q[:, :i] @ F[s, :i]
        q = g / np.linalg.norm(g)
        Q[:, i] = q
        F[:, i] = B.T @ q
        u = np.maximum(u - F[:, i] ** 2, 0.0)
        S.append(s)
    return Q, F, S, u


def test_rpqr_block_one_is_algorithm_4():
    rng = np.random.default_rng(26)
    B = rng.standard_normal((30, 5)) @ rng.standard_normal((5, 50)) + 0.1 * rng.standard_normal((30, 50))
    k, seed = 20, 3
    qr = oracle.rpqr_accel(B, k, 1, seed)
    Q, F, S, u = _rpqr_algorithm4_numpy(B, k, seed)
    assert list(qr["S"]) == S
    assert np.max(np.abs(qr["F"] - F)) <= 1e-10 * np.max(np.abs(F))
    assert np.max(np.abs(qr["Q"] - Q)) <= 1e-10
    assert np.max(np.abs(qr["u"] - u)) <= 1e-10 * np.max(np.sum(B * B, axis=0))


def test_lowmem_block_one_is_simple_rpcholesky():
    X = np.random.default_rng(27).standard_normal((200, 4)).astype(np.float32)
    lo = oracle.rpc_lowmem(30, 1, 6, X=X, kernel="laplace_l2", sigma=1.5)
    pl = oracle.rpc_plain(30, 6, X=X, kernel="laplace_l2", sigma=1.5)
    assert list(lo["S"]) == list(pl["S"])
    assert np.max(np.abs(lo["L"] - pl["F"][pl["S"], :])) <= 1e-12
    assert np.max(np.abs(lo["d"] - pl["d"])) <= 1e-12


def test_rpqr_full_rank_exhaustion():
    B = np.random.default_rng(25).standard_normal((5, 9))
    qr = oracle.rpqr_accel(B, 5, 4, 1)
    assert qr["rank"] == 5
    assert np.linalg.norm(qr["Q"] @ qr["F"].T - B) <= 1e-12 * np.linalg.norm(B)


def test_zero_weight_stop_returns_lower_rank():
    # Exact exhaustion (Sec. 2.1, sum u = 0): a diagonal matrix whose pivots
    # eliminate exactly in FP64 leaves a zero residual after two pivots.
    A = np.diag([4.0, 0.0, 1.0, 0.0, 0.0])
    for out in (oracle.rpc_plain(4, 1, A=A), oracle.rpc_accel(4, 3, 1, A=A)):
        assert out["rank"] == 2
        assert sorted(out["S"]) == [0, 2]
        assert np.array_equal(out["F"] @ out["F"].T, A)
    # Numerically rank-deficient input: after rank(A) pivots the residual is
    # at rounding level and the reconstruction is exact to rounding.
    V = np.random.default_rng(10).standard_normal((7, 2))
    A = V @ V.T
    for out in (oracle.rpc_plain(5, 1, A=A), oracle.rpc_accel(5, 3, 1, A=A)):
        F = out["F"]
        assert np.linalg.norm(A - F[:, :2] @ F[:, :2].T) <= 1e-12 * np.linalg.norm(A)
        assert np.abs(out["d"]).max() <= 1e-12 * np.trace(A)


# ---------------------------------------------------------------- pivot law


LAW_CASES = {
    "gauss": gauss_matrix(6, 2, 0.8, 11)[1],
    "diag": np.diag([3.0, 1.0, 0.5, 0.25, 2.0, 0.05]),
    "lowrank": (lambda V: V @ V.T)(np.random.default_rng(12).standard_normal((6, 3))),
}


@pytest.mark.parametrize("case", list(LAW_CASES))
@pytest.mark.parametrize("algo,T", [("plain", 1), ("accel", 1), ("accel", 2), ("accel", 3),
                                    ("accel", 5), ("accel", 12)])
def test_pivot_law_chi_squared(case, algo, T):
    """Pivot tuples of simple and accelerated RPCholesky follow the exact law
    P = prod A^{(i)}(s,s) / tr A^{(i)} (Eq. 1.3; Sec. 2.2, last paragraph)."""
    A = LAW_CASES[case]
    m = 3
    law = exact_pivot_law(A, m)
    assert abs(sum(law.values()) - 1.0) < 1e-12
    S, ranks = oracle.pivots_many(algo, m, 40000, 1234 + T, T=T, A=A)
    assert np.all(ranks == m)
    assert chi2_against_law(S, law) > 1e-4


def test_one_step_expected_residual():
    """E[A^{(1)}] = A - A^2 / tr A (Sec. 3.2, expected residual function)."""
    _, A = gauss_matrix(6, 2, 1.0, 13)
    n = 6000
    acc = np.zeros_like(A)
    acc2 = np.zeros_like(A)
    for i in range(n):
        F = oracle.rpc_plain(1, 77, A=A, inst=i)["F"]
        R = A - F @ F.T
        acc += R
        acc2 += R * R
    mean = acc / n
    sd = np.sqrt(np.maximum(acc2 / n - mean * mean, 1e-30))
    want = A - A @ A / np.trace(A)
    z = np.abs(mean - want) / (sd / math.sqrt(n))
    assert z.max() < 5.0


def _Phi_b_trace(lam, b, t):
    """tr Phi_b^{(t)}(A) on the eigenvalues (Lemma "central error bound"):
    phi_alpha(x) = x - x^2/alpha applied b times with alpha = tr of the input
    of Phi_b, then Phi_b itself composed t times."""
    lam = np.array(lam, dtype=np.float64)
    for _ in range(t):
        alpha = lam.sum()
        for _ in range(b):
            lam = lam - lam * lam / alpha
    return lam.sum()


@pytest.mark.parametrize("b,t", [(1, 3), (3, 2), (6, 2)])
def test_central_error_bound(b, t):
    X, A = gauss_matrix(8, 2, 1.2, 14)
    tr = oracle.accel_trace_many(A, b, t, 4000, 4242)
    bound = _Phi_b_trace(np.linalg.eigvalsh(A), b, t)
    se = tr.std() / math.sqrt(len(tr))
    assert tr.mean() <= bound + 3 * se
    if b == 1 and t == 1:
        assert abs(tr.mean() - bound) < 5 * se


def test_one_round_b1_meets_bound_with_equality():
    _, A = gauss_matrix(8, 2, 1.2, 15)
    tr = oracle.accel_trace_many(A, 1, 1, 6000, 99)
    bound = _Phi_b_trace(np.linalg.eigvalsh(A), 1, 1)
    assert abs(tr.mean() - bound) < 5 * tr.std() / math.sqrt(len(tr))


def test_points_and_matrix_paths_agree():
    X = np.random.default_rng(16).standard_normal((50, 3)).astype(np.float32)
    A = oracle.kernel_matrix(X, "gaussian", 1.0)
    a = oracle.rpc_accel(20, 5, 8, X=X, kernel="gaussian", sigma=1.0)
    b = oracle.rpc_accel(20, 5, 8, A=A)
    assert list(a["S"]) == list(b["S"])
    assert np.array_equal(a["F"], b["F"])


@pytest.mark.parametrize("algo", ["accel", "block", "plain", "lowmem"])
def test_rank_deficient_kernel_stops_at_its_numerical_rank(algo):
    """The residual floor: 1-D points under a Gaussian kernel give a kernel matrix
    of numerical rank about 20.  Every run must stop there with all weights
    at zero, long before the round limit, with the residual below the floor
    and every accepted pivot's column well scaled (no pivot taken on
    rounding noise)."""
    X = np.random.default_rng(11).standard_normal((300, 1)).astype(np.float32)
    A = oracle.kernel_matrix(X, "gaussian", 1.0)
    ev = np.linalg.eigvalsh(A)
    numrank = int(np.sum(ev > 1e-13 * ev[-1]))
    k = 130
    if algo == "accel":
        o = oracle.rpc_accel(k, 16, 77, X=X, kernel="gaussian", sigma=1.0, max_rounds=4 * k + 64)
    elif algo == "block":
        o = oracle.rpc_block(k, 16, 77, X=X, kernel="gaussian", sigma=1.0, max_rounds=4 * k + 64)
    elif algo == "plain":
        o = oracle.rpc_plain(k, 77, X=X, kernel="gaussian", sigma=1.0)
    else:
        o = oracle.rpc_lowmem(k, 16, 77, X=X, kernel="gaussian", sigma=1.0,
                              max_rounds=4 * k + 64)
    assert 5 <= o["rank"] <= numrank + 2
    assert float(np.sum(o["d"])) == 0.0
    if "rounds" in o and algo != "plain":
        assert o["rounds"] < 4 * o["rank"] + 10
    # the factor reproduces A to the level of the floor on every entry
    if "F" in o:
        F = o["F"]
        assert np.max(np.abs(A - F @ F.T)) < 1e-6
