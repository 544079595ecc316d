"""Where a GPU FP64 pivot sequence may leave the oracle's (test helper).

Both sides draw from the same Philox stream (counter (slot, round, 0,
instance)), so in FP64 their pivot sequences are identical unless a decision
of the method is a near-tie that rounding can flip:

  * a proposal (the sampler of Algorithm 2's step 1, reading c3): the scaled
    uniform U W lies within 1e-12 W of the prefix sum C_j bounding the chosen
    index j, or of C_{j-1};
  * an acceptance (Algorithm 1's test u_i U_i < h_ii, readings c4 and c5):
    |U_i u_i - h_ii| <= 1e-12 u_i.

`accel_divergence` finds the first differing pivot p, replays the oracle to
the START of the round that holds p (from the oracle's own round sizes, so
that no partial round is applied), recomputes that round's proposals from the
oracle's d, forms H = A(S',S') - F(S',:) F(S',:)^* from the oracle's F and
walks Algorithm 1 in numpy, recording each slot's proposal and acceptance
margins.  The divergence is allowed only if a near-tie lies in the window of
slots that decides accepted position q of that round (after the oracle's
(q-1)-th accepted slot, up to and including its q-th), and the GPU's pivot at
p is one of the indices that round could then accept.  The numpy walk only
locates margins: its accepted slots must reproduce the oracle's pivots before
and at the divergence, or the helper itself fails.
"""
from __future__ import annotations

import numpy as np

import oracle

TIE = 1e-12


def first_divergence(S_gpu, S_orc):
    """Index of the first differing pivot, len(shorter) if one sequence is a
    strict prefix of the other, None if identical."""
    n = min(len(S_gpu), len(S_orc))
    for i in range(n):
        if int(S_gpu[i]) != int(S_orc[i]):
            return i
    return None if len(S_gpu) == len(S_orc) else n


def _proposal(d, up):
    """(index, near_tie, neighbours) of the proposal map on weights d for the
    uniform up: j* = min{j : C_j > U W} (else the last positive weight)."""
    C = np.cumsum(d)  # inclusive prefix in index order (reading c3)
    W = float(C[-1])  # the total in index order, as the oracle sums it
    t = up * W
    j = int(np.searchsorted(C, t, side="right"))
    if j >= len(d):
        j = int(np.nonzero(d > 0)[0][-1])
    near = abs(C[j] - t) <= TIE * W or (j > 0 and abs(C[j - 1] - t) <= TIE * W)
    pos = np.nonzero(d > 0)[0]
    k = int(np.searchsorted(pos, j))
    nb = {int(pos[i]) for i in (k - 1, k + 1) if 0 <= i < len(pos)}
    return j, near, nb


def accel_divergence(X, kernel, sigma, k, T, seed, S_gpu, S_orc, inst=0):
    """None if the sequences are identical; otherwise a dict describing the
    divergence: round, accepted position q, rank at the round start, the slot
    window, whether a near-tie lies in it ('allowed') and its kind."""
    p = first_divergence(S_gpu, S_orc)
    if p is None:
        return None
    full = oracle.rpc_accel(k, T, seed, X=X, kernel=kernel, sigma=sigma, inst=inst)
    sizes = np.asarray(full["round_sizes"], dtype=np.int64)
    cum = np.cumsum(sizes)
    rnd = int(np.searchsorted(cum, p, side="right"))
    rank0 = int(cum[rnd - 1]) if rnd > 0 else 0
    q = p - rank0
    N = X.shape[0]
    if rnd > 0:
        start = oracle.rpc_accel(k, T, seed, X=X, kernel=kernel, sigma=sigma, inst=inst,
                                 max_rounds=rnd)
        assert start["rank"] == rank0
        d, F = start["d"], start["F"]
    else:
        d, F = np.ones(N), np.zeros((N, 0))
    props, uacc, ptie, nbs = [], [], [], []
    for j in range(T):
        up, ua = oracle.uniform_pair(seed, j, rnd, inst)
        s, near, nb = _proposal(d, up)
        s = oracle.sample(d, up)  # the oracle's own pick (margins from numpy)
        props.append(s)
        uacc.append(ua)
        ptie.append(near)
        nbs.append(nb)
    props = np.asarray(props, dtype=np.int64)
    A = oracle.kernel_matrix(X, kernel, sigma, rows=props, cols=props)
    H = A - F[props] @ F[props].T
    u = d[props]
    # walk the oracle's round: numpy's decision away from a tie, the oracle's
    # (its next accepted pivot) within one
    expected = [int(x) for x in S_orc[rank0:rank0 + (int(sizes[rnd]) if rnd < len(sizes) else 0)]]
    acc, atie = [], []
    for i in range(T):
        h = H[i, i]
        atie.append(abs(uacc[i] * u[i] - h) <= TIE * u[i])
        if rank0 + len(acc) >= k:
            continue  # reading c7: the round stops at rank k
        nxt = expected[len(acc)] if len(acc) < len(expected) else None
        take = (props[i] == nxt) if atie[i] else (uacc[i] * u[i] < h)
        if take:
            assert props[i] == nxt, "numpy walk of the round does not reproduce the oracle"
            acc.append(i)
            col = H[i:, i] / np.sqrt(h)
            H[i:, i:] -= np.outer(col, col)
    assert len(acc) == len(expected), "numpy walk of the round does not reproduce the oracle"
    lo = acc[q - 1] + 1 if q > 0 else 0
    hi = acc[q] if q < len(acc) else T - 1
    window = list(range(lo, hi + 1))
    kinds = [("proposal" if ptie[j] else "acceptance", j) for j in window if ptie[j] or atie[j]]
    allowed_idx = set(int(x) for x in props[lo:])
    for j in window:
        if ptie[j]:
            allowed_idx |= nbs[j]
    gpu_piv = int(S_gpu[p]) if p < len(S_gpu) else None
    ok = bool(kinds) and (gpu_piv is None or gpu_piv in allowed_idx)
    return {"position": p, "round": rnd, "q": q, "rank0": rank0, "window": (lo, hi),
            "ties": kinds, "allowed": ok}


def plain_divergence(X, kernel, sigma, k, seed, S_gpu, S_orc, inst=0):
    """The same for simple RPCholesky (Algorithm 6): step p's proposal (the
    uniform of counter (0, p, 0, instance)) must be a near-tie of the
    oracle's d after p steps."""
    p = first_divergence(S_gpu, S_orc)
    if p is None:
        return None
    d = (oracle.rpc_plain(p, seed, X=X, kernel=kernel, sigma=sigma, inst=inst)["d"] if p > 0
         else np.ones(X.shape[0]))
    up, _ = oracle.uniform_pair(seed, 0, p, inst)
    s, near, nb = _proposal(d, up)
    assert p >= len(S_orc) or s == int(S_orc[p]), "replay does not reproduce the oracle"
    gpu_piv = int(S_gpu[p]) if p < len(S_gpu) else None
    ok = near and (gpu_piv is None or gpu_piv in nb | {s})
    return {"position": p, "round": p, "ties": [("proposal", 0)] if near else [],
            "allowed": ok, "rank0": p}
