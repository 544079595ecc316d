"""CPU checks of the FP64 divergence analyser used by the GPU parity tests:
identical sequences give no divergence; a pivot changed at random (no
near-tie at that decision) is refused, with the round and position located
from the oracle's own round sizes; the replay of a round reproduces the
oracle's accepted pivots."""
import numpy as np
import pytest

import oracle
import workloads
from divergence import accel_divergence, first_divergence, plain_divergence


def test_first_divergence():
    assert first_divergence([1, 2, 3], [1, 2, 3]) is None
    assert first_divergence([1, 2, 4], [1, 2, 3]) == 2
    assert first_divergence([1, 2], [1, 2, 3]) == 2


@pytest.mark.parametrize("pos", [0, 7, 45, 99])
def test_random_change_is_refused_and_located(pos):
    prob = workloads.gauss8_n2000(0)
    k, T, seed = prob.k, prob.T, 3
    o = oracle.rpc_accel(k, T, seed, X=prob.X, kernel=prob.kernel, sigma=prob.sigma)
    S_bad = o["S"].copy()
    S_bad[pos] = (S_bad[pos] + 977) % prob.N
    r = accel_divergence(prob.X, prob.kernel, prob.sigma, k, T, seed, S_bad, o["S"])
    assert r is not None and r["position"] == pos and not r["allowed"]
    cum = np.cumsum(o["round_sizes"])
    assert r["round"] == int(np.searchsorted(cum, pos, side="right"))
    assert r["rank0"] + r["q"] == pos
    assert accel_divergence(prob.X, prob.kernel, prob.sigma, k, T, seed, o["S"], o["S"]) is None


def test_plain_random_change_is_refused():
    prob = workloads.gauss8_n2000(1)
    o = oracle.rpc_plain(40, 5, X=prob.X, kernel=prob.kernel, sigma=prob.sigma)
    S_bad = o["S"].copy()
    S_bad[20] = (S_bad[20] + 311) % prob.N
    r = plain_divergence(prob.X, prob.kernel, prob.sigma, 40, 5, S_bad, o["S"])
    assert r["position"] == 20 and not r["allowed"]
