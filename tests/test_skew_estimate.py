"""The batch planner's skew estimate (pss_skew_of_pairs, host side).

A stream's first S items hold P pairs of equal items; P / C(S, 2) estimates
the collision rate sum_i p_i^2, which for Zipf(s) over [0, 2^32) is
H(2^32, 2s) / H(2^32, s)^2.  The estimate inverts that by a table.  Pinned by
closed forms of the rate (zeta values, where the finite universe changes
nothing at the precision checked) and by samples of known skew drawn with
the seeded generator."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import paper_1606_04669_gb300 as P


def pairs_of(x: np.ndarray) -> int:
    _, c = np.unique(x, return_counts=True)
    return int((c.astype(np.int64) * (c - 1) // 2).sum())


def rate_to_pairs(q: float, S: int) -> int:
    return int(round(q * S * (S - 1) / 2))


@pytest.mark.parametrize("s,q", [
    (2.0, (math.pi ** 4 / 90) / (math.pi ** 2 / 6) ** 2),          # zeta(4) / zeta(2)^2 = 2/5
    (1.5, 1.2020569031595942 / 2.612375348685488 ** 2),             # zeta(3) / zeta(1.5)^2
    (3.0, 1.0173430619844491 / 1.2020569031595942 ** 2),            # zeta(6) / zeta(3)^2
])
def test_closed_form_rates(s, q):
    # For s > 1 the tail beyond 2^32 is below 1e-4 of H: the rate is the
    # infinite-universe zeta ratio; a sample of 2^31 items pins it to 1e-9.
    S = 1 << 31
    assert abs(P.skew_of_pairs(rate_to_pairs(q, S), S) - s) < 2e-3


def test_monotone_and_clamped():
    S = 4096
    vals = [P.skew_of_pairs(p, S) for p in (0, 1, 10, 100, 1000, 10_000, 100_000, 1_000_000,
                                            S * (S - 1) // 2)]
    assert vals == sorted(vals)
    assert vals[0] == pytest.approx(0.30) and vals[-1] == pytest.approx(4.00)
    assert P.skew_of_pairs(5, 1) == 0.0 and P.skew_of_pairs(0, 0) == 0.0


@pytest.mark.parametrize("s", [0.8, 0.9, 1.0, 1.1, 1.27, 1.4, 1.6, 1.85, 2.0])
def test_estimate_on_seeded_samples(s):
    # The batched workload's range (s in [0.8, 2], universe 2^32): the mean
    # estimate over 8 streams' 4096-item prefixes lands within 0.05 of s.
    est = []
    for stream in range(8):
        x = oracle.gen_zipf(4096, seed=3, s=s, log2u=32, width=8, stream=stream)
        est.append(P.skew_of_pairs(pairs_of(x), 4096))
    assert abs(np.mean(est) - s) < 0.05, (s, est)
    assert max(abs(e - s) for e in est) < 0.15, (s, est)
