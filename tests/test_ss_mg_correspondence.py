"""Space Saving and Misra–Gries, related through the published correspondence
between the two summaries (Agarwal, Cormode, Huang, Phillips, Wei and Yi,
"Mergeable summaries", PODS 2012): Space Saving with k counters and
Misra–Gries with k - 1 counters over the same stream store the same items
above the Space Saving minimum m, with the Space Saving count equal to the
Misra–Gries count plus m.

The two oracles are separate code (the Section 3 update rule for Space Saving,
the 1982 decrement rule for Misra–Gries), so the correspondence pins each
against the other. The second half shows what the correspondence leaves open:
which items hold the minimum count, decided by the eviction order, is not a
function of the Misra–Gries state, so an exact Space Saving summary cannot be
rebuilt from a Misra–Gries run with a base offset.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle


def above_minimum(s, k):
    m = s.m if s.size == k else 0
    return {int(i): int(c) - m for i, c in zip(s.item, s.count) if int(c) > m}, m


@pytest.mark.parametrize("seed", range(6))
def test_counts_above_the_minimum_are_misra_gries_plus_m(seed):
    rng = np.random.default_rng(seed)
    for _ in range(40):
        k = int(rng.integers(2, 48))
        n = int(rng.integers(1, 4000))
        u = int(rng.integers(2, 400))
        x = (rng.zipf(1.05 + 0.5 * rng.random(), n) % u).astype(np.uint32)
        ss = oracle.space_saving(x, k)
        mg = oracle.frequent(x, k)
        above, m = above_minimum(ss, k)
        assert above == {int(i): int(c) for i, c in zip(mg.item, mg.count)}, (k, n, u)
        # the decrement steps of Misra–Gries are the minimum's rises: n minus
        # the stored Misra–Gries counts is k times m when all k counters fill
        if ss.size == k:
            assert n - int(mg.count.sum()) == k * m
        else:
            assert m == 0 and int(mg.count.sum()) == n


def test_minimum_members_are_not_a_function_of_the_misra_gries_state():
    # k = 2: Space Saving keeps two counters, Misra–Gries one.
    a = np.array([1, 2, 3], np.uint32)
    b = np.array([2, 1, 3], np.uint32)
    mga, mgb = oracle.frequent(a, 2), oracle.frequent(b, 2)
    assert mga.entries() == mgb.entries() == [(3, 1, 0)]
    ssa, ssb = oracle.space_saving(a, 2), oracle.space_saving(b, 2)
    # item 3 evicts the least recently updated counter of count 1
    assert ssa.entries() == [(3, 2, 1), (2, 1, 0)]
    assert ssb.entries() == [(3, 2, 1), (1, 1, 0)]
    assert ssa.m == ssb.m == 1


def test_minimum_members_are_a_large_part_of_a_block_summary():
    # One block of the 2^30-item headline stream (Zipf 1.1 over 2^24, k = 2000,
    # 262,144 items): the members at the minimum are those the
    # correspondence leaves open, and they fill a large part of the summary.
    x = oracle.gen_zipf(262144, seed=2, s=1.1, log2u=24)
    ss = oracle.space_saving(x, 2000)
    mg = oracle.frequent(x, 2000)
    at_m = int((ss.count == ss.m).sum())
    assert ss.size == 2000 and ss.m > 0
    assert at_m + mg.size == 2000
    assert at_m > 500
