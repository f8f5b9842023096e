"""Pins of the CPU oracle to what the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: hand-derived
examples (tests/golden), brute-force exact frequencies, the Space Saving error
bounds, closed forms of special streams, and a naive scan implementation."""
from __future__ import annotations

import random
from collections import Counter

import numpy as np
import pytest

import oracle
from tests._helpers import (canonical, check_bounds, exact_counts, naive_space_saving,
                            read_golden, summary_entries)


# ------------------------------------------------------------ golden examples

@pytest.mark.parametrize("name", ["ss_k2_abca.txt", "ss_k2_tie_touch.txt"])
def test_golden_space_saving(name):
    g = read_golden(name)
    s = oracle.space_saving(np.array(g["stream"], np.uint32), g["k"])
    assert summary_entries(s) == g["expect"]
    assert s.m == g["expect_m"]
    q = oracle.query(s, g["query_n"], g["query_k"])
    assert q.item.tolist() == g["query"]


def test_golden_combine():
    g = read_golden("combine_k2.txt")

    def mk(rows, m, n):
        a = np.array(rows, np.uint64).reshape(-1, 3)
        return oracle.Summary(a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy(), m, n)

    a = mk(g["a"], g["a_m"], g["a_n"])
    b = mk(g["b"], g["b_m"], g["b_n"])
    for x, y in ((a, b), (b, a)):
        c = oracle.combine(x, y, g["k"])
        assert summary_entries(c) == g["expect"]
        assert c.m == g["expect_m"]
        assert c.n_covered == g["expect_n"]


# ------------------------------------------------------------ block bounds

def test_block_bounds_examples():
    # Algorithm 1: left = floor(r n / p), right = floor((r + 1) n / p) - 1
    assert [oracle.block_bounds(10, 3, r) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    assert [oracle.block_bounds(2, 5, r) for r in range(5)] == [(0, 0), (0, 0), (0, 1), (1, 1),
                                                                 (1, 2)]


def test_block_bounds_floor_ceil():
    # Section 3: every block holds floor(n/p) or ceil(n/p) items, and they tile [0, n).
    rng = random.Random(5)
    for _ in range(200):
        n = rng.randrange(0, 10 ** 12)
        p = rng.randrange(1, 5000)
        r = rng.randrange(0, p)
        lo, hi = oracle.block_bounds(n, p, r)
        assert hi - lo in (n // p, -(-n // p))
        assert lo == (r * n) // p
    n, p = 1000003, 97
    bounds = [oracle.block_bounds(n, p, r) for r in range(p)]
    assert bounds[0][0] == 0 and bounds[-1][1] == n
    assert all(bounds[i][1] == bounds[i + 1][0] for i in range(p - 1))


# ------------------------------------------------------------ sequential SS

def _rand_stream(rng, n, universe, skew=True):
    if skew:
        w = 1.0 / np.arange(1, universe + 1) ** 1.2
        return rng.choice(np.arange(universe, dtype=np.uint32), size=n, p=w / w.sum())
    return rng.integers(0, universe, size=n, dtype=np.uint32)


def test_naive_twin_agrees():
    rng = np.random.default_rng(11)
    for trial in range(60):
        n = int(rng.integers(0, 600))
        k = int(rng.integers(2, 17))
        u = int(rng.integers(2, 60))
        x = _rand_stream(rng, n, u, skew=bool(trial % 2))
        s = oracle.space_saving(x, k)
        ent, m = naive_space_saving(x, k)
        assert summary_entries(s) == ent
        assert s.m == m


def test_sequential_invariants_and_bounds():
    rng = np.random.default_rng(12)
    for trial in range(80):
        n = int(rng.integers(1, 2000))
        k = int(rng.integers(2, 17))
        x = _rand_stream(rng, n, int(rng.integers(2, 200)), skew=bool(trial % 3))
        s = oracle.space_saving(x, k)
        ent = summary_entries(s)
        assert ent == canonical(ent)
        assert sum(c for _, c, _ in ent) == n  # every item adds exactly one to one counter
        assert len(ent) == min(k, len(set(x.tolist())))
        for _, c, e in ent:
            assert c - e >= 1
            assert e <= s.m
        if len(ent) == k:
            assert s.m == ent[-1][1] and s.m <= n // k
        else:
            assert s.m == 0
        check_bounds(ent, s.m, exact_counts(x))


def test_exact_when_k_exceeds_distinct():
    rng = np.random.default_rng(13)
    x = _rand_stream(rng, 5000, 40)
    s = oracle.space_saving(x, 64)
    vals, cnts = np.unique(x, return_counts=True)
    expect = canonical(list(zip(vals.tolist(), cnts.tolist(), [0] * len(vals))))
    assert summary_entries(s) == expect and s.m == 0


def test_all_distinct_closed_form():
    # n distinct items, k counters: evictions rotate round-robin through the
    # counters (equal counts, oldest touch first); counter j ends with
    # floor((n-1-j)/k)+1 occurrences, the latest item congruent to j mod k,
    # and err = count - 1.
    for n, k in ((1000, 7), (64, 64), (65, 64), (3, 5), (12345, 100)):
        x = np.arange(n, dtype=np.uint32) * 7919 % 1000003  # distinct, not sorted
        s = oracle.space_saving(x, k)
        expect = []
        for j in range(min(k, n)):
            last = j + ((n - 1 - j) // k) * k
            cnt = (n - 1 - j) // k + 1
            expect.append((int(x[last]), cnt, cnt - 1))
        assert summary_entries(s) == canonical(expect)


def test_all_same_item():
    s = oracle.space_saving(np.full(777, 42, np.uint32), 5)
    assert summary_entries(s) == [(42, 777, 0)] and s.m == 0


def test_u64_items():
    rng = np.random.default_rng(14)
    base = rng.integers(0, 2 ** 63, size=50, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    x = base[rng.integers(0, 50, size=3000)]
    ent, m = naive_space_saving(x, 8)
    s = oracle.space_saving(x, 8)
    assert summary_entries(s) == ent and s.m == m


# ------------------------------------------------------------ combine

def _summary_of(x, k):
    return oracle.space_saving(x, k)


def test_combine_properties():
    rng = np.random.default_rng(15)
    for trial in range(60):
        k = int(rng.integers(2, 12))
        u = int(rng.integers(2, 80))
        x1 = _rand_stream(rng, int(rng.integers(0, 400)), u, skew=bool(trial % 2))
        x2 = _rand_stream(rng, int(rng.integers(0, 400)), u, skew=bool(trial % 3))
        a, b = _summary_of(x1, k), _summary_of(x2, k)
        c = oracle.combine(a, b, k)
        c2 = oracle.combine(b, a, k)
        assert summary_entries(c) == summary_entries(c2) and c.m == c2.m  # commutative
        ent = summary_entries(c)
        assert ent == canonical(ent)
        assert c.n_covered == len(x1) + len(x2)
        assert len(ent) <= k
        for _, cnt, _ in ent:
            assert cnt >= a.m + b.m
        if len(ent) == k:
            assert c.m == ent[-1][1] and c.m >= a.m + b.m
        else:
            assert c.m == 0
        both = np.concatenate([x1, x2])
        check_bounds(ent, c.m, exact_counts(both))


def test_combine_exact_union():
    # Both summaries exact and fewer than k distinct items overall: the
    # combined summary is the exact histogram of the concatenation.
    rng = np.random.default_rng(16)
    x1 = _rand_stream(rng, 700, 30)
    x2 = _rand_stream(rng, 500, 30)
    c = oracle.combine(_summary_of(x1, 64), _summary_of(x2, 64), 64)
    vals, cnts = np.unique(np.concatenate([x1, x2]), return_counts=True)
    assert summary_entries(c) == canonical(list(zip(vals.tolist(), cnts.tolist(),
                                                    [0] * len(vals))))


# ------------------------------------------------------------ the whole path

@pytest.mark.parametrize("n,k,p", [(2000, 8, 8), (1999, 5, 7), (300, 16, 1), (10, 4, 16),
                                   (0, 3, 4), (1500, 2, 3)])
def test_tree_levels(n, k, p):
    rng = np.random.default_rng(n + 31 * k + p)
    x = _rand_stream(rng, n, 120)
    levels = oracle.pss_tree(x, k, p)
    assert [len(l) for l in levels] == oracle.tree_level_sizes(p)
    # level 0: the block summaries of Algorithm 1's bounds
    for r, s in enumerate(levels[0]):
        lo, hi = oracle.block_bounds(n, p, r)
        ent, m = naive_space_saving(x[lo:hi], k)
        assert summary_entries(s) == ent and s.m == m and s.n_covered == hi - lo
    # every node of every level respects the bounds over the range it covers
    for li, level in enumerate(levels):
        width = 1 << li
        for j, s in enumerate(level):
            first = j * width
            last = min((j + 1) * width, p)
            lo = oracle.block_bounds(n, p, first)[0]
            hi = oracle.block_bounds(n, p, last - 1)[1]
            assert s.n_covered == hi - lo
            check_bounds(summary_entries(s), s.m, exact_counts(x[lo:hi]))
    root = levels[-1][0]
    assert root.n_covered == n
    # recall: every k-majority item (f * k > n) is reported by the query
    q = oracle.query(root, n, k)
    reported = set(q.item.tolist())
    for item, f in exact_counts(x).items():
        if f * k > n:
            assert item in reported
    assert all(c * k > n for c in q.count.tolist())


@pytest.mark.parametrize("n,k,p,threads", [(200_000, 50, 37, 4), (90_000, 300, 16, 3),
                                           (5, 4, 9, 2), (0, 3, 4, 2), (40_000, 2, 1, 2)])
def test_threaded_tree_equals_tree(n, k, p, threads):
    # The threaded driver used for full-size replays only reschedules the
    # single-threaded calls: every node of every level equals pss_tree's.
    x = oracle.gen_zipf(n, seed=70 + p, s=1.1, log2u=16)
    ref = oracle.pss_tree(x, k, p)
    got = oracle.pss_tree_threads(x, k, p, threads=threads)
    assert [len(l) for l in got] == [len(l) for l in ref]
    for lg, lr in zip(got, ref):
        for g, r in zip(lg, lr):
            assert summary_entries(g) == summary_entries(r)
            assert (g.m, g.n_covered) == (r.m, r.n_covered)


def test_p1_is_sequential():
    rng = np.random.default_rng(17)
    x = _rand_stream(rng, 3000, 500)
    root, _ = oracle.parallel_space_saving(x, 10, 1)
    ent, m = naive_space_saving(x, 10)
    assert summary_entries(root) == ent and root.m == m


def test_exact_when_k_exceeds_distinct_whole_path():
    rng = np.random.default_rng(18)
    x = _rand_stream(rng, 4000, 50)
    root, q = oracle.parallel_space_saving(x, 64, 8)
    vals, cnts = np.unique(x, return_counts=True)
    assert summary_entries(root) == canonical(list(zip(vals.tolist(), cnts.tolist(),
                                                       [0] * len(vals))))
    assert sorted(q.item.tolist()) == sorted(v for v, c in zip(vals.tolist(), cnts.tolist())
                                             if c * 64 > 4000)


def test_query_threshold_boundary():
    # f >= floor(n/k) + 1  <=>  f * k > n  (Section 3)
    s = oracle.Summary(np.array([1, 2, 3], np.uint64), np.array([11, 10, 9], np.uint64),
                       np.zeros(3, np.uint64), 0, 100)
    assert oracle.query(s, 100, 10).item.tolist() == [1]        # floor(100/10)+1 = 11
    assert oracle.query(s, 99, 10).item.tolist() == [1, 2]      # floor(99/10)+1 = 10
    assert oracle.query(s, 2 ** 64 - 1, 2 ** 32 - 1).item.tolist() == []


# ------------------------------------------------------- accuracy (Section 4)

def test_golden_accuracy_metrics():
    from fractions import Fraction
    g = read_golden("accuracy_k4.txt")
    k, n = g["k"], g["n"]
    s = oracle.Summary(np.array([a[0] for a in g["a"]], np.uint64),
                       np.array([a[1] for a in g["a"]], np.uint64),
                       np.array([a[2] for a in g["a"]], np.uint64), 0, n)
    u_bits = 3
    counts = np.zeros((1 << u_bits) + 1, np.uint64)
    for item, f in g["freq"]:
        counts[item] = f
    acc = oracle.accuracy(s, counts, n, k)
    for key in ("reported", "true_frequent", "true_positive", "guaranteed"):
        assert acc[key] == g["expect_" + key], key
    for key in ("are", "precision", "recall"):
        num, den = g["expect_" + key]
        assert Fraction(acc[key]).limit_denominator(1000) == Fraction(num, den), key
    gq = oracle.query_guaranteed(s, n, k)
    assert gq.item.tolist() == [1]


def test_exact_counts_oracle_against_counter():
    rng = np.random.default_rng(4)
    x = rng.integers(0, 1 << 10, size=5000).astype(np.uint32)
    x[::97] = np.uint32(1 << 12)  # outside a 2^10 universe
    c = oracle.exact_counts(x, 10)
    ref = Counter(x.tolist())
    assert int(c[-1]) == ref[1 << 12]
    assert all(int(c[v]) == ref.get(v, 0) for v in range(1 << 10))


@pytest.mark.parametrize("s_,k,p,seed", [(1.1, 50, 4, 31), (0.7, 200, 7, 32), (1.6, 20, 3, 33)])
def test_accuracy_properties(s_, k, p, seed):
    # Space Saving's error bound makes every true k-majority item a reported
    # one (recall 1) and every guaranteed entry truly frequent.
    x = oracle.gen_zipf(80_000, seed=seed, s=s_, log2u=14)
    root, _ = oracle.parallel_space_saving(x, k, p)
    counts = oracle.exact_counts(x, 14)
    acc = oracle.accuracy(root, counts, len(x), k)
    assert acc["recall"] == 1.0
    assert acc["guaranteed"] <= acc["true_positive"] <= acc["reported"]
    assert acc["outside"] == 0 and acc["are"] >= 0.0
    g = oracle.query_guaranteed(root, len(x), k)
    assert all(int(counts[int(v)]) * k > len(x) for v in g.item)
