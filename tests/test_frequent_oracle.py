"""Pins of the CPU oracle's Frequent (Misra–Gries) summary against facts
fixed outside the oracle: the Boyer–Moore majority vote (the algorithm with
one counter), exact histograms, the decrement-count invariant, the error
bounds against brute-force counts, and hand-traced fixtures."""
from __future__ import annotations

from collections import Counter

import numpy as np
import pytest

import oracle
from tests._helpers import read_golden


def entries(s):
    return [(int(i), int(c)) for i, c in zip(s.item, s.count)]


def canonical(d: dict):
    return sorted(((int(x), int(c)) for x, c in d.items() if c > 0), key=lambda e: (-e[1], e[0]))


def boyer_moore(xs):
    """The majority vote of Boyer and Moore (1981): one candidate and a count."""
    cand, cnt = None, 0
    for x in xs:
        if cnt == 0:
            cand, cnt = x, 1
        elif x == cand:
            cnt += 1
        else:
            cnt -= 1
    return cand, cnt


def check_bounds(s, x, k):
    """count <= f <= count + delta for stored items, f <= delta otherwise, and
    no item with f * k > n missing."""
    f = Counter(np.asarray(x).tolist())
    n = len(x)
    d = oracle.frequent_delta(s, k)
    stored = dict(entries(s))
    assert len(stored) == s.size <= k - 1
    for item, c in stored.items():
        assert c <= f[item] <= c + d, (item, c, f[item], d)
    for item, fi in f.items():
        if item not in stored:
            assert fi <= d, (item, fi, d)
        if fi * k > n:
            assert item in stored
    return d


def test_golden_stream():
    g = read_golden("frequent_k3_stream.txt")
    x = np.array(g["stream"], np.uint32)
    s = oracle.frequent(x, g["k"])
    assert entries(s) == [(i, c) for i, c, _ in g["expect"]]
    assert oracle.frequent_delta(s, g["k"]) == g["expect_delta"]
    q = oracle.frequent_query(s, g["query_n"], g["query_k"])
    assert q.item.tolist() == g["query"]
    assert q.err.tolist() == [g["expect_delta"]] * len(g["query"])
    assert oracle.frequent_query(s, g["query_n"], g["query_k"], guaranteed=True).size == 0


@pytest.mark.parametrize("name", ["frequent_combine_k3.txt", "frequent_combine_k3_tie.txt"])
def test_golden_combine(name):
    g = read_golden(name)

    def summ(key):
        rows = g[key]
        return oracle.Summary(np.array([r[0] for r in rows], np.uint64),
                              np.array([r[1] for r in rows], np.uint64),
                              np.zeros(len(rows), np.uint64), 0, g[key + "_n"])

    a, b = summ("a"), summ("b")
    for c in (oracle.frequent_combine(a, b, g["k"]), oracle.frequent_combine(b, a, g["k"])):
        assert entries(c) == [(i, cnt) for i, cnt, _ in g["expect"]]
        assert c.n_covered == g["expect_n"]
        assert oracle.frequent_delta(c, g["k"]) == g["expect_delta"]


def test_one_counter_is_the_majority_vote():
    rng = np.random.default_rng(21)
    for trial in range(300):
        n = int(rng.integers(0, 60))
        alpha = int(rng.integers(1, 5))
        x = rng.integers(0, alpha, n).astype(np.uint32)
        if trial % 3 == 0 and n:
            x[rng.random(n) < 0.6] = 2  # a majority item in a third of the cases
        cand, cnt = boyer_moore(x.tolist())
        s = oracle.frequent(x, 2)
        assert entries(s) == ([(cand, cnt)] if cnt > 0 else [])
        assert oracle.frequent_delta(s, 2) * 2 == n - cnt


def test_exact_when_counters_exceed_distinct_items():
    rng = np.random.default_rng(22)
    for w in (4, 8):
        for _ in range(20):
            d = int(rng.integers(1, 40))
            pool = rng.integers(0, 2 ** (8 * w) - 1, d, dtype=np.uint64)
            x = pool[rng.integers(0, d, 500)].astype(np.uint32 if w == 4 else np.uint64)
            k = len(set(x.tolist())) + 1 + int(rng.integers(0, 3))
            s = oracle.frequent(x, k)
            assert entries(s) == canonical(Counter(x.tolist()))
            assert oracle.frequent_delta(s, k) == 0


@pytest.mark.parametrize("k,zs,log2u", [(2, 1.1, 8), (3, 0.8, 10), (10, 1.1, 16), (64, 0.6, 20),
                                        (100, 1.5, 24), (500, 1.0, 32)])
def test_single_block_invariants(k, zs, log2u):
    x = oracle.gen_zipf(20_000, seed=30 + k, s=zs, log2u=log2u)
    s = oracle.frequent(x, k)
    total = int(s.count.sum())
    assert (len(x) - total) % k == 0  # each decrement step removes k occurrences
    check_bounds(s, x, k)


def test_merge_rules_and_bounds():
    for k, zs, seed in ((3, 1.2, 1), (16, 0.9, 2), (64, 1.1, 3), (200, 0.7, 4)):
        xa = oracle.gen_zipf(8_000, seed=seed, s=zs, log2u=14)
        xb = oracle.gen_zipf(5_000, seed=seed + 100, s=zs, log2u=14)
        a, b = oracle.frequent(xa, k), oracle.frequent(xb, k)
        c, c2 = oracle.frequent_combine(a, b, k), oracle.frequent_combine(b, a, k)
        assert entries(c) == entries(c2)
        assert c.n_covered == a.n_covered + b.n_covered
        assert int(c.count.sum()) <= int(a.count.sum()) + int(b.count.sum())
        check_bounds(c, np.concatenate([xa, xb]), k)


def test_merge_without_cut_adds_counts():
    a = oracle.frequent(np.array([1, 1, 2], np.uint32), 10)
    b = oracle.frequent(np.array([2, 3, 3, 3], np.uint32), 10)
    c = oracle.frequent_combine(a, b, 10)
    assert entries(c) == [(3, 3), (1, 2), (2, 2)]


def test_tree_and_query():
    x = oracle.gen_zipf(30_000, seed=5, s=1.1, log2u=16)
    for k, p in ((20, 1), (20, 7), (100, 16), (3, 5)):
        levels = oracle.frequent_tree(x, k, p)
        assert [len(lv) for lv in levels] == oracle.tree_level_sizes(p)
        for r, s in enumerate(levels[0]):
            lo, hi = oracle.block_bounds(len(x), p, r)
            assert entries(s) == entries(oracle.frequent(x[lo:hi], k))
            assert s.n_covered == hi - lo
        root = levels[-1][0]
        if p == 1:
            assert entries(root) == entries(oracle.frequent(x, k))
        check_bounds(root, x, k)
        f = Counter(x.tolist())
        n = len(x)
        cand = set(oracle.frequent_query(root, n, k).item.tolist())
        assert {i for i, fi in f.items() if fi * k > n} <= cand
        for i in oracle.frequent_query(root, n, k, guaranteed=True).item.tolist():
            assert f[i] * k > n
