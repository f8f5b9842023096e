"""Shared test helpers: golden-fixture parsing, brute-force frequencies and
independent checks of summaries (nothing here imports the CUDA path)."""
from __future__ import annotations

import os
from collections import Counter

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    out = {"stream": [], "a": [], "b": [], "expect": [], "query": [], "freq": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            ints = [int(v) for v in vals]
            if key in ("a", "b", "expect", "freq"):
                out[key].append(tuple(ints))
            elif key in ("stream", "query"):
                out[key].extend(ints)
            elif len(ints) == 2:
                out[key] = (ints[0], ints[1])  # a fraction num / den
            else:
                out[key] = ints[0]
    return out


def exact_counts(items) -> dict:
    return Counter(np.asarray(items).tolist())


def naive_space_saving(items, k):
    """Deliberately naive Space Saving (Section 3): a list of counters and a
    linear scan for the minimum (count, touch).  Independent of the oracle's
    hash map + indexed heap."""
    ctr = []  # [item, count, err, touch]
    for t, x in enumerate(np.asarray(items).tolist()):
        for c in ctr:
            if c[0] == x:
                c[1] += 1
                c[3] = t
                break
        else:
            if len(ctr) < k:
                ctr.append([x, 1, 0, t])
            else:
                v = min(ctr, key=lambda c: (c[1], c[3]))
                v[2] = v[1]
                v[1] += 1
                v[0] = x
                v[3] = t
    ent = sorted(((c[0], c[1], c[2]) for c in ctr), key=lambda e: (-e[1], e[0]))
    m = ent[-1][1] if len(ent) == k else 0
    return ent, m


def canonical(entries):
    return sorted(entries, key=lambda e: (-e[1], e[0]))


def check_bounds(entries, m, true_counts: dict):
    """The Space Saving guarantees for a summary of a sub-stream: every stored
    entry has count - err <= f <= count; every unstored item has f <= m."""
    stored = {}
    for item, count, err in entries:
        f = true_counts.get(item, 0)
        assert count - err <= f <= count, (item, count, err, f)
        stored[item] = True
    for item, f in true_counts.items():
        if item not in stored:
            assert f <= m, (item, f, m)


def summary_entries(s) -> list:
    return list(zip(np.asarray(s.item).tolist(), np.asarray(s.count).tolist(),
                    np.asarray(s.err).tolist()))
