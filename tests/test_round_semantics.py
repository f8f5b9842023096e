"""The round decompositions the warp kernels use, restated in plain Python and
checked against the oracle on the CPU: applying a stream 32 items at a time,
in prefixes whose effects commute, gives exactly the sequential result.

* Space Saving (csrc/summarize_round.cu): hits add; new items take free
  counters; on a full summary the first occurrence of each missing item is an
  event taking the next counter of the minimum count in touch order, skipping
  counters hit earlier in the round; a victim hit later ends the prefix; when
  the queue of the minimum runs out it is rebuilt (counters at m + 1 from
  before the epoch in touch order, then the log of those that reached m + 1
  during it).
* Frequent (csrc/frequent.cu): hits add; new items take free counters; on a
  full summary a run of missing occurrences shorter than the smallest count
  is that many decrement steps at once.

No code is shared with the kernels; this pins the argument, the GPU parity
tests pin the kernels."""
from __future__ import annotations

import numpy as np

import oracle


def ss_rounds(xs, k):
    """Space Saving applied in rounds of 32 items (the round kernel's rules)."""
    item, cnt, touch, err = [], [], [], []
    table = {}
    full = False
    state = {"m": 0, "q": [], "qh": 0, "log": [], "epoch": 0}

    def rebuild(now, incremental):
        mn = min(cnt)
        if incremental and mn == state["m"] + 1:
            old = sorted((s for s in range(k) if cnt[s] == mn and touch[s] < state["epoch"]),
                         key=lambda s: touch[s])
            q = old + [s for s in state["log"] if cnt[s] == mn]
        else:
            q = sorted((s for s in range(k) if cnt[s] == mn), key=lambda s: touch[s])
        state.update(m=mn, q=q, qh=0, log=[], epoch=now)

    for t0 in range(0, len(xs), 32):
        chunk = xs[t0:t0 + 32]
        here = len(chunk)
        start = 0
        while start < here:
            lanes = range(start, here)
            probe = {l: table.get(chunk[l], -1) for l in lanes}
            miss = {l: probe[l] < 0 for l in lanes}
            first = {}
            for l in lanes:
                if miss[l] and chunk[l] not in first:
                    first[chunk[l]] = l
            leaders = sorted(first.values())
            if not full:
                free = k - len(item)
                end = here if len(leaders) <= free else leaders[free]
                for l in leaders:
                    if l >= end:
                        break
                    table[chunk[l]] = len(item)
                    item.append(chunk[l]); cnt.append(0); touch.append(0); err.append(0)
                for l in range(start, end):
                    s = table[chunk[l]]
                    cnt[s] += 1
                    touch[s] = t0 + l
                start = end
                if len(item) == k:
                    full = True
                    rebuild(t0 + start, False)
                continue
            m = state["m"]
            earliest = {}
            for l in lanes:
                if not miss[l] and cnt[probe[l]] == m and probe[l] not in earliest:
                    earliest[probe[l]] = l
            end, victim, qp, exhausted = here, {}, state["qh"], False
            q = state["q"]
            for lam in leaders:
                if lam >= end:
                    break
                while qp < len(q) and (cnt[q[qp]] != m or earliest.get(q[qp], 99) < lam):
                    qp += 1
                if qp >= len(q):
                    end, exhausted = lam, True
                    break
                v = q[qp]
                qp += 1
                victim[lam] = v
                if v in earliest and earliest[v] < end:
                    end = earliest[v]
            state["qh"] = qp
            reached = {}
            for lam, v in victim.items():
                if lam < end:
                    del table[item[v]]
                    item[v], err[v], cnt[v] = chunk[lam], m, m
                    table[chunk[lam]] = v
            for l in range(start, end):
                s = table[chunk[l]]
                if cnt[s] == m and s not in reached:
                    reached[s] = l
                cnt[s] += 1
                touch[s] = t0 + l
            for s, _ in sorted(reached.items(), key=lambda e: e[1]):
                if cnt[s] == m + 1:
                    state["log"].append(s)
            start = end
            if exhausted:
                rebuild(t0 + start, True)
    out = [(int(a), int(c), int(e)) for a, c, e in zip(item, cnt, err)]
    return sorted(out, key=lambda e: (-e[1], e[0]))


def mg_rounds(xs, k):
    """Misra-Gries (k - 1 counters) in rounds of 32 with a decrement offset."""
    kc = k - 1
    key, sc = [], []
    table = {}
    base = minc = 0
    for t0 in range(0, len(xs), 32):
        chunk = xs[t0:t0 + 32]
        here = len(chunk)
        start = 0
        while start < here:
            lanes = range(start, here)
            probe = {l: table.get(chunk[l], -1) for l in lanes}
            miss = {l: probe[l] < 0 for l in lanes}
            if len(key) < kc:
                first = {}
                for l in lanes:
                    if miss[l] and chunk[l] not in first:
                        first[chunk[l]] = l
                leaders = sorted(first.values())
                free = kc - len(key)
                end = here if len(leaders) <= free else leaders[free]
                for l in leaders:
                    if l < end:
                        table[chunk[l]] = len(key)
                        key.append(chunk[l]); sc.append(base)
                for l in range(start, end):
                    sc[table[chunk[l]]] += 1
                if len(key) == kc:
                    minc = 1
                start = end
                continue
            misses = [l for l in lanes if miss[l]]
            take = min(len(misses), minc)
            end = here if len(misses) < minc else misses[minc - 1] + 1
            for l in range(start, end):
                if not miss[l]:
                    sc[probe[l]] += 1
            base += take
            minc -= take
            if minc == 0:
                if any(c == base for c in sc):
                    live = [(a, c) for a, c in zip(key, sc) if c != base]
                    key, sc = [a for a, _ in live], [c for _, c in live]
                    table = {a: i for i, a in enumerate(key)}
                else:
                    minc = min(c - base for c in sc)
            start = end
    return sorted(((int(a), c - base) for a, c in zip(key, sc)), key=lambda e: (-e[1], e[0]))


def streams(count, seed):
    rng = np.random.default_rng(seed)
    for t in range(count):
        n = int(rng.integers(0, 400))
        k = int(rng.integers(2, 40))
        if t % 3 == 0:
            x = oracle.gen_zipf(n, seed=t, s=float(rng.uniform(0.5, 2.0)),
                                log2u=int(rng.integers(2, 12)))
        else:
            x = rng.integers(0, int(rng.integers(1, 80)), n).astype(np.uint32)
        yield x, k


def test_space_saving_rounds_equal_the_sequential_rule():
    for x, k in streams(400, 3):
        s = oracle.space_saving(x, k)
        ref = list(zip(s.item.tolist(), s.count.tolist(), s.err.tolist()))
        assert ss_rounds(x.tolist(), k) == ref, (len(x), k)


def test_misra_gries_rounds_equal_the_sequential_rule():
    for x, k in streams(400, 4):
        s = oracle.frequent(x, k)
        assert mg_rounds(x.tolist(), k) == list(zip(s.item.tolist(), s.count.tolist())), (len(x), k)


def test_rounds_on_a_block_of_the_headline_shape():
    x = oracle.gen_zipf(20_000, seed=2, s=1.1, log2u=16)
    s = oracle.space_saving(x, 500)
    assert ss_rounds(x.tolist(), 500) == list(zip(s.item.tolist(), s.count.tolist(), s.err.tolist()))
