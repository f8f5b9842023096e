"""The combine kernel's decomposition (csrc/merge.cu), restated in plain
Python and checked against the oracle's combine on the CPU.

* The union is laid out in the order of the merged sequence of the two
  item-sorted inputs (S1 first on equal items); each thread walks its own run
  of merged positions (odd length) from one merge-path search, and S2's copy
  of an item in both leaves its position empty.
* Prune(k) is a most-significant-digit radix select of c*, 8 bits a pass,
  the digit found by 32 lanes holding 8 bins each (a walk down from digit 255
  that takes digit 0 without checking its bin).
* The keep phase gives each warp a run of merged positions: entries above c*
  stay, and of those equal to c* the first `need` in item order (none for the
  Misra-Gries merge, which subtracts c* instead).

No code is shared with the kernel; this pins the decomposition, the GPU
parity tests pin the kernel."""
from __future__ import annotations

import numpy as np

import oracle

EMPTY = None


def merge_path(a, b, d):
    lo, hi = max(0, d - len(b)), min(d, len(a))
    while lo < hi:
        mid = (lo + hi) // 2
        if a[mid] <= b[d - mid - 1]:
            lo = mid + 1
        else:
            hi = mid
    return lo


def union_in_merged_order(ia, ca, ea, ma, ib, cb, eb, mb, threads):
    """(count, err, item) per merged position, or EMPTY."""
    n = len(ia) + len(ib)
    per = ((n + threads - 1) // threads) | 1
    slots = [0] * n
    for tid in range(threads):
        d0 = min(n, tid * per)
        d1 = min(n, d0 + per)
        i = merge_path(ia, ib, d0)
        j = d0 - i
        for d in range(d0, d1):
            if j >= len(ib) or (i < len(ia) and ia[i] <= ib[j]):
                if j < len(ib) and ib[j] == ia[i]:
                    slots[d] = (ca[i] + cb[j], ea[i] + eb[j], ia[i])
                else:
                    slots[d] = (ca[i] + mb, ea[i] + mb, ia[i])
                i += 1
            else:
                if i > 0 and ia[i - 1] == ib[j]:
                    slots[d] = EMPTY
                else:
                    slots[d] = (cb[j] + ma, eb[j] + ma, ib[j])
                j += 1
    return slots


def digit_of_need(hist, need):
    """32 lanes of 8 bins (lane l: digits 255 - 8l down to 248 - 8l): the
    first lane whose running total reaches `need` walks its bins."""
    sums = [sum(hist[255 - 8 * lane - t] for t in range(8)) for lane in range(32)]
    inc = np.cumsum(sums).tolist()
    reach = [lane for lane in range(32) if inc[lane] >= need]
    lane = reach[0] if reach else 31
    acc = inc[lane] - sums[lane]
    for t in range(8):
        dd = 255 - 8 * lane - t
        v = hist[dd]
        if dd == 0 or acc + v >= need:
            return dd, acc
        acc += v
    raise AssertionError("unreachable")


def radix_select(counts, need):
    """The need-th largest of counts, and how many equal to it are needed."""
    mx = max(counts)
    shift = ((mx.bit_length() - 1) // 8) * 8 if mx else 0
    prefix = pmask = 0
    while shift >= 0:
        hist = [0] * 256
        for c in counts:
            if c & pmask == prefix:
                hist[(c >> shift) & 255] += 1
        d, acc = digit_of_need(hist, need)
        need -= acc
        prefix |= d << shift
        pmask |= 255 << shift
        shift -= 8
    return prefix, need


def keep_by_warp_runs(slots, cut, cstar, need, mg, warps):
    n = len(slots)
    seg = (n + warps - 1) // warps
    runs = [(min(n, w * seg), min(n, min(n, w * seg) + seg)) for w in range(warps)]
    gt_tot = [sum(1 for u in range(a, b) if slots[u] is not EMPTY and (not cut or slots[u][0] > cstar))
              for a, b in runs]
    eq_tot = [sum(1 for u in range(a, b) if slots[u] is not EMPTY and cut and not mg
                  and slots[u][0] == cstar) for a, b in runs]
    out = [None] * (sum(gt_tot) + min(sum(eq_tot), need))
    for w, (a, b) in enumerate(runs):
        gb, eb_ = sum(gt_tot[:w]), sum(eq_tot[:w])
        for u in range(a, b):
            s = slots[u]
            if s is EMPTY:
                continue
            gt = not cut or s[0] > cstar
            eq = cut and not mg and s[0] == cstar
            if gt or (eq and eb_ < need):
                pos = gb + min(eb_, need)
                c = s[0] - cstar if (mg and cut) else s[0]
                out[pos] = (s[2], c, s[1])
            gb += gt
            eb_ += eq
    assert None not in out
    return out


def kernel_combine(a, b, k, threads=64, mg=False):
    """The combine as the kernel decomposes it (k: the capacity of a node)."""
    def by_item(s):
        o = np.argsort(s.item, kind="stable")
        return s.item[o].tolist(), s.count[o].tolist(), s.err[o].tolist()
    ia, ca, ea = by_item(a)
    ib, cb, eb = by_item(b)
    ma, mb = (0, 0) if mg else (a.m, b.m)
    slots = union_in_merged_order(ia, ca, ea, ma, ib, cb, eb, mb, threads)
    live = [s[0] for s in slots if s is not EMPTY]
    cut = len(live) > k
    cstar, need = 0, 0
    if cut:
        cstar, need = radix_select(live, k + 1 if mg else k)
    out = keep_by_warp_runs(slots, cut, cstar, need, mg, max(1, threads // 32))
    if mg:
        m = 0
    elif cut:
        m = cstar
    elif len(live) == k:
        m = min(live)
    else:
        m = 0
    return out, m


def canonical(entries):
    return sorted(entries, key=lambda e: (-e[1], e[0]))


def summaries(seed, count):
    rng = np.random.default_rng(seed)
    for t in range(count):
        k = int(rng.integers(2, 60))
        n1, n2 = (int(rng.integers(0, 600)) for _ in range(2))
        u = int(rng.integers(1, 200))
        if t % 4 == 0:
            x1 = oracle.gen_zipf(n1, seed=t, s=float(rng.uniform(0.6, 2.0)), log2u=int(rng.integers(3, 20)))
            x2 = oracle.gen_zipf(n2, seed=t, s=float(rng.uniform(0.6, 2.0)), log2u=int(rng.integers(3, 20)),
                                 stream=1)
        else:
            x1 = rng.integers(0, u, n1).astype(np.uint32)
            x2 = rng.integers(0, u, n2).astype(np.uint32)
        yield x1, x2, k, int(rng.choice([32, 64, 128, 512]))


def test_space_saving_combine_decomposition_equals_the_oracle():
    for x1, x2, k, threads in summaries(5, 300):
        a, b = oracle.space_saving(x1, k), oracle.space_saving(x2, k)
        ref = oracle.combine(a, b, k)
        out, m = kernel_combine(a, b, k, threads)
        assert canonical(out) == ref.entries(), (len(x1), len(x2), k, threads)
        assert [e[0] for e in out] == sorted(e[0] for e in out)  # item order
        assert m == ref.m


def test_misra_gries_merge_decomposition_equals_the_oracle():
    for x1, x2, k, threads in summaries(6, 300):
        a, b = oracle.frequent(x1, k), oracle.frequent(x2, k)
        ref = oracle.frequent_combine(a, b, k)
        out, _ = kernel_combine(a, b, k - 1, threads, mg=True)
        assert canonical(out) == ref.entries(), (len(x1), len(x2), k, threads)


def test_radix_select_on_wide_counts():
    """Counts spanning several digits (the upper tree levels): the selected
    value is the need-th largest and the tie remainder is exact."""
    rng = np.random.default_rng(7)
    for _ in range(300):
        n = int(rng.integers(1, 400))
        counts = [int(c) for c in rng.integers(1, 1 << int(rng.integers(1, 40)), n)]
        if rng.random() < 0.3:
            counts = [counts[0]] * n  # all equal
        need = int(rng.integers(1, n + 1))
        c, rem = radix_select(counts, need)
        s = sorted(counts, reverse=True)
        assert c == s[need - 1]
        assert rem == need - sum(1 for x in counts if x > c)


def test_headline_shaped_combine():
    x = oracle.gen_zipf(2 * 60_000, seed=2, s=1.1, log2u=16)
    a = oracle.space_saving(x[:60_000], 500)
    b = oracle.space_saving(x[60_000:], 500)
    ref = oracle.combine(a, b, 500)
    out, m = kernel_combine(a, b, 500, threads=512)
    assert canonical(out) == ref.entries()
    assert m == ref.m
