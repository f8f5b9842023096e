"""Autotuner for the batched and served forms.

The number of blocks p changes the result (Algorithm 1 reduces p block
summaries), so it must be a pure function of the request -- (n, k, skew) --
and never of load; the plan is recorded so that the oracle can replay it.
`plan_blocks` reads a table of block lengths per (k class, skew class)
produced by `sweep()` on a GB300 (TABLE below; the library's own
`pss_plan_blocks` is the default when no table is used).

The skew class need not come from the caller: `pss_estimate_skew`
(P.estimate_skew) estimates each stream's Zipf exponent on the device from
the pairs of equal items among its first 4096 items -- an exact count, so the
plan stays a pure function of the stream's bytes and can be replayed.  The
batched benchmark plans from those estimates, not from the generator's s.

What is tuned and what is not:
  * block length (hence p): tuned here, per (k class, skew class);
  * summarize kernel (window-parallel CTA kernel, or one warp per block with
    the counters in registers, for k <= 256): the result does not depend on
    it, so the library picks it per stream from k and the skew hint; the
    skew bands it uses are measured by `sweep_kernels()`;
  * CTA shape of the window-parallel kernel (512 or 256 threads): picked per
    k by the library from the occupancy calculator, not tuned here;
  * CTA count: the persistent kernels run SMs x resident CTAs per SM (from the
    occupancy calculator for the k's shared memory), not tuned;
  * table load factor: fixed at <= 1/2 (k counters plus one window of pending
    items) by the kernel's layout;
  * merge fan-in: the binary tree over adjacent pairs is part of the result
    (combine is not associative), so it is not a tunable.
"""
from __future__ import annotations

import json
import time

K_CLASSES = (64, 256, 1024, 4096)
SKEW_CLASSES = (0.8, 1.4, 2.0)
LENGTHS = (1 << 15, 1 << 16, 1 << 17, 1 << 18, 1 << 19)
FREQUENT_LENGTHS = (1 << 12, 1 << 13, 1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18)

# Measured by sweep() on a GB300 (one stream of 2^27 u64 items per point,
# through the batch path): the block length with the highest items/s for each
# (k class, skew class).  Short blocks win for small k (more blocks in flight,
# and the warp kernel's per-block work is small); k = 4096 (one CTA per SM)
# prefers 2^17, where the per-block set-up and output are amortized.
TABLE = {
    64: {0.8: 1 << 15, 1.4: 1 << 15, 2.0: 1 << 15},
    256: {0.8: 1 << 15, 1.4: 1 << 15, 2.0: 1 << 15},
    1024: {0.8: 1 << 15, 1.4: 1 << 16, 2.0: 1 << 16},
    4096: {0.8: 1 << 17, 1.4: 1 << 17, 2.0: 1 << 17},
}


# The same measurement for the Frequent batch (sweep(frequent=True), lengths
# 2^12 .. 2^16): one warp per block favours shorter blocks.
FREQUENT_TABLE = {
    64: {0.8: 1 << 15, 1.4: 1 << 15, 2.0: 1 << 15},
    256: {0.8: 1 << 15, 1.4: 1 << 15, 2.0: 1 << 15},
    1024: {0.8: 1 << 14, 1.4: 1 << 14, 2.0: 1 << 15},
    4096: {0.8: 1 << 16, 1.4: 1 << 16, 2.0: 1 << 16},
}


def _nearest(v, options):
    return min(options, key=lambda o: (abs(o - v), o))


def block_length(k: int, skew: float, frequent: bool = False) -> int:
    kc = min((c for c in K_CLASSES if c >= k), default=K_CLASSES[-1])
    return (FREQUENT_TABLE if frequent else TABLE)[kc][_nearest(skew, SKEW_CLASSES)]


def plan_blocks(n: int, k: int, skew: float = 1.0, frequent: bool = False) -> int:
    """Blocks for a stream of n items with k counters and Zipf skew `skew`
    (frequent: the Frequent summary's table)."""
    length = block_length(k, skew, frequent)
    p = max(1, (n + length - 1) // length)
    while (n + p - 1) // p >= 1 << 32:
        p += 1
    return p


def _time_batch(P, torch, x, k, p, skew, steps, frequent=False):
    """ms per run of one stream through the batch path (the kernel the batch
    picks for k and the skew hint; frequent: the Frequent summary)."""
    stream = torch.cuda.current_stream()
    b = P.Batch([x], [k], ps=[p], skews=[skew], frequent=frequent)
    b.run(use_graph=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.run(use_graph=False)
    e1.record(stream)
    torch.cuda.synchronize()
    b.close()
    return e0.elapsed_time(e1) / steps


def sweep(n: int = 1 << 27, item_bytes: int = 8, steps: int = 3, seed: int = 77,
          frequent: bool = False, lengths=None):
    """Items/s of the batch path for one stream of n items (about the largest
    stream of the batched workload) for every (k, skew, block length), so
    that the length trades per-block fixed work against the number of blocks
    in flight; returns (results, table).  frequent: the Frequent summary
    (lengths FREQUENT_LENGTHS).  Runs on the current CUDA device."""
    import torch

    import paper_1606_04669_gb300 as P
    lengths = lengths or (FREQUENT_LENGTHS if frequent else LENGTHS)
    results, table = [], {}
    for zs in SKEW_CLASSES:
        x = P.gen_zipf(n, seed=seed, s=zs, log2u=32, item_bytes=item_bytes)
        for k in K_CLASSES:
            table.setdefault(k, {})
            best = None
            for length in lengths:
                p = (n + length - 1) // length
                ms = _time_batch(P, torch, x, k, p, zs, steps, frequent)
                rate = n / (ms / 1e3)
                results.append({"k": k, "skew": zs, "block_length": length, "p": p, "ms": ms,
                                "items_per_s": rate})
                if best is None or rate > best[1]:
                    best = (length, rate)
            table[k][zs] = best[0]
        del x
    return results, table


KERNEL_KS = (32, 48, 64, 96, 128, 160, 192, 224, 256, 320, 384, 448)
KERNEL_SKEWS = (0.5, 0.7, 0.9, 1.0, 1.1, 1.2, 1.3, 1.4, 1.5, 1.6, 1.7, 1.8, 1.9)


def sweep_kernels(n: int = 1 << 28, item_bytes: int = 8, length: int = 1 << 15, steps: int = 4,
                  seed: int = 11):
    """Items/s of the summarize kernels at full occupancy (n / length
    blocks), per (skew, k): the warp kernel (k <= 256), the round kernel and
    the CTA kernel -- the data behind the skew bands by which the batch picks
    a stream's kernel."""
    import torch

    import paper_1606_04669_gb300 as P
    stream = torch.cuda.current_stream()

    def timeit(x, k, p):
        P.summarize(x, k, p).close()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            P.summarize(x, k, p, stream=stream).close()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    out = []
    prev_w = P.set_warp_kmax(0)
    prev_r = P.set_round_kmax(0)
    try:
        for zs in KERNEL_SKEWS:
            x = P.gen_zipf(n, seed=seed, s=zs, log2u=32, item_bytes=item_bytes)
            for k in KERNEL_KS:
                p = n // length
                row = {"skew": zs, "k": k, "block_length": length, "p": p}
                kernels = [("round", 0, P.PSS_MAX_K_RESIDENT), ("cta", 0, 0)]
                if k <= 256:
                    kernels.append(("warp", 256, 0))
                for name, wk, rk in kernels:
                    P.set_warp_kmax(wk)
                    P.set_round_kmax(rk)
                    row[name + "_items_per_s"] = n / (timeit(x, k, p) / 1e3)
                others = [row[nm + "_items_per_s"] for nm in ("cta", "warp") if nm + "_items_per_s" in row]
                row["round_over_best_other"] = row["round_items_per_s"] / max(others)
                if k <= 256:
                    row["warp_over_cta"] = row["warp_items_per_s"] / row["cta_items_per_s"]
                out.append(row)
            del x
    finally:
        P.set_warp_kmax(prev_w)
        P.set_round_kmax(prev_r)
    return out


if __name__ == "__main__":
    t = time.time()
    res, tab = sweep()
    for r in res:
        print(json.dumps(r))
    print(json.dumps({"table": {str(k): {str(s): v for s, v in d.items()} for k, d in tab.items()},
                      "seconds": time.time() - t}))
    for r in sweep_kernels():
        print(json.dumps(r))
