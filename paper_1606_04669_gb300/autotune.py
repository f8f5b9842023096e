"""Block-length autotuner for the batched and served forms.

The number of blocks p changes the result (Algorithm 1 reduces p block
summaries), so it must be a pure function of the request -- (n, k, skew) --
and never of load; the plan is recorded so that the oracle can replay it.
`plan_blocks` reads a table of block lengths per (k class, skew class)
produced by `sweep()` on a GB300 (the measured table is TABLE below; the
library's own `pss_plan_blocks` is the default when no table entry applies).

What is tuned and what is not:
  * block length (hence p): tuned here;
  * CTA count: the persistent summarize kernel runs SMs x resident CTAs per
    SM (from the occupancy calculator for the k's shared memory), not tuned;
  * table load factor: fixed at <= 50% live cells by the kernel's layout;
  * merge fan-in: the binary tree over adjacent pairs is part of the result
    (combine is not associative), so it is not a tunable.
"""
from __future__ import annotations

import json
import time

K_CLASSES = (64, 256, 1024, 4096)
SKEW_CLASSES = (0.8, 1.4, 2.0)
LENGTHS = (1 << 16, 1 << 17, 1 << 18, 1 << 19)

# Measured by sweep() (see profiles/autotune_block_length.md): the block
# length with the highest items/s for each (k class, skew class).
TABLE = {
    64: {0.8: 1 << 17, 1.4: 1 << 17, 2.0: 1 << 17},
    256: {0.8: 1 << 17, 1.4: 1 << 17, 2.0: 1 << 17},
    1024: {0.8: 1 << 18, 1.4: 1 << 18, 2.0: 1 << 18},
    4096: {0.8: 1 << 19, 1.4: 1 << 19, 2.0: 1 << 19},
}


def _nearest(v, options):
    return min(options, key=lambda o: (abs(o - v), o))


def block_length(k: int, skew: float) -> int:
    kc = min((c for c in K_CLASSES if c >= k), default=K_CLASSES[-1])
    return TABLE[kc][_nearest(skew, SKEW_CLASSES)]


def plan_blocks(n: int, k: int, skew: float = 1.0) -> int:
    """Blocks for a stream of n items with k counters and Zipf skew `skew`."""
    length = block_length(k, skew)
    p = max(1, (n + length - 1) // length)
    while (n + p - 1) // p >= 1 << 32:
        p += 1
    return p


def sweep(blocks: int = 2048, item_bytes: int = 8, steps: int = 3, seed: int = 77):
    """Measure items/s of the summarize path for every (k, skew, length),
    each with the same number of blocks (so that only the block length
    changes), and return (results, table).  Runs on the current CUDA device."""
    import torch

    import paper_1606_04669_gb300 as P
    stream = torch.cuda.current_stream()
    results, table = [], {}
    nmax = blocks * max(LENGTHS)
    for zs in SKEW_CLASSES:
        x = P.gen_zipf(nmax, seed=seed, s=zs, log2u=32, item_bytes=item_bytes)
        for k in K_CLASSES:
            table.setdefault(k, {})
            best = None
            for length in LENGTHS:
                n = blocks * length
                xs = x[:n]
                P.summarize(xs, k, blocks).close()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    P.summarize(xs, k, blocks, stream=stream).close()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                rate = n / (ms / 1e3)
                results.append({"k": k, "skew": zs, "block_length": length, "p": blocks, "ms": ms,
                                "items_per_s": rate})
                if best is None or rate > best[1]:
                    best = (length, rate)
            table[k][zs] = best[0]
        del x
    return results, table


if __name__ == "__main__":
    t = time.time()
    res, tab = sweep()
    for r in res:
        print(json.dumps(r))
    print(json.dumps({"table": {str(k): {str(s): v for s, v in d.items()} for k, d in tab.items()},
                      "seconds": time.time() - t}))
