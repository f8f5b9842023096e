"""Seeded parameters of the multi-stream synthetic workloads.

The batched workload (many independent streams of uneven length) and the
served workload (an open-loop Poisson arrival process of stream segments)
draw their per-stream parameters here; the items themselves come from the
seeded Zipf generator (pss_zipf.h, `pss_gen_zipf`).  Draws use Philox4x32-10
in plain Python so that every machine derives the same parameters from a
seed.  Nothing here belongs to the Space Saving method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon et al., SC 2011)."""
    c0, c1, c2, c3 = (x & M32 for x in ctr)
    k0, k1 = key[0] & M32, key[1] & M32
    for r in range(10):
        if r:
            k0 = (k0 + 0x9E3779B9) & M32
            k1 = (k1 + 0xBB67AE85) & M32
        p0 = 0xD2511F53 * c0
        p1 = 0xCD9E8D57 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & M32, p1 & M32, ((p0 >> 32) ^ c3 ^ k1) & M32, p0 & M32
    return [c0, c1, c2, c3]


def uniforms(seed: int, tag: int, index: int):
    """Two uniforms in (0, 1) (52-bit) for draw `index` of purpose `tag`."""
    w = philox4x32_10([index & M32, index >> 32, tag, 0], [seed & M32, seed >> 32])
    u = []
    for a, b in ((w[0], w[1]), (w[2], w[3])):
        j = ((a >> 6) << 26) | (b >> 6)
        u.append((j + 0.5) * 2.0 ** -52)
    return u


def log_uniform_int(u: float, lo: float, hi: float) -> int:
    return int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))))


@dataclass
class StreamSpec:
    index: int
    n: int
    s: float
    k: int
    seed: int
    log2u: int
    item_bytes: int


BATCH_KS = (64, 256, 1024, 4096)


def batched_streams(seed: int = 3, nstreams: int = 1024, lo: float = 1e4, hi: float = 1e8):
    """The batched workload: stream i has a log-uniform length in [lo, hi],
    Zipf skew s uniform in [0.8, 2.0], k uniform over {64, 256, 1024, 4096},
    uint64 items over [0, 2^32); its items are stream id i of `seed`."""
    out = []
    for i in range(nstreams):
        u0, u1 = uniforms(seed, 0x42415443, 2 * i)
        u2, _ = uniforms(seed, 0x42415443, 2 * i + 1)
        out.append(StreamSpec(i, log_uniform_int(u0, lo, hi), 0.8 + 1.2 * u1,
                              BATCH_KS[min(3, int(4 * u2))], seed, 32, 8))
    return out


@dataclass
class Request:
    index: int
    arrival: float   # scheduled arrival, seconds from the start
    tenant: int
    n: int
    s: float
    seed: int
    log2u: int


def served_requests(seed: int = 4, rate: float = 2000.0, duration: float = 60.0,
                    tenants: int = 256, lo: float = 1e4, hi: float = 1e7, log2u: int = 24):
    """The served workload: open-loop Poisson arrivals at `rate` per second
    for `duration` seconds; each request is a segment of log-uniform length
    in [lo, hi] uint32 items, Zipf skew s uniform in [1, 2] over [0, 2^log2u),
    for a tenant drawn uniformly; its items are stream id = request index."""
    out, t, i = [], 0.0, 0
    while True:
        u0, u1 = uniforms(seed, 0x53455256, 2 * i)
        u2, u3 = uniforms(seed, 0x53455256, 2 * i + 1)
        t += -math.log(u0) / rate
        if t >= duration:
            break
        out.append(Request(i, t, min(tenants - 1, int(tenants * u1)), log_uniform_int(u2, lo, hi),
                           1.0 + u3, seed, log2u))
        i += 1
    return out
