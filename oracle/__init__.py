"""CPU oracle for Parallel Space Saving (arXiv:1606.04669).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this package.

Thin ctypes wrapper over ``pss_oracle.cpp`` (Space Saving) and
``frequent_oracle.cpp`` (the Frequent / Misra–Gries summary), plain
single-threaded C++; see those files for the passages and published
definitions each function follows.  Summaries are returned in canonical
order: count descending, item ascending.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "pss_oracle.cpp"), os.path.join(_HERE, "frequent_oracle.cpp")]
_GEN = os.path.join(_HERE, "..", "paper_1606_04669_gb300", "gen", "pss_zipf.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

u64p = ctypes.POINTER(ctypes.c_uint64)
u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (two translation units, a few seconds)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest_src = max([os.path.getmtime(f) for f in _SRCS] + [os.path.getmtime(_GEN)])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest_src:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-pthread", "-o", tmp, *_SRCS]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_space_saving.restype = ctypes.c_uint32
        lib.oracle_space_saving.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_uint32, u64p, u64p, u64p, u64p]
        lib.oracle_combine.restype = ctypes.c_uint32
        lib.oracle_combine.argtypes = ([u64p, u64p, u64p, ctypes.c_uint32, ctypes.c_uint64,
                                        ctypes.c_uint64] * 2
                                       + [ctypes.c_uint32, u64p, u64p, u64p, u64p, u64p])
        lib.oracle_tree_nodes.restype = ctypes.c_uint64
        lib.oracle_tree_nodes.argtypes = [ctypes.c_uint64]
        lib.oracle_pss_tree.restype = ctypes.c_int
        lib.oracle_pss_tree.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_uint32, ctypes.c_uint32, u64p, u64p, u64p, u32p,
                                        u64p, u64p]
        lib.oracle_block_summary.restype = ctypes.c_uint32
        lib.oracle_block_summary.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             u64p, u64p, u64p, u64p]
        lib.oracle_query.restype = ctypes.c_uint32
        lib.oracle_query.argtypes = [u64p, u64p, u64p, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_uint32, u64p, u64p, u64p]
        lib.oracle_block_bounds.restype = None
        lib.oracle_block_bounds.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                            u64p, u64p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_philox4x32_10.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint32]
        lib.oracle_gen_zipf.restype = None
        lib.oracle_gen_zipf.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_double, ctypes.c_int]
        lib.oracle_gen_zipf_mt.restype = None
        lib.oracle_gen_zipf_mt.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.oracle_gen_zipf_ranks.restype = None
        lib.oracle_gen_zipf_ranks.argtypes = [u64p, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                              ctypes.c_uint64]
        lib.oracle_rank_to_item.restype = ctypes.c_uint64
        lib.oracle_rank_to_item.argtypes = [ctypes.c_uint64, ctypes.c_int]
        lib.oracle_gen_log.restype = ctypes.c_double
        lib.oracle_gen_log.argtypes = [ctypes.c_double]
        lib.oracle_gen_exp.restype = ctypes.c_double
        lib.oracle_gen_exp.argtypes = [ctypes.c_double]
        for name in ("oracle_gen_log_t", "oracle_gen_exp_t"):
            getattr(lib, name).restype = ctypes.c_double
            getattr(lib, name).argtypes = [ctypes.c_double]
        lib.oracle_frequent.restype = ctypes.c_uint32
        lib.oracle_frequent.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_uint32, u64p, u64p]
        lib.oracle_frequent_combine.restype = ctypes.c_uint32
        lib.oracle_frequent_combine.argtypes = ([u64p, u64p, ctypes.c_uint32, ctypes.c_uint64] * 2
                                                + [ctypes.c_uint32, u64p, u64p, u64p])
        lib.oracle_frequent_tree.restype = ctypes.c_int
        lib.oracle_frequent_tree.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                             ctypes.c_uint32, ctypes.c_uint32, u64p, u64p, u32p,
                                             u64p]
        lib.oracle_frequent_query.restype = ctypes.c_uint32
        lib.oracle_frequent_query.argtypes = [u64p, u64p, ctypes.c_uint32, ctypes.c_uint64,
                                              ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                              u64p, u64p, u64p]
        _lib = lib
        return lib


def _p64(a: np.ndarray):
    return a.ctypes.data_as(u64p)


def _p32(a: np.ndarray):
    return a.ctypes.data_as(u32p)


@dataclass
class Summary:
    """Canonical summary: parallel arrays sorted by (count desc, item asc)."""
    item: np.ndarray
    count: np.ndarray
    err: np.ndarray
    m: int = 0
    n_covered: int = 0

    @property
    def size(self) -> int:
        return int(self.item.shape[0])

    def entries(self):
        return list(zip(self.item.tolist(), self.count.tolist(), self.err.tolist()))


def _items_array(items) -> tuple[np.ndarray, int]:
    a = np.ascontiguousarray(items)
    if a.dtype == np.uint32:
        return a, 4
    if a.dtype == np.uint64:
        return a, 8
    raise TypeError(f"items must be uint32 or uint64, got {a.dtype}")


def block_bounds(n: int, p: int, r: int) -> tuple[int, int]:
    """Algorithm 1 bounds of block r of p: half-open [left, right)."""
    lib = _load()
    lo = np.zeros(1, np.uint64)
    hi = np.zeros(1, np.uint64)
    lib.oracle_block_bounds(n, p, r, _p64(lo), _p64(hi))
    return int(lo[0]), int(hi[0])


def space_saving(items, k: int) -> Summary:
    """Sequential Space Saving with k counters over the whole array (Section 3)."""
    lib = _load()
    a, w = _items_array(items)
    it = np.zeros(k, np.uint64); ct = np.zeros(k, np.uint64); er = np.zeros(k, np.uint64)
    m = np.zeros(1, np.uint64)
    sz = lib.oracle_space_saving(a.ctypes.data_as(ctypes.c_void_p), a.shape[0], w, k,
                                 _p64(it), _p64(ct), _p64(er), _p64(m))
    return Summary(it[:sz].copy(), ct[:sz].copy(), er[:sz].copy(), int(m[0]), int(a.shape[0]))


def block_summary(items, k: int, p: int, r: int) -> Summary:
    """Space Saving summary of block r of p (Algorithm 1 bounds)."""
    lib = _load()
    a, w = _items_array(items)
    it = np.zeros(k, np.uint64); ct = np.zeros(k, np.uint64); er = np.zeros(k, np.uint64)
    m = np.zeros(1, np.uint64)
    sz = lib.oracle_block_summary(a.ctypes.data_as(ctypes.c_void_p), a.shape[0], w, k, p, r,
                                  _p64(it), _p64(ct), _p64(er), _p64(m))
    lo, hi = block_bounds(a.shape[0], p, r)
    return Summary(it[:sz].copy(), ct[:sz].copy(), er[:sz].copy(), int(m[0]), hi - lo)


def combine(a: Summary, b: Summary, k: int) -> Summary:
    """Algorithm 2: combine(S1, S2, k) with Prune(k)."""
    lib = _load()
    arrs = []
    for s in (a, b):
        arrs.append([np.ascontiguousarray(s.item, np.uint64), np.ascontiguousarray(s.count, np.uint64),
                     np.ascontiguousarray(s.err, np.uint64)])
    it = np.zeros(k, np.uint64); ct = np.zeros(k, np.uint64); er = np.zeros(k, np.uint64)
    m = np.zeros(1, np.uint64); cov = np.zeros(1, np.uint64)
    (ai, ac, ae), (bi, bc, be) = arrs
    sz = lib.oracle_combine(_p64(ai), _p64(ac), _p64(ae), a.size, a.m, a.n_covered,
                            _p64(bi), _p64(bc), _p64(be), b.size, b.m, b.n_covered, k,
                            _p64(it), _p64(ct), _p64(er), _p64(m), _p64(cov))
    return Summary(it[:sz].copy(), ct[:sz].copy(), er[:sz].copy(), int(m[0]), int(cov[0]))


def tree_level_sizes(p: int) -> list[int]:
    sizes = [p]
    while sizes[-1] > 1:
        sizes.append((sizes[-1] + 1) // 2)
    return sizes


def pss_tree(items, k: int, p: int) -> list[list[Summary]]:
    """The whole path of Algorithm 1: every level of the reduction tree.

    Level 0 holds the p block summaries; the last level holds the root."""
    lib = _load()
    a, w = _items_array(items)
    nodes = int(lib.oracle_tree_nodes(p))
    it = np.zeros(nodes * k, np.uint64); ct = np.zeros(nodes * k, np.uint64)
    er = np.zeros(nodes * k, np.uint64); sz = np.zeros(nodes, np.uint32)
    m = np.zeros(nodes, np.uint64); cov = np.zeros(nodes, np.uint64)
    lib.oracle_pss_tree(a.ctypes.data_as(ctypes.c_void_p), a.shape[0], w, k, p, _p64(it), _p64(ct),
                        _p64(er), _p32(sz), _p64(m), _p64(cov))
    levels, node = [], 0
    for width in tree_level_sizes(p):
        level = []
        for _ in range(width):
            s = int(sz[node]); base = node * k
            level.append(Summary(it[base:base + s].copy(), ct[base:base + s].copy(),
                                 er[base:base + s].copy(), int(m[node]), int(cov[node])))
            node += 1
        levels.append(level)
    return levels


def pss_tree_threads(items, k: int, p: int, threads: int | None = None) -> list[list[Summary]]:
    """pss_tree with its independent calls spread over host threads.

    Level 0 is the p calls of block_summary (one block each, Algorithm 1
    bounds); every later level is the combines of adjacent pairs of the level
    below (Algorithm 2), the odd last node carried up unchanged.  Each call is
    the same single-threaded C++ as pss_tree's (ctypes releases the GIL, so
    calls on different threads run on different cores); only their
    scheduling differs, and a CPU test checks that the levels equal
    pss_tree's."""
    from concurrent.futures import ThreadPoolExecutor

    a, _ = _items_array(items)
    threads = threads or min(32, os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        levels = [list(ex.map(lambda r: block_summary(a, k, p, r), range(p)))]
        while len(levels[-1]) > 1:
            cur = levels[-1]
            nxt = list(ex.map(lambda i: combine(cur[2 * i], cur[2 * i + 1], k),
                              range(len(cur) // 2)))
            if len(cur) % 2:
                nxt.append(cur[-1])
            levels.append(nxt)
    return levels


def query(s: Summary, n: int, k: int) -> Summary:
    """Pruned(global, n, k): entries with count * k > n, canonical order."""
    lib = _load()
    si = np.ascontiguousarray(s.item, np.uint64); sc = np.ascontiguousarray(s.count, np.uint64)
    se = np.ascontiguousarray(s.err, np.uint64)
    cap = max(s.size, 1)
    it = np.zeros(cap, np.uint64); ct = np.zeros(cap, np.uint64); er = np.zeros(cap, np.uint64)
    sz = lib.oracle_query(_p64(si), _p64(sc), _p64(se), s.size, n, k, _p64(it), _p64(ct), _p64(er))
    return Summary(it[:sz].copy(), ct[:sz].copy(), er[:sz].copy(), s.m, s.n_covered)


def parallel_space_saving(items, k: int, p: int) -> tuple[Summary, Summary]:
    """Algorithm 1 end to end: (root summary, frequent items)."""
    levels = pss_tree(items, k, p)
    root = levels[-1][0]
    n = int(np.asarray(items).shape[0])
    return root, query(root, n, k)


# ----------------------------------------------- accuracy (Section 4 metrics)

def query_guaranteed(s: Summary, n: int, k: int) -> Summary:
    """Entries whose lower bound count - err exceeds n/k ((count - err) * k > n;
    count - err <= f makes each a true k-majority item), canonical order."""
    keep = [i for i in range(s.size) if (int(s.count[i]) - int(s.err[i])) * k > n]
    order = sorted(keep, key=lambda i: (-int(s.count[i]), int(s.item[i])))
    idx = np.array(order, np.int64)
    return Summary(s.item[idx].copy(), s.count[idx].copy(), s.err[idx].copy(), s.m, s.n_covered)


def exact_counts(items, log2u: int) -> np.ndarray:
    """Exact occurrences of every item of [0, 2^log2u); the last entry counts
    the items outside (the exact reference of Section 4's metrics)."""
    x = np.asarray(items).astype(np.uint64)
    u = 1 << log2u
    inside = x < np.uint64(u)
    c = np.bincount(x[inside].astype(np.int64), minlength=u).astype(np.uint64)
    return np.append(c, np.uint64(int((~inside).sum())))


def accuracy(s: Summary, counts: np.ndarray, n: int, k: int) -> dict:
    """Section 4: the relative error |f - f^| / f of each reported frequency
    averaged over the reported items (ARE); precision = true k-majority items
    reported / items reported; recall = true k-majority items reported / true
    k-majority items (f * k > n).  Reported = the query's answer (count * k >
    n).  Empty denominators: ARE 0, precision 1, recall 1."""
    u = counts.shape[0] - 1
    rep = query(s, n, k)
    freq = [int(counts[int(x)]) if int(x) < u else 0 for x in rep.item]
    true_frequent = int(sum(1 for f in counts[:u] if int(f) * k > n))
    tp = sum(1 for f in freq if f * k > n)
    guaranteed = sum(1 for c, e in zip(rep.count, rep.err) if (int(c) - int(e)) * k > n)
    rel = [abs(int(c) - f) / f for c, f in zip(rep.count, freq) if f > 0]
    r = rep.size
    return {"reported": r, "true_frequent": true_frequent, "true_positive": tp,
            "guaranteed": guaranteed, "outside": int(counts[u]),
            "are": (sum(rel) / r) if r else 0.0,
            "precision": (tp / r) if r else 1.0,
            "recall": (tp / true_frequent) if true_frequent else 1.0}


# ------------------------------------------- Frequent (Misra–Gries) summary

def _frequent_summary(it, ct, size, n_covered) -> Summary:
    return Summary(it[:size].copy(), ct[:size].copy(), np.zeros(size, np.uint64), 0,
                   int(n_covered))


def frequent(items, k: int) -> Summary:
    """Misra–Gries with k - 1 counters over the whole array (err and m are 0;
    the bound is frequent_delta)."""
    lib = _load()
    a, w = _items_array(items)
    it = np.zeros(max(k - 1, 1), np.uint64); ct = np.zeros(max(k - 1, 1), np.uint64)
    sz = lib.oracle_frequent(a.ctypes.data_as(ctypes.c_void_p), a.shape[0], w, k, _p64(it), _p64(ct))
    return _frequent_summary(it, ct, sz, a.shape[0])


def frequent_combine(a: Summary, b: Summary, k: int) -> Summary:
    """The merge of two Misra–Gries summaries (k - 1 counters each)."""
    lib = _load()
    ai = np.ascontiguousarray(a.item, np.uint64); ac = np.ascontiguousarray(a.count, np.uint64)
    bi = np.ascontiguousarray(b.item, np.uint64); bc = np.ascontiguousarray(b.count, np.uint64)
    it = np.zeros(max(k - 1, 1), np.uint64); ct = np.zeros(max(k - 1, 1), np.uint64)
    cov = np.zeros(1, np.uint64)
    sz = lib.oracle_frequent_combine(_p64(ai), _p64(ac), a.size, a.n_covered, _p64(bi), _p64(bc),
                                     b.size, b.n_covered, k, _p64(it), _p64(ct), _p64(cov))
    return _frequent_summary(it, ct, sz, int(cov[0]))


def frequent_tree(items, k: int, p: int) -> list[list[Summary]]:
    """p Misra–Gries block summaries and every level of the binary merge tree."""
    lib = _load()
    a, w = _items_array(items)
    nodes = int(lib.oracle_tree_nodes(p))
    stride = k - 1
    it = np.zeros(nodes * stride, np.uint64); ct = np.zeros(nodes * stride, np.uint64)
    sz = np.zeros(nodes, np.uint32); cov = np.zeros(nodes, np.uint64)
    lib.oracle_frequent_tree(a.ctypes.data_as(ctypes.c_void_p), a.shape[0], w, k, p, _p64(it),
                             _p64(ct), _p32(sz), _p64(cov))
    levels, node = [], 0
    for width in tree_level_sizes(p):
        level = []
        for _ in range(width):
            base = node * stride
            level.append(_frequent_summary(it[base:base + stride], ct[base:base + stride],
                                           int(sz[node]), int(cov[node])))
            node += 1
        levels.append(level)
    return levels


def frequent_delta(s: Summary, k: int) -> int:
    """floor((n_covered - sum of counts) / k): count <= f <= count + delta."""
    return (s.n_covered - int(np.asarray(s.count, np.uint64).sum())) // k


def frequent_query(s: Summary, n: int, k: int, guaranteed: bool = False) -> Summary:
    """Entries with (count + delta) * k > n (guaranteed: count * k > n), err =
    delta, canonical order."""
    lib = _load()
    si = np.ascontiguousarray(s.item, np.uint64); sc = np.ascontiguousarray(s.count, np.uint64)
    cap = max(s.size, 1)
    it = np.zeros(cap, np.uint64); ct = np.zeros(cap, np.uint64); er = np.zeros(cap, np.uint64)
    sz = lib.oracle_frequent_query(_p64(si), _p64(sc), s.size, s.n_covered, n, k,
                                   1 if guaranteed else 0, _p64(it), _p64(ct), _p64(er))
    return Summary(it[:sz].copy(), ct[:sz].copy(), er[:sz].copy(), 0, s.n_covered)


def parallel_frequent(items, k: int, p: int) -> tuple[Summary, Summary]:
    """p block summaries, the merge tree and the query: (root, candidates)."""
    root = frequent_tree(items, k, p)[-1][0]
    n = int(np.asarray(items).shape[0])
    return root, frequent_query(root, n, k)


# ---------------------------------------------------------------- generator

def philox4x32_10(counter, key):
    lib = _load()
    c = np.array(counter, np.uint32)
    lib.oracle_philox4x32_10(_p32(c), int(key[0]), int(key[1]))
    return [int(x) for x in c]


def gen_zipf(count: int, *, seed: int, s: float, log2u: int, width: int = 4, stream: int = 0,
             start: int = 0, threads: int = 1) -> np.ndarray:
    """Items [start, start+count) of the seeded Zipf stream (host side)."""
    lib = _load()
    out = np.empty(count, np.uint32 if width == 4 else np.uint64)
    if threads > 1:
        lib.oracle_gen_zipf_mt(out.ctypes.data_as(ctypes.c_void_p), start, count, width, seed,
                               stream, float(s), log2u, threads)
    else:
        lib.oracle_gen_zipf(out.ctypes.data_as(ctypes.c_void_p), start, count, width, seed,
                            stream, float(s), log2u)
    return out


def gen_zipf_ranks(count: int, *, seed: int, s: float, n_ranks: int, stream: int = 0,
                   start: int = 0) -> np.ndarray:
    lib = _load()
    out = np.empty(count, np.uint64)
    lib.oracle_gen_zipf_ranks(_p64(out), start, count, seed, stream, float(s), n_ranks)
    return out


def rank_to_item(r: int, log2u: int) -> int:
    return int(_load().oracle_rank_to_item(r, log2u))


def gen_log(x: float) -> float:
    return float(_load().oracle_gen_log(x))


def gen_exp(x: float) -> float:
    return float(_load().oracle_gen_exp(x))


def gen_log_t(x: float) -> float:
    """The sampler's table-driven log (the generator module's pssg_log_t)."""
    return float(_load().oracle_gen_log_t(x))


def gen_exp_t(x: float) -> float:
    """The sampler's table-driven exp (the generator module's pssg_exp_t)."""
    return float(_load().oracle_gen_exp_t(x))
