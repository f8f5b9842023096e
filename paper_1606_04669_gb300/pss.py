"""Python binding of libpss (include/pss.h): argument marshalling only.

Every step of Parallel Space Saving runs in the library's CUDA kernels; this
module turns torch tensors into device pointers, torch streams into
cudaStream_t handles and PSS_E* codes into exceptions.  There is no CPU
fallback: if libpss cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

PSS_OK = 0
PSS_EINVAL = -1
PSS_EMISMATCH = -2
PSS_ENOMEM = -3
PSS_ECUDA = -4
PSS_ETIMEOUT = -5
PSS_EDEVICE = -6
PSS_ERANGE = -7
PSS_MAX_K = 8192
PSS_MAX_K_RESIDENT = 4096

_lock = threading.Lock()
_lib = None

vp = ctypes.c_void_p
u32 = ctypes.c_uint32
u64 = ctypes.c_uint64
u64p = ctypes.POINTER(ctypes.c_uint64)
u32p = ctypes.POINTER(ctypes.c_uint32)


class PssError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("summarize_calls", ctypes.c_uint64),
                ("merge_levels", ctypes.c_uint64), ("query_calls", ctypes.c_uint64),
                ("summarize_ms", ctypes.c_double), ("merge_ms", ctypes.c_double),
                ("query_ms", ctypes.c_double)]


class Entry(ctypes.Structure):
    _fields_ = [("item", ctypes.c_uint64), ("count", ctypes.c_uint64), ("err", ctypes.c_uint64)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("nstreams", ctypes.c_uint32), ("item_bytes", ctypes.c_int),
                ("d_items", ctypes.POINTER(ctypes.c_void_p)), ("n", ctypes.POINTER(ctypes.c_uint64)),
                ("k", ctypes.POINTER(ctypes.c_uint32)), ("p", ctypes.POINTER(ctypes.c_uint32)),
                ("skew_hint", ctypes.POINTER(ctypes.c_double))]


class Accuracy(ctypes.Structure):
    _fields_ = [("reported", ctypes.c_uint64), ("true_frequent", ctypes.c_uint64),
                ("true_positive", ctypes.c_uint64), ("guaranteed", ctypes.c_uint64),
                ("outside", ctypes.c_uint64), ("are", ctypes.c_double),
                ("precision", ctypes.c_double), ("recall", ctypes.c_double)]


QUERY_CANDIDATES = 0
QUERY_GUARANTEED = 1
KIND_SPACE_SAVING = 0
KIND_FREQUENT = 1


class ServerConfig(ctypes.Structure):
    _fields_ = [("tenants", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("arrival", ctypes.c_double), ("tenant", ctypes.c_uint32),
                ("n", ctypes.c_uint64), ("d_items", ctypes.c_void_p), ("s", ctypes.c_double),
                ("log2u", ctypes.c_int), ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32),
                ("p", ctypes.c_uint32)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tenant", ctypes.c_uint32), ("p", ctypes.c_uint32),
                ("arrival", ctypes.c_double), ("admitted", ctypes.c_double),
                ("completed", ctypes.c_double), ("n_segment", ctypes.c_uint32),
                ("n_tenant", ctypes.c_uint32), ("tenant_items", ctypes.c_uint64),
                ("status", ctypes.c_int)]


# Every function of include/pss.h: name -> (restype, argtypes).
SIGNATURES = {
    "pss_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pss_abi_version": (ctypes.c_int, []),
    "pss_summarize": (ctypes.c_int, [vp, u64, ctypes.c_int, u32, u32, vp, ctypes.POINTER(vp)]),
    "pss_summarize_host": (ctypes.c_int, [vp, u64, ctypes.c_int, u32, u32, vp, ctypes.POINTER(vp)]),
    "pss_summarize_noalloc": (ctypes.c_int, [vp, u64, ctypes.c_int, u32, u32, vp, u64p, u64p, u64p,
                                             vp]),
    "pss_summarize_tree": (ctypes.c_int, [vp, u64, ctypes.c_int, u32, u32, vp, ctypes.POINTER(vp)]),
    "pss_frequent_summarize": (ctypes.c_int, [vp, u64, ctypes.c_int, u32, u32, vp,
                                              ctypes.POINTER(vp)]),
    "pss_frequent_summarize_tree": (ctypes.c_int, [vp, u64, ctypes.c_int, u32, u32, vp,
                                                   ctypes.POINTER(vp)]),
    "pss_frequent_summarize_host": (ctypes.c_int, [vp, u64, ctypes.c_int, u32, u32, vp,
                                                   ctypes.POINTER(vp)]),
    "pss_summary_kind": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
    "pss_tree_kind": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
    "pss_tree_levels": (ctypes.c_int, [vp, u32p]),
    "pss_tree_level_nodes": (ctypes.c_int, [vp, u32, u32p]),
    "pss_tree_read_level": (ctypes.c_int, [vp, u32, u64p, u64p, u64p, u32p, u64p, u64p, vp]),
    "pss_tree_root": (ctypes.c_int, [vp, vp, ctypes.POINTER(vp)]),
    "pss_tree_free": (None, [vp]),
    "pss_merge": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(vp)]),
    "pss_query": (ctypes.c_int, [vp, u64, u32, ctypes.POINTER(Entry), u32, u32p, vp]),
    "pss_query_mode": (ctypes.c_int, [vp, u64, u32, ctypes.c_int, ctypes.POINTER(Entry), u32, u32p, vp]),
    "pss_exact_counts": (ctypes.c_int, [vp, u64, ctypes.c_int, ctypes.c_int, vp, vp]),
    "pss_accuracy_of": (ctypes.c_int, [vp, vp, ctypes.c_int, u64, u32, ctypes.POINTER(Accuracy), vp]),
    "pss_export": (ctypes.c_int, [vp, ctypes.POINTER(Entry), u32, u32p, u64p, u64p, vp]),
    "pss_summary_info": (ctypes.c_int, [vp, u32p, ctypes.POINTER(ctypes.c_int)]),
    "pss_free": (None, [vp]),
    "pss_plan_blocks": (ctypes.c_uint32, [u64, u32, ctypes.c_int, ctypes.c_double]),
    "pss_frequent_plan_blocks": (ctypes.c_uint32, [u64, u32, ctypes.c_int, ctypes.c_double]),
    "pss_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchDesc), vp, ctypes.POINTER(vp)]),
    "pss_frequent_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchDesc), vp,
                                                 ctypes.POINTER(vp)]),
    "pss_batch_plan": (ctypes.c_int, [vp, u32p]),
    "pss_batch_info": (ctypes.c_int, [vp, u32p, u64p, u64p, u32p]),
    "pss_batch_run": (ctypes.c_int, [vp, ctypes.c_int, vp]),
    "pss_batch_results": (ctypes.c_int, [vp, ctypes.POINTER(Entry), u32p, vp]),
    "pss_batch_export": (ctypes.c_int, [vp, u32, ctypes.POINTER(Entry), u32, u32p, u64p, u64p, vp]),
    "pss_batch_free": (None, [vp]),
    "pss_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
    "pss_frequent_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig),
                                                  ctypes.POINTER(vp)]),
    "pss_server_submit": (ctypes.c_int, [vp, ctypes.POINTER(Request), u32]),
    "pss_server_start": (ctypes.c_int, [vp]),
    "pss_server_wait": (ctypes.c_int, [vp, ctypes.c_double]),
    "pss_server_poll": (ctypes.c_int, [vp, ctypes.POINTER(Completion), u32, u32p]),
    "pss_server_result": (ctypes.c_int, [vp, u64, ctypes.POINTER(Entry), u32p, ctypes.POINTER(Entry),
                                         u32p]),
    "pss_import": (ctypes.c_int, [ctypes.POINTER(Entry), u32, u64, u64, u32, ctypes.c_int, vp,
                                  ctypes.POINTER(vp)]),
    "pss_frequent_import": (ctypes.c_int, [ctypes.POINTER(Entry), u32, u64, u32, ctypes.c_int, vp,
                                           ctypes.POINTER(vp)]),
    "pss_server_tenant_import": (ctypes.c_int, [vp, u32, ctypes.POINTER(Entry), u32, u64, u64]),
    "pss_server_inject_alloc_failures": (ctypes.c_int, [vp, u32]),
    "pss_server_tenant_export": (ctypes.c_int, [vp, u32, ctypes.POINTER(Entry), u32, u32p, u64p,
                                                u64p]),
    "pss_server_destroy": (None, [vp]),
    "pss_estimate_skew": (ctypes.c_int, [ctypes.POINTER(vp), u64p, u32, ctypes.c_int, u32, vp,
                                         ctypes.POINTER(ctypes.c_double), u64p]),
    "pss_skew_of_pairs": (ctypes.c_double, [u64, u64]),
    "pss_set_warp_kmax": (ctypes.c_uint32, [ctypes.c_uint32]),
    "pss_set_round_kmax": (ctypes.c_uint32, [ctypes.c_uint32]),
    "pss_plan_kernel": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int]),
    "pss_plan_cta_shape": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pss_set_host_direct": (ctypes.c_int, [ctypes.c_int]),
    "pss_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "pss_profile_read": (ctypes.c_int, [ctypes.POINTER(Profile), ctypes.c_int]),
    "pss_gen_zipf": (ctypes.c_int, [vp, u64, ctypes.c_int, u64, u32, u64, ctypes.c_double,
                                    ctypes.c_int, vp]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpss.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libpss.so is not built ({_build.LIB}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().pss_strerror(code).decode()
    except Exception:  # the library itself failed to load
        return f"error {code}"


def _check(rc: int, what: str):
    if rc != PSS_OK:
        raise PssError(rc, what)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _item_bytes(t) -> int:
    import torch
    if t.dtype in (torch.int32, torch.uint32):
        return 4
    if t.dtype in (torch.int64, torch.uint64):
        return 8
    raise TypeError(f"items must be a 4- or 8-byte integer tensor, got {t.dtype}")


def _check_items(items):
    if not items.is_cuda:
        raise ValueError("items must be a CUDA tensor (the library has no CPU path)")
    if not items.is_contiguous():
        raise ValueError("items must be contiguous")
    return _item_bytes(items)


@dataclass
class Exported:
    """A summary in canonical order (count desc, item asc)."""
    item: np.ndarray
    count: np.ndarray
    err: np.ndarray
    m: int
    n_covered: int

    @property
    def size(self) -> int:
        return int(self.item.shape[0])


def _entries_to_arrays(buf, n):
    if not n:
        z = np.zeros(0, np.uint64)
        return z, z.copy(), z.copy()
    raw = np.frombuffer(memoryview(buf), dtype=np.uint64, count=3 * n).reshape(n, 3)
    return raw[:, 0].copy(), raw[:, 1].copy(), raw[:, 2].copy()


class Summary:
    """A device-resident summary owned by libpss (freed on close / GC):
    Space Saving (kind KIND_SPACE_SAVING) or Frequent / Misra–Gries
    (KIND_FREQUENT: at most k - 1 entries, counts are lower bounds, export's
    m is delta and the queries report err = delta)."""

    def __init__(self, handle: int, stream=None):
        self._h = vp(handle)
        k = u32()
        w = ctypes.c_int()
        kind = ctypes.c_int()
        _check(load().pss_summary_info(self._h, ctypes.byref(k), ctypes.byref(w)), "pss_summary_info")
        _check(load().pss_summary_kind(self._h, ctypes.byref(kind)), "pss_summary_kind")
        self.k = int(k.value)
        self.item_bytes = int(w.value)
        self.kind = int(kind.value)

    @property
    def handle(self):
        return self._h

    def export(self, stream=None) -> Exported:
        buf = (Entry * self.k)()
        size = u32()
        m = u64()
        cov = u64()
        _check(load().pss_export(self._h, buf, self.k, ctypes.byref(size), ctypes.byref(m),
                                 ctypes.byref(cov), vp(_stream_handle(stream))), "pss_export")
        it, ct, er = _entries_to_arrays(buf, size.value)
        return Exported(it, ct, er, int(m.value), int(cov.value))

    def query(self, n: int, k: int | None = None, stream=None, guaranteed: bool = False) -> Exported:
        """pss_query (count k > n), or with guaranteed=True pss_query_mode's
        guaranteed entries ((count - err) k > n)."""
        kq = self.k if k is None else int(k)
        buf = (Entry * self.k)()
        nout = u32()
        if guaranteed:
            _check(load().pss_query_mode(self._h, int(n), kq, QUERY_GUARANTEED, buf, self.k,
                                         ctypes.byref(nout), vp(_stream_handle(stream))),
                   "pss_query_mode")
        else:
            _check(load().pss_query(self._h, int(n), kq, buf, self.k, ctypes.byref(nout),
                                    vp(_stream_handle(stream))), "pss_query")
        it, ct, er = _entries_to_arrays(buf, nout.value)
        return Exported(it, ct, er, 0, int(n))

    def accuracy(self, counts, log2u: int, n: int, k: int | None = None, stream=None) -> dict:
        """pss_accuracy_of against exact counts (a CUDA tensor from exact_counts)."""
        kq = self.k if k is None else int(k)
        if not counts.is_cuda or counts.numel() < (1 << log2u) + 1:
            raise ValueError("counts must be a CUDA tensor of 2^log2u + 1 words")
        a = Accuracy()
        _check(load().pss_accuracy_of(self._h, vp(counts.data_ptr()), int(log2u), int(n), kq,
                                      ctypes.byref(a), vp(_stream_handle(stream))), "pss_accuracy_of")
        return {name: getattr(a, name) for name, _ in Accuracy._fields_}

    def close(self):
        if self._h is not None and self._h.value:
            load().pss_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tree:
    """Every level of one reduction tree (level 0 = block summaries)."""

    def __init__(self, handle: int, k: int | None = None):
        self._h = vp(handle)
        lv = u32()
        kind = ctypes.c_int()
        _check(load().pss_tree_levels(self._h, ctypes.byref(lv)), "pss_tree_levels")
        _check(load().pss_tree_kind(self._h, ctypes.byref(kind)), "pss_tree_kind")
        self.levels = int(lv.value)
        self.kind = int(kind.value)
        self.k = k

    def nodes(self, level: int) -> int:
        n = u32()
        _check(load().pss_tree_level_nodes(self._h, level, ctypes.byref(n)), "pss_tree_level_nodes")
        return int(n.value)

    def read_level(self, level: int, k: int | None = None, stream=None):
        """Raw device layout of one level: list of (items, counts, errs, m, n_covered) per node,
        entries sorted by item ascending (a Frequent tree's nodes hold k - 1 entries)."""
        k = self.k if k is None else int(k)
        if self.kind == KIND_FREQUENT:
            k -= 1
        nodes = self.nodes(level)
        it = np.zeros(nodes * k, np.uint64)
        ct = np.zeros(nodes * k, np.uint64)
        er = np.zeros(nodes * k, np.uint64)
        sz = np.zeros(nodes, np.uint32)
        m = np.zeros(nodes, np.uint64)
        cov = np.zeros(nodes, np.uint64)
        _check(load().pss_tree_read_level(
            self._h, level, it.ctypes.data_as(u64p), ct.ctypes.data_as(u64p),
            er.ctypes.data_as(u64p), sz.ctypes.data_as(u32p), m.ctypes.data_as(u64p),
            cov.ctypes.data_as(u64p), vp(_stream_handle(stream))), "pss_tree_read_level")
        out = []
        for j in range(nodes):
            b, s = j * k, int(sz[j])
            out.append((it[b:b + s].copy(), ct[b:b + s].copy(), er[b:b + s].copy(), int(m[j]),
                        int(cov[j])))
        return out

    def root(self, stream=None) -> Summary:
        h = vp()
        _check(load().pss_tree_root(self._h, vp(_stream_handle(stream)), ctypes.byref(h)),
               "pss_tree_root")
        return Summary(h.value)

    def close(self):
        if self._h is not None and self._h.value:
            load().pss_tree_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def summarize(items, k: int, p: int, stream=None) -> Summary:
    """pss_summarize: block summaries of p blocks merged by the binary tree."""
    w = _check_items(items)
    h = vp()
    _check(load().pss_summarize(vp(items.data_ptr()), items.numel(), w, int(k), int(p),
                                vp(_stream_handle(stream)), ctypes.byref(h)), "pss_summarize")
    return Summary(h.value)


def summarize_host(items, k: int, p: int, stream=None) -> Summary:
    """pss_summarize_host: the same computation on a CPU tensor (pinned for overlap)."""
    if items.is_cuda:
        raise ValueError("summarize_host takes a CPU tensor")
    if not items.is_contiguous():
        raise ValueError("items must be contiguous")
    w = _item_bytes(items)
    h = vp()
    _check(load().pss_summarize_host(vp(items.data_ptr()), items.numel(), w, int(k), int(p),
                                     vp(_stream_handle(stream)), ctypes.byref(h)),
           "pss_summarize_host")
    return Summary(h.value)


def summarize_tree(items, k: int, p: int, stream=None) -> Tree:
    """pss_summarize_tree: as summarize, keeping every tree level."""
    w = _check_items(items)
    h = vp()
    _check(load().pss_summarize_tree(vp(items.data_ptr()), items.numel(), w, int(k), int(p),
                                     vp(_stream_handle(stream)), ctypes.byref(h)),
           "pss_summarize_tree")
    return Tree(h.value, int(k))


def frequent(items, k: int, p: int, stream=None) -> Summary:
    """pss_frequent_summarize: Misra–Gries summaries (k - 1 counters) of p
    blocks merged by the binary tree of Frequent merges."""
    w = _check_items(items)
    h = vp()
    _check(load().pss_frequent_summarize(vp(items.data_ptr()), items.numel(), w, int(k), int(p),
                                         vp(_stream_handle(stream)), ctypes.byref(h)),
           "pss_frequent_summarize")
    return Summary(h.value)


def frequent_host(items, k: int, p: int, stream=None) -> Summary:
    """pss_frequent_summarize_host: frequent() on a CPU tensor (pinned: read
    in place or copies overlapped)."""
    if items.is_cuda:
        raise ValueError("frequent_host takes a CPU tensor")
    if not items.is_contiguous():
        raise ValueError("items must be contiguous")
    w = _item_bytes(items)
    h = vp()
    _check(load().pss_frequent_summarize_host(vp(items.data_ptr()), items.numel(), w, int(k),
                                              int(p), vp(_stream_handle(stream)), ctypes.byref(h)),
           "pss_frequent_summarize_host")
    return Summary(h.value)


def frequent_tree(items, k: int, p: int, stream=None) -> Tree:
    """pss_frequent_summarize_tree: as frequent, keeping every tree level."""
    w = _check_items(items)
    h = vp()
    _check(load().pss_frequent_summarize_tree(vp(items.data_ptr()), items.numel(), w, int(k),
                                              int(p), vp(_stream_handle(stream)), ctypes.byref(h)),
           "pss_frequent_summarize_tree")
    return Tree(h.value, int(k))


def _entries_from(ex: "Exported"):
    n = ex.size
    buf = (Entry * max(n, 1))()
    for i in range(n):
        buf[i].item = int(ex.item[i])
        buf[i].count = int(ex.count[i])
        buf[i].err = int(ex.err[i])
    return buf, n


def import_summary(ex: "Exported", k: int, item_bytes: int = 4, stream=None,
                   frequent: bool = False) -> Summary:
    """pss_import: a device summary from an exported one (a checkpoint);
    frequent: pss_frequent_import (a Frequent summary's export)."""
    buf, n = _entries_from(ex)
    h = vp()
    if frequent:
        _check(load().pss_frequent_import(buf, n, int(ex.n_covered), int(k), int(item_bytes),
                                          vp(_stream_handle(stream)), ctypes.byref(h)),
               "pss_frequent_import")
        return Summary(h.value)
    _check(load().pss_import(buf, n, int(ex.m), int(ex.n_covered), int(k), int(item_bytes),
                             vp(_stream_handle(stream)), ctypes.byref(h)), "pss_import")
    return Summary(h.value)


def merge(a: Summary, b: Summary, stream=None) -> Summary:
    """pss_merge: combine(a, b, k) of Algorithm 2."""
    h = vp()
    _check(load().pss_merge(a.handle, b.handle, vp(_stream_handle(stream)), ctypes.byref(h)),
           "pss_merge")
    return Summary(h.value)


def gen_zipf(count: int, *, seed: int, s: float, log2u: int, item_bytes: int = 4,
             stream_id: int = 0, start: int = 0, out=None, device=None, stream=None):
    """pss_gen_zipf into a new (or the given) CUDA tensor of int32/int64 bit patterns."""
    import torch
    if out is None:
        dt = torch.int32 if item_bytes == 4 else torch.int64
        out = torch.empty(count, dtype=dt, device=device or "cuda")
    else:
        item_bytes = _check_items(out)
        if out.numel() < count:
            raise ValueError("out is too small")
    _check(load().pss_gen_zipf(vp(out.data_ptr()), int(count), int(item_bytes), int(seed),
                               int(stream_id), int(start), float(s), int(log2u),
                               vp(_stream_handle(stream))), "pss_gen_zipf")
    return out


def exact_counts(items, log2u: int, out=None, stream=None):
    """pss_exact_counts: occurrences of every item of [0, 2^log2u) (int32 bit
    patterns of u32 counts; the last word counts items outside)."""
    import torch
    w = _check_items(items)
    if out is None:
        out = torch.empty((1 << log2u) + 1, dtype=torch.int32, device=items.device)
    elif out.numel() < (1 << log2u) + 1:
        raise ValueError("out is too small")
    _check(load().pss_exact_counts(vp(items.data_ptr()), int(items.numel()), int(w), int(log2u),
                                   vp(out.data_ptr()), vp(_stream_handle(stream))), "pss_exact_counts")
    return out


def set_host_direct(on: bool) -> int:
    """pss_summarize_host reads mapped pinned host memory in place (True) or
    stages copies (False).  Returns the previous setting."""
    return int(load().pss_set_host_direct(1 if on else 0))


KERNEL_NAMES = {0: "ss_block_kernel", 1: "ssw_block_kernel", 2: "ssr_block_kernel"}


def plan_kernel(k: int, count: int, item_bytes: int = 4) -> str:
    """pss_plan_kernel: the name of the block-summary kernel the plain path
    runs for `count` blocks with k counters."""
    code = int(load().pss_plan_kernel(int(k), int(count), int(item_bytes)))
    if code < 0:
        raise ValueError("invalid k or item width")
    return KERNEL_NAMES[code]


def plan_cta_shape(k: int, item_bytes: int = 4, batch: bool = False) -> tuple[int, int]:
    """pss_plan_cta_shape: (threads per CTA, items per thread) of the
    window-parallel block-summary kernel for k counters (launches of more
    blocks than the wide shape keeps resident)."""
    t = ctypes.c_int()
    ipt = ctypes.c_int()
    _check(load().pss_plan_cta_shape(int(k), int(item_bytes), 1 if batch else 0, ctypes.byref(t),
                                     ctypes.byref(ipt)), "pss_plan_cta_shape")
    return int(t.value), int(ipt.value)


def set_round_kmax(kmax: int) -> int:
    """pss_set_round_kmax: the largest k the plain path runs on the round
    kernel (0: none); returns the previous value."""
    return int(load().pss_set_round_kmax(int(kmax)))


def set_warp_kmax(kmax: int) -> int:
    """Blocks with k <= kmax counters use the warp-per-block kernel (kmax <= 256;
    0 forces the window-parallel CTA kernel).  Returns the previous value."""
    return int(load().pss_set_warp_kmax(int(kmax)))


def profile_enable(on: bool = True):
    """Time the library's kernel groups with CUDA events from now on."""
    _check(load().pss_profile_enable(1 if on else 0), "pss_profile_enable")


def profile_read(reset: bool = False) -> dict:
    """Launch count and accumulated device times (waits for recorded events)."""
    p = Profile()
    _check(load().pss_profile_read(ctypes.byref(p), 1 if reset else 0), "pss_profile_read")
    return {name: getattr(p, name) for name, _ in Profile._fields_}


def plan_blocks(n: int, k: int, item_bytes: int = 4, skew_hint: float = 0.0,
                frequent: bool = False) -> int:
    """The library's default block count for a stream (pss_plan_blocks, or
    pss_frequent_plan_blocks for the Frequent summary)."""
    fn = load().pss_frequent_plan_blocks if frequent else load().pss_plan_blocks
    return int(fn(int(n), int(k), int(item_bytes), float(skew_hint)))


def estimate_skew(items, sample: int = 4096, stream=None):
    """pss_estimate_skew: (skews, pairs) per stream, from the pairs of equal
    items among each stream's first min(n, sample) items."""
    if not items:
        return [], []
    widths = {_check_items(t) for t in items}
    if len(widths) != 1:
        raise ValueError("every stream must have the same item width")
    ns = len(items)
    ptrs = (vp * ns)(*[t.data_ptr() for t in items])
    n = (ctypes.c_uint64 * ns)(*[t.numel() for t in items])
    sk = (ctypes.c_double * ns)()
    pr = (ctypes.c_uint64 * ns)()
    _check(load().pss_estimate_skew(ptrs, n, ns, widths.pop(), int(sample),
                                    vp(_stream_handle(stream)), sk, pr), "pss_estimate_skew")
    return list(sk), [int(v) for v in pr]


def skew_of_pairs(pairs: int, sample: int) -> float:
    """pss_skew_of_pairs (host only)."""
    return float(load().pss_skew_of_pairs(int(pairs), int(sample)))


class Batch:
    """Many independent streams summarized in one launch graph (pss_batch_*).

    items: CUDA tensors of one item width (borrowed for the batch's life);
    ks: counters per stream; ps: blocks per stream (None / 0 = planned);
    skews: per-stream skew hints for the planner, None (unknown), or
    "estimate" (pss_estimate_skew on each stream's first 4096 items);
    frequent: Frequent (Misra–Gries) summaries instead of Space Saving."""

    def __init__(self, items, ks, ps=None, skews=None, stream=None, frequent: bool = False):
        if not items:
            raise ValueError("a batch needs at least one stream")
        if isinstance(skews, str):
            if skews != "estimate":
                raise ValueError('skews must be a sequence, None or "estimate"')
            skews, _ = estimate_skew(items, stream=stream)
        self.skews = list(skews) if skews is not None else None
        widths = {_check_items(t) for t in items}
        if len(widths) != 1:
            raise ValueError("every stream of a batch must have the same item width")
        self._items = list(items)
        ns = len(items)
        self.item_bytes = widths.pop()
        self._ptrs = (ctypes.c_void_p * ns)(*[t.data_ptr() for t in items])
        self._n = (ctypes.c_uint64 * ns)(*[t.numel() for t in items])
        self._k = (ctypes.c_uint32 * ns)(*[int(k) for k in ks])
        self._p = (ctypes.c_uint32 * ns)(*[int(p or 0) for p in (ps or [0] * ns)])
        self._skew = (ctypes.c_double * ns)(*[float(x or 0.0) for x in (skews or [0.0] * ns)])
        d = BatchDesc(ns, self.item_bytes, self._ptrs, self._n, self._k, self._p, self._skew)
        h = vp()
        create = "pss_frequent_batch_create" if frequent else "pss_batch_create"
        _check(getattr(load(), create)(ctypes.byref(d), vp(_stream_handle(stream)), ctypes.byref(h)),
               create)
        self._h = h
        self.kind = KIND_FREQUENT if frequent else KIND_SPACE_SAVING
        self.nstreams = ns
        self.ks = [int(k) for k in ks]

    def plan(self) -> list[int]:
        out = (ctypes.c_uint32 * self.nstreams)()
        _check(load().pss_batch_plan(self._h, out), "pss_batch_plan")
        return list(out)

    def run(self, use_graph: bool = True, stream=None):
        _check(load().pss_batch_run(self._h, 1 if use_graph else 0, vp(_stream_handle(stream))),
               "pss_batch_run")

    def results(self, stream=None) -> list[Exported]:
        total = sum(self.ks)
        buf = (Entry * total)()
        counts = (ctypes.c_uint32 * self.nstreams)()
        _check(load().pss_batch_results(self._h, buf, counts, vp(_stream_handle(stream))),
               "pss_batch_results")
        raw = np.frombuffer(memoryview(buf), dtype=np.uint64).reshape(total, 3)
        out, off = [], 0
        for i in range(self.nstreams):
            c = int(counts[i])
            r = raw[off:off + c]
            out.append(Exported(r[:, 0].copy(), r[:, 1].copy(), r[:, 2].copy(), 0,
                                int(self._n[i])))
            off += self.ks[i]
        return out

    def export(self, index: int, stream=None) -> Exported:
        k = self.ks[index]
        buf = (Entry * k)()
        size = u32()
        m = u64()
        cov = u64()
        _check(load().pss_batch_export(self._h, int(index), buf, k, ctypes.byref(size),
                                       ctypes.byref(m), ctypes.byref(cov),
                                       vp(_stream_handle(stream))), "pss_batch_export")
        it, ct, er = _entries_to_arrays(buf, size.value)
        return Exported(it, ct, er, int(m.value), int(cov.value))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().pss_batch_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop with continuous batching over resident tenant summaries
    (pss_server_*).  Requests carry scheduled arrival times (open loop).
    frequent: Frequent (Misra–Gries) summaries instead of Space Saving."""

    def __init__(self, tenants: int, k: int, budget_bytes: int = 16 << 30, max_batch: int = 256,
                 max_inflight: int = 2048, frequent: bool = False):
        cfg = ServerConfig(int(tenants), int(k), int(budget_bytes), int(max_batch), int(max_inflight))
        h = vp()
        create = "pss_frequent_server_create" if frequent else "pss_server_create"
        _check(getattr(load(), create)(ctypes.byref(cfg), ctypes.byref(h)), create)
        self._h = h
        self.kind = KIND_FREQUENT if frequent else KIND_SPACE_SAVING
        self.k = int(k)
        self.tenants = int(tenants)
        self._keep = []  # device buffers of caller-provided segments

    def submit(self, requests):
        """requests: iterable of dicts with id, arrival, tenant, n and either
        items (a CUDA uint32 tensor) or s, log2u, seed, stream_id; optional p."""
        reqs = list(requests)
        arr = (Request * len(reqs))()
        for i, r in enumerate(reqs):
            items = r.get("items")
            if items is not None:
                if _check_items(items) != 4:
                    raise ValueError("served segments are 4-byte items")
                self._keep.append(items)
            arr[i] = Request(int(r["id"]), float(r.get("arrival", 0.0)), int(r["tenant"]),
                             int(r["n"]), items.data_ptr() if items is not None else None,
                             float(r.get("s", 1.0)), int(r.get("log2u", 24)), int(r.get("seed", 0)),
                             int(r.get("stream_id", 0)), int(r.get("p", 0) or 0))
        _check(load().pss_server_submit(self._h, arr, len(reqs)), "pss_server_submit")

    def start(self):
        _check(load().pss_server_start(self._h), "pss_server_start")

    def wait(self, timeout_s: float = 600.0):
        _check(load().pss_server_wait(self._h, float(timeout_s)), "pss_server_wait")

    def poll(self, cap: int = 1 << 16) -> list[dict]:
        out = []
        buf = (Completion * cap)()
        while True:
            n = u32()
            _check(load().pss_server_poll(self._h, buf, cap, ctypes.byref(n)), "pss_server_poll")
            for i in range(n.value):
                c = buf[i]
                out.append({f: getattr(c, f) for f, _ in Completion._fields_})
            if n.value < cap:
                return out

    def result(self, rid: int):
        """(segment query, tenant query) of a completed request, as Exported."""
        a = (Entry * self.k)()
        b = (Entry * self.k)()
        na = u32()
        nb = u32()
        _check(load().pss_server_result(self._h, int(rid), a, ctypes.byref(na), b, ctypes.byref(nb)),
               "pss_server_result")
        sa = _entries_to_arrays(a, na.value)
        sb = _entries_to_arrays(b, nb.value)
        return Exported(*sa, 0, 0), Exported(*sb, 0, 0)

    def inject_alloc_failures(self, count: int):
        """pss_server_inject_alloc_failures (fault injection for tests)."""
        _check(load().pss_server_inject_alloc_failures(self._h, int(count)),
               "pss_server_inject_alloc_failures")

    def tenant_import(self, tenant: int, ex: Exported):
        """pss_server_tenant_import: restore a tenant from a checkpoint (before start)."""
        buf, n = _entries_from(ex)
        _check(load().pss_server_tenant_import(self._h, int(tenant), buf, n, int(ex.m),
                                               int(ex.n_covered)), "pss_server_tenant_import")

    def tenant_export(self, tenant: int) -> Exported:
        buf = (Entry * self.k)()
        size = u32()
        m = u64()
        cov = u64()
        _check(load().pss_server_tenant_export(self._h, int(tenant), buf, self.k, ctypes.byref(size),
                                               ctypes.byref(m), ctypes.byref(cov)),
               "pss_server_tenant_export")
        it, ct, er = _entries_to_arrays(buf, size.value)
        return Exported(it, ct, er, int(m.value), int(cov.value))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().pss_server_destroy(self._h)
        self._h = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
