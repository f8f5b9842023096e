"""The allocation-free entry point against the allocating one.

pss_summarize_noalloc serves callers that cannot let the library allocate
device memory: processes whose own allocator owns all device memory, or that
run under a fixed budget and must not allocate after start-up.  It works in a
fixed array inside the library and writes the root summary into buffers the
caller passes in.  This file calls it through the C ABI, twice in a row with
different inputs (the array is shared and keeps the previous call's
contents), and checks every entry and the header against pss_summarize +
pss_export on the same input: exact equality, as everywhere in this integer
path.  It is named to run after every other test file."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_04669_gb300 as P  # noqa: E402

u64p = ctypes.POINTER(ctypes.c_uint64)


def _ptr64(t):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), u64p)


def run_noalloc(x, k, p):
    lib = P.load()
    w = 4 if x.dtype == torch.int32 else 8
    items = torch.full((k,), -1, dtype=x.dtype, device=x.device)
    counts = torch.zeros(k, dtype=torch.int64, device=x.device)
    errs = torch.zeros(k, dtype=torch.int64, device=x.device)
    header = torch.zeros(4, dtype=torch.int64, device=x.device)
    stream = torch.cuda.current_stream()
    rc = lib.pss_summarize_noalloc(ctypes.c_void_p(x.data_ptr()), x.numel(), w, k, p,
                                   ctypes.c_void_p(items.data_ptr()), _ptr64(counts), _ptr64(errs),
                                   _ptr64(header), ctypes.c_void_p(stream.cuda_stream))
    assert rc == P.PSS_OK, P.strerror(rc)
    torch.cuda.synchronize()
    h = header.cpu().numpy().view(np.uint64)
    size, m, ncov, status = (int(v) for v in h)
    it = items.cpu().numpy().view(np.uint32 if w == 4 else np.uint64)[:size].astype(np.uint64)
    ct = counts.cpu().numpy().view(np.uint64)[:size]
    er = errs.cpu().numpy().view(np.uint64)[:size]
    assert np.all(it[1:] > it[:-1]), "root not sorted by item"
    order = np.lexsort((it, -ct.astype(np.float64)))
    entries = list(zip(it[order].tolist(), ct[order].tolist(), er[order].tolist()))
    return entries, m, ncov, status


def run_reference(x, k, p):
    e = P.summarize(x, k, p).export()
    return list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist())), e.m, e.n_covered


@pytest.mark.parametrize("repeat", [0, 1])
def test_noalloc_matches_summarize_on_consecutive_calls(repeat):
    cases = [
        dict(n=1 << 18, seed=1, s=1.1, log2u=18, item_bytes=4, k=100, p=8),
        dict(n=150_000, seed=3, s=1.3, log2u=32, item_bytes=8, k=64, p=5),
    ]
    for c in cases:
        x = P.gen_zipf(c["n"], seed=c["seed"], s=c["s"], log2u=c["log2u"],
                       item_bytes=c["item_bytes"])
        got, m, ncov, status = run_noalloc(x, c["k"], c["p"])
        ref, rm, rcov = run_reference(x, c["k"], c["p"])
        assert status == 0
        assert got == ref
        assert (m, ncov) == (rm, rcov)


def test_noalloc_rejects_sizes_beyond_the_array():
    lib = P.load()
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(4096, dtype=torch.int64, device="cuda")
    rc = lib.pss_summarize_noalloc(ctypes.c_void_p(x.data_ptr()), 1 << 30, 4, 4096, 4096,
                                   ctypes.c_void_p(out.data_ptr()), _ptr64(out), _ptr64(out),
                                   _ptr64(out), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == P.PSS_ERANGE
