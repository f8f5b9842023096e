"""GPU path vs the CPU oracle, through the C ABI (bit-exact: integer work).

Every block summary, every node of every tree level, the root and the query
are compared entry by entry on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests._helpers import canonical, check_bounds, exact_counts, summary_entries

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_04669_gb300 as P  # noqa: E402


def to_dev(x: np.ndarray):
    if x.dtype == np.uint32:
        return torch.from_numpy(x.view(np.int32)).cuda()
    return torch.from_numpy(x.view(np.int64)).cuda()


def node_entries(node):
    it, ct, er, m, cov = node
    return list(zip(it.tolist(), ct.tolist(), er.tolist())), m, cov


def compare_tree(x: np.ndarray, k: int, p: int):
    tree = P.summarize_tree(to_dev(x), k, p)
    ref = oracle.pss_tree(x, k, p)
    assert tree.levels == len(ref)
    for lv, ref_level in enumerate(ref):
        got = tree.read_level(lv, k)
        assert len(got) == len(ref_level)
        for j, (g, r) in enumerate(zip(got, ref_level)):
            ent, m, cov = node_entries(g)
            items = [e[0] for e in ent]
            assert items == sorted(items), f"level {lv} node {j}: device layout not item-sorted"
            assert canonical(ent) == summary_entries(r), f"level {lv} node {j}"
            assert (m, cov) == (r.m, r.n_covered), f"level {lv} node {j}"
    root = tree.root()
    e = root.export()
    r = ref[-1][0]
    assert list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist())) == summary_entries(r)
    assert (e.m, e.n_covered) == (r.m, r.n_covered)
    n = len(x)
    q = root.query(n, k)
    rq = oracle.query(r, n, k)
    assert list(zip(q.item.tolist(), q.count.tolist(), q.err.tolist())) == summary_entries(rq)
    tree.close()
    return root


def test_generator_device_matches_host():
    for (s, log2u, w, start) in ((1.1, 20, 4, 0), (1.0, 32, 4, 12345), (0.5, 32, 8, 7),
                                 (3.0, 24, 4, 1 << 33), (1.8, 32, 8, 999)):
        host = oracle.gen_zipf(100_000, seed=42, s=s, log2u=log2u, width=w, start=start)
        dev = P.gen_zipf(100_000, seed=42, s=s, log2u=log2u, item_bytes=w, start=start)
        got = dev.cpu().numpy().view(np.uint32 if w == 4 else np.uint64)
        assert np.array_equal(got, host), (s, log2u, w)


def test_config1_full_tree():
    # n = 2^20 u32 Zipf(1.1) over [0, 2^20), seed 1, k = 100, p = 8
    x = oracle.gen_zipf(1 << 20, seed=1, s=1.1, log2u=20)
    compare_tree(x, 100, 8)


@pytest.mark.parametrize("n,k,p,w,s,log2u,seed", [
    (50_000, 64, 4, 4, 1.1, 16, 101),
    (123_457, 200, 13, 4, 0.8, 20, 102),     # odd p: carried nodes
    (200_000, 500, 5, 4, 1.5, 32, 103),
    (300_000, 1000, 3, 4, 1.0, 32, 104),
    (100_000, 2000, 8, 8, 1.2, 32, 105),     # u64 items
    (80_000, 4096, 2, 4, 0.9, 24, 106),      # the largest k
    (80_000, 4096, 3, 8, 1.3, 40, 107),
    (60_000, 2, 9, 4, 1.1, 12, 108),          # k = 2
    (70_000, 333, 31, 4, 0.5, 32, 109),       # nearly every item misses
    (150_000, 1024, 1, 8, 2.0, 32, 110),      # p = 1: plain sequential Space Saving
    (262_144, 2000, 1, 4, 1.1, 24, 2),        # one block of the 2^30 stream's shape
    (300_000, 3000, 5, 4, 1.0, 32, 111),      # 2048 < k <= 3072: the large-k form in shared memory
    (200_000, 2500, 3, 8, 1.5, 32, 112),
])
def test_random_configs(n, k, p, w, s, log2u, seed):
    x = oracle.gen_zipf(n, seed=seed, s=s, log2u=log2u, width=w)
    compare_tree(x, k, p)


def shape_switches(w: int):
    """The k where the CTA kernel's shape changes (last k of one shape, first
    of the next), found through pss_plan_cta_shape."""
    out = []
    prev = P.plan_cta_shape(2, w)
    for k in range(3, 4097):
        cur = P.plan_cta_shape(k, w)
        if cur != prev:
            out.append((k - 1, k, prev, cur))
        prev = cur
    return out


def test_cta_shapes_in_order():
    # 256 x 4 (1024-item window) at the smallest k, then 256 x 2 (512-item
    # window), then 512 x 2.  Where k is so large that every shape keeps the
    # same 512 threads resident, the tie order picks again (256 x 4 first).
    for w in (4, 8):
        seq = [P.plan_cta_shape(2, w)] + [c[3] for c in shape_switches(w)]
        assert seq[:3] == [(256, 4), (256, 2), (512, 2)], (w, seq)
        assert set(seq) == {(256, 4), (256, 2), (512, 2)}, (w, seq)
    assert P.plan_cta_shape(8192, 4) == (512, 2)
    with pytest.raises(P.PssError):
        P.plan_cta_shape(1, 4)


@pytest.mark.parametrize("w", [4, 8])
def test_cta_shape_boundaries(w):
    # Both sides of every shape switch, with cut windows (weak skew over a
    # large universe) and with hits (strong skew over a small one).  Launches
    # that fit on the SMs at once in the wide shape run it, so a few blocks of
    # the k-sized state test the wide shape and 320 blocks (more than the 304
    # wide CTAs a GB300 keeps resident below k ~ 2000) the shape of the switch.
    for last, first, _, _ in shape_switches(w):
        for k in (last, first):
            x = oracle.gen_zipf(180_000 + k, seed=900 + k, s=0.9, log2u=32, width=w)
            compare_tree(x, k, 3)
            y = oracle.gen_zipf(120_000, seed=950 + k, s=1.8, log2u=18, width=w)
            compare_tree(y, k, 2)
            z = oracle.gen_zipf(320 * 1536 + k, seed=970 + k, s=0.9, log2u=32, width=w)
            compare_tree(z, k, 320)


def test_edge_empty_and_tiny():
    compare_tree(np.zeros(0, np.uint32), 5, 4)            # n = 0
    compare_tree(np.array([7, 7, 9], np.uint32), 4, 8)     # n < p: empty blocks
    compare_tree(np.array([3, 1, 2], np.uint32), 16, 1)    # n < k
    compare_tree(np.array([1, 2, 3, 1], np.uint32), 2, 1)  # the golden example
    compare_tree(np.array([1, 2, 2, 1, 3], np.uint32), 2, 1)


def test_edge_all_same_and_all_distinct():
    compare_tree(np.full(100_000, 0xFFFFFFFF, np.uint32), 10, 7)   # sentinel-valued item
    compare_tree(np.arange(100_000, dtype=np.uint32) * np.uint32(2654435761), 100, 4)
    compare_tree(np.full(5000, np.uint64(2 ** 64 - 1)), 3, 2)


def test_edge_hash_collisions():
    # Items that are multiples of large powers of two collide in naive hashes.
    rng = np.random.default_rng(5)
    base = (np.arange(3000, dtype=np.uint64) << np.uint64(20)).astype(np.uint32)
    x = base[rng.zipf(1.3, size=200_000) % 3000]
    compare_tree(x, 512, 4)
    x64 = (np.arange(5000, dtype=np.uint64) << np.uint64(40))[rng.zipf(1.2, 100_000) % 5000]
    compare_tree(x64, 256, 3)


def test_interleaved_hits_misses_windows():
    # Periodic streams hit the window-prefix logic (conflicts between hits and
    # evictions in one window, bucket exhaustion mid-window).
    pat = np.concatenate([np.arange(40, dtype=np.uint32), np.arange(20, dtype=np.uint32)])
    x = np.tile(pat, 3000)
    compare_tree(x, 30, 3)
    y = np.tile(np.arange(300, dtype=np.uint32), 800)
    compare_tree(y, 256, 2)
    z = np.repeat(np.arange(1000, dtype=np.uint32), 3)[np.random.default_rng(3).permutation(3000)]
    compare_tree(np.tile(z, 50), 100, 5)


def test_merge_api():
    xa = oracle.gen_zipf(200_000, seed=7, s=1.1, log2u=20)
    xb = oracle.gen_zipf(150_000, seed=8, s=1.3, log2u=20)
    for k in (2, 100, 1000):
        a = P.summarize(to_dev(xa), k, 4)
        b = P.summarize(to_dev(xb), k, 3)
        ra, _ = oracle.parallel_space_saving(xa, k, 4)
        rb, _ = oracle.parallel_space_saving(xb, k, 3)
        for (u, v, ru, rv) in ((a, b, ra, rb), (b, a, rb, ra)):
            c = P.merge(u, v)
            e = c.export()
            rc = oracle.combine(ru, rv, k)
            assert list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist())) == \
                summary_entries(rc)
            assert (e.m, e.n_covered) == (rc.m, rc.n_covered)
    a = P.summarize(to_dev(xa), 10, 2)
    b = P.summarize(to_dev(xb), 11, 2)
    with pytest.raises(P.PssError) as ei:
        P.merge(a, b)
    assert ei.value.code == P.PSS_EMISMATCH


def select_edge_pair(rng, k: int, gap: int, w: int):
    """Two summaries of disjoint items (fewer than k entries each, so m = 0
    and every union count is the entry's own count) whose union keeps k of
    U > k entries, with the cut value c* exactly `gap` above the union's
    minimum, ties at c* on both sides of the cut."""
    U = k + 1 + int(rng.integers(0, k - 2))   # <= 2k - 2: both sides fit below k
    r = U - k + 1                      # c* is the r-th smallest
    base = int(rng.integers(1, 1000))
    low = [base] + [base + int(rng.integers(0, gap + 1)) for _ in range(r - 2)] if r >= 2 else []
    cstar = base + gap
    high = [cstar + (0 if rng.random() < 0.3 else int(rng.integers(1, 10_000))) for _ in range(U - r)]
    counts = np.array(low + [cstar] + high, np.uint64)
    rng.shuffle(counts)
    hi_item = (1 << 32) if w == 4 else (1 << 40)
    items = rng.choice(hi_item, size=U, replace=False).astype(np.uint64)
    na = int(rng.integers(max(1, U - k + 1), k))   # both sides below k entries
    parts = []
    for it, ct in ((items[:na], counts[:na]), (items[na:], counts[na:])):
        order = np.lexsort((it, -ct.astype(np.int64)))
        parts.append(oracle.Summary(it[order], ct[order], np.zeros(len(it), np.uint64), 0,
                                    int(ct.sum())))
    return parts


@pytest.mark.parametrize("w", [4, 8])
def test_merge_select_both_paths(w):
    # The combine finds c* with one histogram of distances from the union's
    # minimum when c* lies within 254 of it, else with the radix select:
    # distances on both sides of that edge, against Algorithm 2 in the oracle.
    rng = np.random.default_rng(400 + w)
    for gap in (0, 1, 253, 254, 255, 256, 70_000, 5_000_000_000):
        for k in (3, 5, 100, 2000):
            ra, rb = select_edge_pair(rng, k, gap, w)
            da = P.import_summary(P.Exported(ra.item, ra.count, ra.err, 0, ra.n_covered), k, w)
            db = P.import_summary(P.Exported(rb.item, rb.count, rb.err, 0, rb.n_covered), k, w)
            e = P.merge(da, db).export()
            rc = oracle.combine(ra, rb, k)
            assert list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist())) == \
                summary_entries(rc), (gap, k)
            assert (e.m, e.n_covered) == (rc.m, rc.n_covered), (gap, k)
            # the Frequent merge selects the same way (k - 1 counters: the
            # entries fit, and U > k - 1 cuts at the k-th largest)
            fa = P.import_summary(P.Exported(ra.item, ra.count, ra.err, 0, ra.n_covered), k, w,
                                  frequent=True)
            fb = P.import_summary(P.Exported(rb.item, rb.count, rb.err, 0, rb.n_covered), k, w,
                                  frequent=True)
            f = P.merge(fa, fb).export()
            rf = oracle.frequent_combine(ra, rb, k)
            assert list(zip(f.item.tolist(), f.count.tolist())) == \
                list(zip(rf.item.tolist(), rf.count.tolist())), ("frequent", gap, k)


def test_argument_errors():
    x = to_dev(np.arange(100, dtype=np.uint32))
    for k, p in ((1, 4), (P.PSS_MAX_K + 1, 4), (10, 0)):
        with pytest.raises(P.PssError) as ei:
            P.summarize(x, k, p)
        assert ei.value.code == P.PSS_EINVAL
    s = P.summarize(x, 8, 2)
    lib = P.load()
    import ctypes
    buf = (P.pss.Entry * 1)()
    n = ctypes.c_uint32()
    rc = lib.pss_export(s.handle, buf, 1, ctypes.byref(n), None, None,
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == P.PSS_ERANGE


def test_config2_sampled_blocks_and_full_size_properties():
    # n = 2^30 u32 Zipf(1.1) over [0, 2^24), seed 2, k = 2000, p = 4096.
    n, k, p = 1 << 30, 2000, 4096
    x = P.gen_zipf(n, seed=2, s=1.1, log2u=24)
    tree = P.summarize_tree(x, k, p)
    level0 = tree.read_level(0, k)
    for r in (0, 1, 777, 2048, 4094, 4095):
        lo, hi = oracle.block_bounds(n, p, r)
        xr = oracle.gen_zipf(hi - lo, seed=2, s=1.1, log2u=24, start=lo)
        ref = oracle.space_saving(xr, k)
        ent, m, cov = node_entries(level0[r])
        assert canonical(ent) == summary_entries(ref), r
        assert (m, cov) == (ref.m, hi - lo)
    # Root against exact frequencies of the whole stream (torch histogram).
    root = tree.root()
    e = root.export()
    f = torch.bincount(x.view(torch.int32).to(torch.int64), minlength=1 << 24).cpu().numpy()
    assert e.n_covered == n and e.size == k
    assert np.all(e.count - e.err <= f[e.item.astype(np.int64)])
    assert np.all(f[e.item.astype(np.int64)] <= e.count)
    mask = np.ones(1 << 24, bool)
    mask[e.item.astype(np.int64)] = False
    assert f[mask].max() <= e.m
    q = root.query(n, k)
    truly = set(np.nonzero(f * k > n)[0].tolist())
    assert truly <= set(q.item.tolist())  # 100% recall
    tree.close()


@pytest.mark.parametrize("direct,pinned", [(True, True), (False, True), (True, False)])
def test_host_input_path(direct, pinned):
    # pss_summarize_host: pinned memory read in place by the kernels, or slab
    # copies overlapping the kernels (direct reads off, or pageable memory).
    prev = P.set_host_direct(direct)
    try:
        for (n, k, p, w) in ((500_000, 300, 37, 4), (300_000, 1000, 16, 8), (1000, 50, 40, 4),
                             (200_000, 6000, 3, 4)):
            x = oracle.gen_zipf(n, seed=21 + k, s=1.1, log2u=20, width=w)
            h = torch.from_numpy(x.view(np.int32 if w == 4 else np.int64))
            if pinned:
                h = h.pin_memory()
            e = P.summarize_host(h, k, p).export()
            r, q = oracle.parallel_space_saving(x, k, p)
            assert list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist())) == summary_entries(r)
            assert (e.m, e.n_covered) == (r.m, r.n_covered)
    finally:
        P.set_host_direct(bool(prev))


def test_fuzz_small_universes():
    # Many skips, conversions and in-window epoch ends: small k, small
    # universes, skewed draws, windows cut at every kind of boundary.
    rng = np.random.default_rng(20261203)
    for trial in range(60):
        k = int(rng.integers(2, 300))
        n = int(rng.integers(0, 60_000))
        p = int(rng.integers(1, 9))
        u = int(rng.integers(2, 4 * k + 50))
        a = 1.05 + 1.5 * rng.random()
        ranks = np.minimum(rng.zipf(a, size=n), u) - 1
        perm = rng.permutation(u).astype(np.uint64)
        w = 8 if trial % 3 == 0 else 4
        vals = perm[ranks] * np.uint64(2654435761 if w == 4 else 0x9E3779B97F4A7C15 >> 1)
        x = vals.astype(np.uint32) if w == 4 else vals.astype(np.uint64)
        compare_tree(x, k, p)


@pytest.fixture
def warp_kmax():
    prev = P.set_warp_kmax(256)
    yield P.set_warp_kmax
    P.set_warp_kmax(prev)


@pytest.mark.parametrize("kmax", [0, 256])
def test_small_k_both_kernels(warp_kmax, kmax):
    # k <= 256 runs one warp per block (counters in registers) by default;
    # kmax = 0 sends the same blocks through the window-parallel CTA kernel.
    warp_kmax(kmax)
    rng = np.random.default_rng(77 + kmax)
    for k in (2, 3, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256):
        w = 8 if k % 2 else 4
        s = 0.6 + 1.6 * rng.random()
        x = oracle.gen_zipf(40_000 + 97 * k, seed=500 + k, s=s, log2u=14 if k < 64 else 32, width=w)
        compare_tree(x, k, 1 + k % 7)
    compare_tree(np.full(5000, 0xFFFFFFFF, np.uint32), 64, 3)
    compare_tree(np.arange(20_000, dtype=np.uint32), 256, 2)   # every item a miss
    compare_tree(np.zeros(0, np.uint32), 16, 3)


def test_fuzz_small_universes_cta_kernel(warp_kmax):
    # The fuzz cases again with every block on the window-parallel CTA kernel.
    warp_kmax(0)
    test_fuzz_small_universes()


@pytest.mark.parametrize("n,k,p,w,s,log2u,seed", [
    (120_000, 4097, 3, 4, 0.9, 20, 201),
    (200_000, 6000, 2, 8, 1.1, 24, 202),
    (150_000, 8000, 3, 4, 0.6, 32, 203),    # the paper's largest k; nearly every item misses
    (300_000, 8192, 2, 8, 1.5, 32, 204),
    (40_000, 8192, 5, 4, 1.0, 12, 205),     # fewer distinct items than k
])
def test_large_k_beyond_shared_memory(n, k, p, w, s, log2u, seed):
    # k > 4096 keeps part of the block and combine state in HBM scratch.
    x = oracle.gen_zipf(n, seed=seed, s=s, log2u=log2u, width=w)
    compare_tree(x, k, p)


def test_large_k_merge_and_resident_limits():
    xa = oracle.gen_zipf(100_000, seed=211, s=0.8, log2u=24)
    xb = oracle.gen_zipf(90_000, seed=212, s=1.2, log2u=24)
    a = P.summarize(to_dev(xa), 8000, 2)
    b = P.summarize(to_dev(xb), 8000, 3)
    ra, _ = oracle.parallel_space_saving(xa, 8000, 2)
    rb, _ = oracle.parallel_space_saving(xb, 8000, 3)
    e = P.merge(a, b).export()
    rc = oracle.combine(ra, rb, 8000)
    assert list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist())) == summary_entries(rc)
    # the batch and server keep every summary in shared memory: k <= 4096
    with pytest.raises(P.PssError) as ei:
        P.Batch([to_dev(xa)], [P.PSS_MAX_K_RESIDENT + 1])
    assert ei.value.code == P.PSS_EINVAL
    with pytest.raises(P.PssError) as ei:
        P.Server(2, P.PSS_MAX_K_RESIDENT + 1)
    assert ei.value.code == P.PSS_EINVAL


@pytest.mark.parametrize("w,off", [(4, 1), (4, 2), (4, 3), (8, 1)])
def test_input_pointer_offsets(w, off):
    # Windows are copied in 16-byte pieces aligned to global memory, so every
    # offset of the input pointer within 16 bytes (a view starting `off`
    # items into an aligned tensor) is compared with the oracle, with blocks,
    # cut windows and the stream's end at every offset as well.
    x = oracle.gen_zipf(300_001 + off, seed=60 + off, s=1.0, log2u=20, width=w)
    dev = to_dev(x)[off:]
    assert dev.data_ptr() % 16 == off * w
    for k, p in ((700, 7), (2000, 3), (100, 1)):
        e = P.summarize(dev, k, p).export()
        r, _ = oracle.parallel_space_saving(x[off:], k, p)
        assert list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist())) == summary_entries(r)
        assert (e.m, e.n_covered) == (r.m, r.n_covered)
