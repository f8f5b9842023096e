"""Frequent (Misra–Gries) path on the GPU vs the CPU oracle, through the C ABI
(bit-exact: integer work).  Every block summary, every node of every merge
level, the root with its delta and both queries are compared entry by entry."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests._helpers import canonical

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_04669_gb300 as P  # noqa: E402


def to_dev(x: np.ndarray):
    if x.dtype == np.uint32:
        return torch.from_numpy(x.view(np.int32)).cuda()
    return torch.from_numpy(x.view(np.int64)).cuda()


def ents(s):
    return list(zip(s.item.tolist(), s.count.tolist(), s.err.tolist()))


def compare_frequent(x: np.ndarray, k: int, p: int):
    tree = P.frequent_tree(to_dev(x), k, p)
    assert tree.kind == P.KIND_FREQUENT
    ref = oracle.frequent_tree(x, k, p)
    assert tree.levels == len(ref)
    for lv, ref_level in enumerate(ref):
        got = tree.read_level(lv)
        assert len(got) == len(ref_level)
        for j, (g, r) in enumerate(zip(got, ref_level)):
            it, ct, er, m, cov = g
            items = it.tolist()
            assert items == sorted(items), f"level {lv} node {j}: device layout not item-sorted"
            assert len(items) <= k - 1
            assert canonical(list(zip(items, ct.tolist(), er.tolist()))) == ents(r), \
                f"level {lv} node {j}"
            assert (m, cov) == (0, r.n_covered), f"level {lv} node {j}"
    root = tree.root()
    assert root.kind == P.KIND_FREQUENT
    r = ref[-1][0]
    e = root.export()
    assert ents(e) == ents(r)
    assert (e.m, e.n_covered) == (oracle.frequent_delta(r, k), r.n_covered)
    n = len(x)
    for g in (False, True):
        q = root.query(n, k, guaranteed=g)
        assert ents(q) == ents(oracle.frequent_query(r, n, k, guaranteed=g))
    tree.close()
    s = P.frequent(to_dev(x), k, p)
    assert ents(s.export()) == ents(r)
    return s, r


@pytest.mark.parametrize("n,k,p,w,s,log2u,seed", [
    (60_000, 2, 5, 4, 1.1, 8, 301),          # one counter: the majority vote
    (50_000, 3, 4, 4, 1.2, 10, 302),
    (123_457, 64, 13, 4, 0.8, 20, 303),      # odd p: carried nodes
    (200_000, 500, 5, 4, 1.5, 32, 304),
    (300_000, 1000, 3, 4, 1.0, 32, 305),
    (100_000, 2000, 8, 8, 1.2, 32, 306),     # u64 items
    (80_000, 4096, 2, 4, 0.9, 24, 307),      # the largest k
    (80_000, 4096, 3, 8, 1.3, 40, 308),
    (70_000, 333, 31, 4, 0.5, 32, 309),      # nearly every item a decrement
    (150_000, 1024, 1, 8, 2.0, 32, 310),     # p = 1: plain sequential Misra-Gries
    (262_144, 2000, 1, 4, 1.1, 24, 2),       # one block of the 2^30 stream's shape
    (400_000, 100, 64, 4, 1.1, 20, 311),     # many merge levels
])
def test_random_configs(n, k, p, w, s, log2u, seed):
    x = oracle.gen_zipf(n, seed=seed, s=s, log2u=log2u, width=w)
    compare_frequent(x, k, p)


def test_edge_cases():
    compare_frequent(np.zeros(0, np.uint32), 5, 4)                       # n = 0
    compare_frequent(np.array([7, 7, 9], np.uint32), 4, 8)               # n < p: empty blocks
    compare_frequent(np.array([1, 2, 1, 3, 4, 1, 2, 2], np.uint32), 3, 1)  # the golden stream
    compare_frequent(np.full(100_000, 0xFFFFFFFF, np.uint32), 10, 7)     # sentinel-valued item
    compare_frequent(np.full(5000, np.uint64(2 ** 64 - 1)), 3, 2)
    compare_frequent(np.arange(100_000, dtype=np.uint32) * np.uint32(2654435761), 100, 4)
    # items that collide in weak hashes, and periodic streams (decrements
    # that free many counters at once)
    base = (np.arange(3000, dtype=np.uint64) << np.uint64(20)).astype(np.uint32)
    rng = np.random.default_rng(5)
    compare_frequent(base[rng.zipf(1.3, size=200_000) % 3000], 512, 4)
    compare_frequent(np.tile(np.arange(300, dtype=np.uint32), 800), 256, 2)
    compare_frequent(np.tile(np.arange(31, dtype=np.uint32), 2000), 32, 3)


def test_small_universes_fuzz():
    rng = np.random.default_rng(99)
    for t in range(40):
        w = 4 if t % 2 else 8
        u = int(rng.integers(1, 200))
        n = int(rng.integers(0, 20_000))
        x = rng.integers(0, u, n).astype(np.uint32 if w == 4 else np.uint64)
        k = int(rng.integers(2, 300))
        p = int(rng.integers(1, 12))
        compare_frequent(x, k, p)


def test_merge_api_and_kind_checks():
    xa = oracle.gen_zipf(200_000, seed=7, s=1.1, log2u=20)
    xb = oracle.gen_zipf(150_000, seed=8, s=1.3, log2u=20)
    k = 300
    a, b = P.frequent(to_dev(xa), k, 4), P.frequent(to_dev(xb), k, 3)
    ra = oracle.frequent_tree(xa, k, 4)[-1][0]
    rb = oracle.frequent_tree(xb, k, 3)[-1][0]
    for c in (P.merge(a, b), P.merge(b, a)):
        r = oracle.frequent_combine(ra, rb, k)
        e = c.export()
        assert ents(e) == ents(r)
        assert (e.m, e.n_covered) == (oracle.frequent_delta(r, k), r.n_covered)
    ss = P.summarize(to_dev(xa), k, 4)
    with pytest.raises(P.PssError) as ei:
        P.merge(a, ss)
    assert ei.value.code == P.PSS_EMISMATCH
    # accuracy with the Frequent bounds, against the oracle's query and exact counts
    counts = P.exact_counts(to_dev(xa), 20)
    acc = a.accuracy(counts, 20, len(xa), k)
    n = len(xa)
    f = np.bincount(xa.astype(np.int64), minlength=1 << 20)
    q = oracle.frequent_query(ra, n, k)
    fq = f[q.item.astype(np.int64)]
    cq = q.count.astype(np.int64)
    assert acc["reported"] == q.size
    assert acc["true_frequent"] == int((f * k > n).sum())
    assert acc["true_positive"] == int((fq * k > n).sum())
    assert acc["guaranteed"] == int((cq * k > n).sum())
    assert abs(acc["are"] - float(np.mean(np.abs(fq - cq) / fq))) < 1e-12
    assert acc["recall"] == 1.0
    with pytest.raises(P.PssError) as ei:
        P.frequent(to_dev(xa), 4097, 4)
    assert ei.value.code == P.PSS_EINVAL
    with pytest.raises(P.PssError) as ei:
        P.frequent(to_dev(xa), 1, 4)
    assert ei.value.code == P.PSS_EINVAL


def test_full_size_sampled_blocks_and_bounds():
    # n = 2^28 u32 Zipf(1.1) over [0, 2^24), k = 2000, p = 1024 (the block shape of
    # the 2^30 workload): sampled block summaries against the oracle, and the
    # root's bounds against exact counts taken on the device.
    n, k, p, log2u = 1 << 28, 2000, 1024, 24
    x = P.gen_zipf(n, seed=2, s=1.1, log2u=log2u)
    tree = P.frequent_tree(x, k, p)
    level0 = tree.read_level(0)
    xs = x.cpu().numpy().view(np.uint32)
    for r in (0, 1, 511, 1023):
        lo, hi = oracle.block_bounds(n, p, r)
        ref = oracle.frequent(xs[lo:hi], k)
        it, ct, er, m, cov = level0[r]
        assert canonical(list(zip(it.tolist(), ct.tolist(), er.tolist()))) == ents(ref)
        assert cov == hi - lo
    root = tree.root()
    e = root.export()
    delta = e.m
    f = P.exact_counts(x, log2u).cpu().numpy().view(np.uint32).astype(np.int64)
    stored = dict(zip(e.item.tolist(), e.count.tolist()))
    assert len(stored) <= k - 1
    for item, c in stored.items():
        assert c <= f[item] <= c + delta
    mask = np.ones(1 << log2u, bool)
    mask[list(stored)] = False
    assert int(f[:-1][mask].max(initial=0)) <= delta
    frequent_items = set(np.nonzero(f[:-1] * k > n)[0].tolist())
    assert frequent_items <= set(root.query(n, k).item.tolist())
    tree.close()


@pytest.mark.parametrize("width", [8, 4])
def test_frequent_batch_equals_plain_and_oracle(width):
    # pss_frequent_batch_create: every stream's query and root equal the plain
    # Frequent path with the batch's block count, and the oracle's
    rng = np.random.default_rng(40 + width)
    lens = [0, 7, 999, 50_000, 123_457, 300_000, 700_001]
    ks = [2, 64, 256, 1024, 4096, 300, 3]
    specs = [dict(n=lens[i % len(lens)], k=ks[(3 * i) % len(ks)], s=float(0.8 + 1.2 * rng.random()),
                  stream=i) for i in range(18)]
    items = [P.gen_zipf(sp["n"], seed=7, s=sp["s"], log2u=32, item_bytes=width,
                        stream_id=sp["stream"]) for sp in specs]
    batch = P.Batch(items, [sp["k"] for sp in specs], frequent=True)
    assert batch.kind == P.KIND_FREQUENT
    plan = batch.plan()
    for use_graph in (False, True, True):
        batch.run(use_graph=use_graph)
        res = batch.results()
        for i, sp in enumerate(specs):
            n, k = sp["n"], sp["k"]
            plain = P.frequent(items[i], k, plan[i])
            assert ents(res[i]) == ents(plain.query(n, k)), i
            e, pe = batch.export(i), plain.export()
            assert ents(e) == ents(pe) and (e.m, e.n_covered) == (pe.m, pe.n_covered), i
            if use_graph is False and n <= 300_000:
                x = oracle.gen_zipf(n, seed=7, s=sp["s"], log2u=32, width=width, stream=sp["stream"])
                root, cand = oracle.parallel_frequent(x, k, plan[i])
                assert ents(e) == ents(root) and e.m == oracle.frequent_delta(root, k), i
                assert ents(res[i]) == ents(cand), i
    batch.close()


@pytest.mark.parametrize("direct,pinned", [(True, True), (False, True), (True, False)])
def test_frequent_host_input(direct, pinned):
    # mapped pinned memory read in place, pinned memory staged, pageable memory staged
    x = oracle.gen_zipf(700_001, seed=61, s=1.1, log2u=20, width=8)
    h = torch.from_numpy(x.view(np.int64))
    if pinned:
        h = h.pin_memory()
    prev = P.set_host_direct(direct)
    try:
        s = P.frequent_host(h, 300, 19)
        e = s.export()
        torch.cuda.synchronize()
    finally:
        P.set_host_direct(prev)
    root, q = oracle.parallel_frequent(x, 300, 19)
    assert s.kind == P.KIND_FREQUENT
    assert ents(e) == ents(root)
    assert (e.m, e.n_covered) == (oracle.frequent_delta(root, 300), root.n_covered)
    assert ents(s.query(len(x), 300)) == ents(q)
