"""Batched form (pss_batch_*): every stream's result equals the plain path
with the same k and p, and the oracle's on streams small enough to replay."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1606_04669_gb300.gen import workloads as W
from tests._helpers import summary_entries

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_04669_gb300 as P  # noqa: E402


def ents(e):
    return list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist()))


def make_streams(width, seed):
    rng = np.random.default_rng(seed)
    lens = [0, 7, 999, 50_000, 123_457, 300_000, 700_001, 2_000_000]
    ks = [2, 64, 256, 1024, 4096, 300]
    specs = []
    for i in range(22):
        specs.append(dict(n=int(lens[i % len(lens)]), k=int(ks[(3 * i) % len(ks)]),
                          s=float(0.8 + 1.2 * rng.random()), stream=i))
    items = [P.gen_zipf(sp["n"], seed=seed, s=sp["s"], log2u=32, item_bytes=width,
                        stream_id=sp["stream"]) for sp in specs]
    return specs, items


@pytest.mark.parametrize("width", [8, 4])
def test_batch_equals_plain_and_oracle(width):
    specs, items = make_streams(width, 3 if width == 8 else 5)
    batch = P.Batch(items, [sp["k"] for sp in specs])
    plan = batch.plan()
    assert plan == [P.plan_blocks(sp["n"], sp["k"], width) for sp in specs]
    batch.run(use_graph=False)
    res = batch.results()
    for i, sp in enumerate(specs):
        plain = P.summarize(items[i], sp["k"], plan[i])
        q = plain.query(sp["n"], sp["k"])
        assert ents(res[i]) == ents(q), i
        e = batch.export(i)
        pe = plain.export()
        assert ents(e) == ents(pe) and (e.m, e.n_covered) == (pe.m, pe.n_covered), i
        if sp["n"] <= 300_000:
            x = oracle.gen_zipf(sp["n"], seed=3 if width == 8 else 5, s=sp["s"], log2u=32,
                                width=width, stream=sp["stream"])
            root, rq = oracle.parallel_space_saving(x, sp["k"], plan[i])
            assert ents(e) == summary_entries(root) and e.m == root.m, i
            assert ents(res[i]) == summary_entries(rq), i
    # the graph form, replayed twice, gives the same results
    for _ in range(2):
        batch.run(use_graph=True)
        res2 = batch.results()
        assert all(ents(a) == ents(b) for a, b in zip(res, res2))
    batch.close()


def test_batch_explicit_plan_and_workload_params():
    specs = W.batched_streams(seed=3, nstreams=16, lo=1e3, hi=3e5)
    items = [P.gen_zipf(sp.n, seed=sp.seed, s=sp.s, log2u=sp.log2u, item_bytes=sp.item_bytes,
                        stream_id=sp.index) for sp in specs]
    ps = [1 + (i % 5) for i in range(len(specs))]
    batch = P.Batch(items, [sp.k for sp in specs], ps=ps)
    assert batch.plan() == ps
    batch.run(use_graph=True)
    res = batch.results()
    for i, sp in enumerate(specs):
        x = oracle.gen_zipf(sp.n, seed=sp.seed, s=sp.s, log2u=sp.log2u, width=8, stream=sp.index)
        root, rq = oracle.parallel_space_saving(x, sp.k, ps[i])
        assert ents(res[i]) == summary_entries(rq), i


@pytest.mark.parametrize("kmax", [0, 64])
def test_batch_kernel_choice_by_skew(kmax):
    # Streams with k <= 256 go to the warp kernel where the skew hint says
    # misses dominate, the others to the CTA kernel (kmax = 0: all CTA);
    # every result against the oracle.
    prev = P.set_warp_kmax(kmax)
    try:
        ks = [64, 128, 256, 64, 128, 256, 2, 100, 1024, 192, 192, 160, 32]
        skews = [0.6, 0.9, 0.5, 2.5, 1.9, 1.2, 1.0, 0.0, 0.8, 1.0, 0.6, 1.2, 1.9]
        items = [P.gen_zipf(60_000 + 1000 * i, seed=11, s=max(sk, 0.7), log2u=20, item_bytes=8,
                            stream_id=i) for i, sk in enumerate(skews)]
        ps = [1 + i % 4 for i in range(len(ks))]
        batch = P.Batch(items, ks, ps=ps, skews=skews)
        batch.run(use_graph=True)
        res = batch.results()
        for i, (k, sk) in enumerate(zip(ks, skews)):
            x = oracle.gen_zipf(60_000 + 1000 * i, seed=11, s=max(sk, 0.7), log2u=20, width=8,
                                stream=i)
            root, rq = oracle.parallel_space_saving(x, k, ps[i])
            e = batch.export(i)
            assert ents(e) == summary_entries(root) and (e.m, e.n_covered) == (root.m, len(x)), i
            assert ents(res[i]) == summary_entries(rq), i
        batch.close()
    finally:
        P.set_warp_kmax(prev)


def _pairs_of(x: np.ndarray) -> int:
    _, c = np.unique(x, return_counts=True)
    return int((c.astype(np.int64) * (c - 1) // 2).sum())


@pytest.mark.parametrize("width", [4, 8])
def test_estimate_skew_counts_pairs_exactly(width):
    # The device count of equal pairs in each stream's first min(n, 4096)
    # items equals a numpy recount of the same prefix; the skew is
    # pss_skew_of_pairs of that count (so a pure function of the bytes).
    xs = [oracle.gen_zipf(n, seed=31, s=s, log2u=32, width=width, stream=i)
          for i, (n, s) in enumerate([(100_000, 0.8), (5000, 1.3), (4096, 2.0), (4095, 1.1),
                                      (37, 3.0), (1, 1.5), (0, 1.5)])]
    dt = np.uint32 if width == 4 else np.uint64
    xs += [np.full(9000, np.iinfo(dt).max, dt), np.arange(9000, dtype=dt)]
    dev = [torch.from_numpy(x.view(np.int32 if width == 4 else np.int64)).cuda() for x in xs]
    skews, pairs = P.estimate_skew(dev)
    for x, sk, pr in zip(xs, skews, pairs):
        S = min(len(x), 4096)
        assert pr == _pairs_of(x[:S])
        assert sk == P.skew_of_pairs(pr, S)
    assert pairs[-2] == 4096 * 4095 // 2 and pairs[-1] == 0
    # the same bytes give the same estimate again
    assert P.estimate_skew(dev) == (skews, pairs)


def test_batch_planned_from_estimated_skew():
    # A batch planned from the estimated skews (block lengths and kernel
    # choice) gives every stream the result of the plain path with the plan's
    # p, and the oracle's.
    from paper_1606_04669_gb300 import autotune
    specs = W.batched_streams(seed=3, nstreams=24, lo=1e3, hi=4e5)
    items = [P.gen_zipf(sp.n, seed=sp.seed, s=sp.s, log2u=sp.log2u, item_bytes=8,
                        stream_id=sp.index) for sp in specs]
    est, _ = P.estimate_skew(items)
    assert all(abs(e - sp.s) < 0.25 for e, sp in zip(est, specs) if sp.n >= 4096)
    ps = [autotune.plan_blocks(sp.n, sp.k, e) for sp, e in zip(specs, est)]
    batch = P.Batch(items, [sp.k for sp in specs], ps=ps, skews=est)
    batch.run(use_graph=True)
    res = batch.results()
    for i, sp in enumerate(specs):
        x = oracle.gen_zipf(sp.n, seed=sp.seed, s=sp.s, log2u=sp.log2u, width=8, stream=sp.index)
        root, rq = oracle.parallel_space_saving(x, sp.k, ps[i])
        e = batch.export(i)
        assert ents(e) == summary_entries(root) and (e.m, e.n_covered) == (root.m, sp.n), i
        assert ents(res[i]) == summary_entries(rq), i
    batch.close()


def test_batch_skews_estimate_option():
    # Batch(skews="estimate") plans from pss_estimate_skew: the same plan as
    # passing the estimates by hand.
    specs = W.batched_streams(seed=3, nstreams=6, lo=1e4, hi=2e5)
    items = [P.gen_zipf(sp.n, seed=sp.seed, s=sp.s, log2u=sp.log2u, item_bytes=8,
                        stream_id=sp.index) for sp in specs]
    ks = [sp.k for sp in specs]
    est, _ = P.estimate_skew(items)
    a = P.Batch(items, ks, skews="estimate")
    b = P.Batch(items, ks, skews=est)
    assert a.plan() == b.plan() and a.skews == est
    a.run()
    b.run()
    assert all(ents(x) == ents(y) for x, y in zip(a.results(), b.results()))
    a.close()
    b.close()
    with pytest.raises(ValueError):
        P.Batch(items, ks, skews="guess")
