"""Exact counts, the guaranteed query and the accuracy metrics (Section 4) on
the GPU against the oracle: counts and every integer field bit-exact, ARE
within 1e-12 relative (a sum of at most k fp64 quotients in another order)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests._helpers import summary_entries

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_04669_gb300 as P  # noqa: E402

INT_FIELDS = ("reported", "true_frequent", "true_positive", "guaranteed", "outside")


def to_dev(x):
    return torch.from_numpy(x.view(np.int32 if x.dtype == np.uint32 else np.int64)).cuda()


def ents(e):
    return list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist()))


def test_exact_counts_match_oracle():
    for w, log2u in ((4, 20), (8, 16), (4, 1)):
        x = oracle.gen_zipf(300_000, seed=60 + log2u, s=1.2, log2u=20, width=w)
        got = P.exact_counts(to_dev(x), log2u).cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got, oracle.exact_counts(x, log2u)), (w, log2u)
    e = P.exact_counts(torch.zeros(0, dtype=torch.int32, device="cuda"), 5)
    assert int(e.sum()) == 0


@pytest.mark.parametrize("n,k,p,w,s,log2u,seed", [
    (1 << 20, 100, 8, 4, 1.1, 20, 1),       # the small plain configuration
    (200_000, 500, 5, 4, 0.8, 18, 71),
    (150_000, 64, 3, 8, 1.5, 16, 72),       # warp-per-block summaries
    (100_000, 2000, 4, 4, 1.2, 20, 73),
    (90_000, 7, 1, 4, 2.5, 12, 74),
])
def test_accuracy_and_guaranteed_match_oracle(n, k, p, w, s, log2u, seed):
    x = oracle.gen_zipf(n, seed=seed, s=s, log2u=log2u, width=w)
    xd = to_dev(x)
    sm = P.summarize(xd, k, p)
    root, _ = oracle.parallel_space_saving(x, k, p)
    counts = P.exact_counts(xd, log2u)
    got = sm.accuracy(counts, log2u, n, k)
    ref = oracle.accuracy(root, oracle.exact_counts(x, log2u), n, k)
    for f in INT_FIELDS:
        assert got[f] == ref[f], f
    assert got["are"] == pytest.approx(ref["are"], rel=1e-12, abs=1e-300)
    assert got["precision"] == ref["precision"] and got["recall"] == ref["recall"] == 1.0
    g = sm.query(n, k, guaranteed=True)
    assert ents(g) == summary_entries(oracle.query_guaranteed(root, n, k))
    sm.close()


def test_accuracy_at_the_2p30_shape():
    # n = 2^30 u32 Zipf(1.1) over [0, 2^24), k = 2000, p = 4096: the device
    # metrics against the same metrics from torch's histogram on the host.
    n, k, p, log2u = 1 << 30, 2000, 4096, 24
    x = P.gen_zipf(n, seed=2, s=1.1, log2u=log2u)
    sm = P.summarize(x, k, p)
    counts = P.exact_counts(x, log2u)
    got = sm.accuracy(counts, log2u, n, k)
    f = torch.bincount(x.view(torch.int32).to(torch.int64), minlength=1 << log2u).cpu().numpy()
    assert np.array_equal(counts[:-1].cpu().numpy().view(np.uint32).astype(np.int64), f)
    q = sm.query(n, k)
    fq = f[q.item.astype(np.int64)]
    assert got["reported"] == q.size
    assert got["true_frequent"] == int((f * k > n).sum())
    assert got["true_positive"] == int((fq * k > n).sum())
    assert got["recall"] == 1.0
    are = float(np.mean(np.abs(q.count.astype(np.float64) - fq) / fq))
    assert got["are"] == pytest.approx(are, rel=1e-12)
    sm.close()
