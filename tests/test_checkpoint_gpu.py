"""Checkpoint and resume: a canonical summary plus the length it covers is a
complete state (summaries are mergeable, Algorithm 2).  Export -> import
round trips bit for bit, merging an imported summary equals merging the
original, and a server resumed from exported tenants gives every later
request and every tenant exactly what one uninterrupted server gives."""
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
from tests.test_serve_gpu import make_requests  # noqa: E402


def ents(e):
    return list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist()))


def to_dev(x):
    return torch.from_numpy(x.view(np.int32 if x.dtype == np.uint32 else np.int64)).cuda()


@pytest.mark.parametrize("k,w", [(64, 4), (1000, 8), (6000, 4)])
def test_export_import_round_trip_and_merge(k, w):
    xa = oracle.gen_zipf(200_000, seed=81, s=1.0, log2u=20, width=w)
    xb = oracle.gen_zipf(150_000, seed=82, s=1.3, log2u=20, width=w)
    a = P.summarize(to_dev(xa), k, 4)
    b = P.summarize(to_dev(xb), k, 3)
    ea = a.export()
    ia = P.import_summary(ea, k, w)
    ei = ia.export()
    assert ents(ei) == ents(ea) and (ei.m, ei.n_covered) == (ea.m, ea.n_covered)
    assert ents(P.merge(ia, b).export()) == ents(P.merge(a, b).export())
    q = ia.query(ea.n_covered, k)
    ra, rq = oracle.parallel_space_saving(xa, k, 4)
    assert ents(q) == summary_entries(rq)


@pytest.mark.parametrize("k,w", [(64, 4), (1000, 8), (4096, 4)])
def test_frequent_export_import_round_trip_and_merge(k, w):
    xa = oracle.gen_zipf(200_000, seed=84, s=1.0, log2u=20, width=w)
    xb = oracle.gen_zipf(150_000, seed=85, s=1.3, log2u=20, width=w)
    a = P.frequent(to_dev(xa), k, 4)
    b = P.frequent(to_dev(xb), k, 3)
    ea = a.export()
    ia = P.import_summary(ea, k, w, frequent=True)
    assert ia.kind == P.KIND_FREQUENT
    ei = ia.export()
    assert ents(ei) == ents(ea) and (ei.m, ei.n_covered) == (ea.m, ea.n_covered)
    assert ents(P.merge(ia, b).export()) == ents(P.merge(a, b).export())
    ra, rq = oracle.parallel_frequent(xa, k, 4)
    assert ents(ia.query(ea.n_covered, k)) == ents(rq)
    with pytest.raises(P.PssError) as er:
        P.import_summary(ea, ea.size, w, frequent=True)  # k - 1 < entries
    assert er.value.code == P.PSS_EINVAL


def test_import_rejects_bad_checkpoints():
    x = oracle.gen_zipf(50_000, seed=83, s=1.1, log2u=16)
    e = P.summarize(to_dev(x), 32, 2).export()
    dup = P.Exported(np.concatenate([e.item[:2], e.item[:1]]), np.concatenate([e.count[:3]]),
                     np.concatenate([e.err[:3]]), e.m, e.n_covered)
    for bad, k, w in ((dup, 32, 4), (e, 16, 4)):   # a duplicate item; more entries than k
        with pytest.raises(P.PssError) as ei:
            P.import_summary(bad, k, w)
        assert ei.value.code == P.PSS_EINVAL
    wide = P.Exported(np.array([1 << 40], np.uint64), np.array([5], np.uint64),
                      np.array([0], np.uint64), 0, 5)
    with pytest.raises(P.PssError):
        P.import_summary(wide, 32, 4)   # a 4-byte summary cannot hold a 41-bit item
    assert ents(P.import_summary(wide, 32, 8).export()) == [(1 << 40, 5, 0)]


def run(reqs, tenants, k, start_from=None, frequent=False):
    srv = P.Server(tenants, k, budget_bytes=64 << 20, max_batch=8, frequent=frequent)
    if start_from:
        for t, ex in start_from.items():
            srv.tenant_import(t, ex)
    srv.submit(reqs)
    srv.start()
    srv.wait(300)
    res = {r["id"]: srv.result(r["id"]) for r in reqs}
    comps = {c["id"]: c for c in srv.poll()}
    final = {t: srv.tenant_export(t) for t in range(tenants)}
    if start_from is None:
        with pytest.raises(P.PssError):
            srv.tenant_import(0, final[0])  # only before start
    srv.close()
    return res, comps, final


@pytest.mark.parametrize("frequent", [False, True])
def test_server_resume_equals_uninterrupted_run(frequent):
    tenants, k = 5, 64
    reqs = sorted(make_requests(120, tenants, seed=12), key=lambda r: r["arrival"])
    first, second = reqs[:50], reqs[50:]
    res_all, comps_all, final_all = run(reqs, tenants, k, frequent=frequent)
    _, _, ckpt = run(first, tenants, k, frequent=frequent)
    shift = second[0]["arrival"]
    resumed = [dict(r, arrival=r["arrival"] - shift) for r in second]
    res2, comps2, final2 = run(resumed, tenants, k, start_from=ckpt, frequent=frequent)
    for r in second:
        assert ents(res2[r["id"]][0]) == ents(res_all[r["id"]][0]), r["id"]
        assert ents(res2[r["id"]][1]) == ents(res_all[r["id"]][1]), r["id"]
        assert comps2[r["id"]]["tenant_items"] == comps_all[r["id"]]["tenant_items"]
    for t in range(tenants):
        assert ents(final2[t]) == ents(final_all[t])
        assert (final2[t].m, final2[t].n_covered) == (final_all[t].m, final_all[t].n_covered)
