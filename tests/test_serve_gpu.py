"""Served form (pss_server_*): every request's two results against the
oracle, and the same results alone and in the mix."""
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


def ents(e):
    return list(zip(e.item.tolist(), e.count.tolist(), e.err.tolist()))


def make_requests(count, tenants, seed=4, span=0.25):
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for i in range(count):
        t += rng.exponential(span / count)
        n = int(np.exp(np.log(1e3) + rng.random() * (np.log(1.2e5) - np.log(1e3))))
        reqs.append(dict(id=1000 + i, arrival=t, tenant=int(rng.integers(0, tenants)), n=n,
                         s=float(1.0 + rng.random()), log2u=24, seed=seed, stream_id=i))
    return reqs


def run_server(reqs, tenants, k, **kw):
    srv = P.Server(tenants, k, **kw)
    srv.submit(reqs)
    srv.start()
    srv.wait(300)
    comps = {c["id"]: c for c in srv.poll()}
    res = {r["id"]: srv.result(r["id"]) for r in reqs}
    tenant_final = {t: srv.tenant_export(t) for t in range(tenants)}
    srv.close()
    return comps, res, tenant_final


def oracle_expectations(reqs, tenants, k):
    """Per request: Pruned(segment) and Pruned(tenant after it), tenant
    summaries combined with Algorithm 2 in arrival order."""
    tenant = {t: oracle.Summary(np.zeros(0, np.uint64), np.zeros(0, np.uint64),
                                np.zeros(0, np.uint64), 0, 0) for t in range(tenants)}
    out = {}
    for r in sorted(reqs, key=lambda r: r["arrival"]):
        x = oracle.gen_zipf(r["n"], seed=r["seed"], s=r["s"], log2u=r["log2u"], stream=r["stream_id"])
        p = P.plan_blocks(r["n"], k, 4, r["s"])
        seg, segq = oracle.parallel_space_saving(x, k, p)
        tenant[r["tenant"]] = oracle.combine(tenant[r["tenant"]], seg, k)
        tq = oracle.query(tenant[r["tenant"]], tenant[r["tenant"]].n_covered, k)
        out[r["id"]] = (segq, tq, tenant[r["tenant"]].n_covered)
    return out, tenant


def test_served_results_match_oracle_and_are_mix_independent():
    tenants, k = 6, 64
    reqs = make_requests(160, tenants)
    comps, res, final = run_server(reqs, tenants, k, budget_bytes=64 << 20, max_batch=12)
    assert len(comps) == len(reqs)
    expect, tenant_ref = oracle_expectations(reqs, tenants, k)
    for r in reqs:
        c = comps[r["id"]]
        assert c["status"] == 0
        assert c["admitted"] >= c["arrival"] - 1e-9 and c["completed"] >= c["admitted"]
        segq, tq, ncum = expect[r["id"]]
        got_seg, got_ten = res[r["id"]]
        assert ents(got_seg) == summary_entries(segq), r["id"]
        assert ents(got_ten) == summary_entries(tq), r["id"]
        assert c["tenant_items"] == ncum
    for t in range(tenants):
        assert ents(final[t]) == summary_entries(tenant_ref[t])
        assert (final[t].m, final[t].n_covered) == (tenant_ref[t].m, tenant_ref[t].n_covered)
    # alone: one tenant's requests through their own server give the same results
    alone = [r for r in reqs if r["tenant"] == 2]
    comps2, res2, _ = run_server(alone, tenants, k, budget_bytes=1 << 30, max_batch=1)
    for r in alone:
        assert ents(res2[r["id"]][0]) == ents(res[r["id"]][0])
        assert ents(res2[r["id"]][1]) == ents(res[r["id"]][1])


def test_served_tiny_budget_and_caller_segments():
    # a budget below a single request still serves (one request at a time);
    # caller-provided segments use the same path
    tenants, k = 3, 32
    reqs = make_requests(24, tenants, seed=9, span=0.02)
    for r in reqs[::3]:
        x = oracle.gen_zipf(r["n"], seed=r["seed"], s=r["s"], log2u=r["log2u"], stream=r["stream_id"])
        r["items"] = torch.from_numpy(x.view(np.int32)).cuda()
    comps, res, _ = run_server(reqs, tenants, k, budget_bytes=1024, max_batch=4)
    expect, _ = oracle_expectations(reqs, tenants, k)
    for r in reqs:
        assert comps[r["id"]]["status"] == 0
        segq, tq, _ = expect[r["id"]]
        assert ents(res[r["id"]][0]) == summary_entries(segq)
        assert ents(res[r["id"]][1]) == summary_entries(tq)


def test_served_duplicate_ids_rejected():
    srv = P.Server(2, 32, budget_bytes=64 << 20, max_batch=4)
    reqs = make_requests(4, 2, seed=5, span=0.01)
    srv.submit(reqs[:2])
    for bad in ([reqs[1]], [reqs[2], dict(reqs[2])]):  # a live id; a repeat inside one call
        with pytest.raises(P.PssError) as ei:
            srv.submit(bad)
        assert ei.value.code == P.PSS_EINVAL
    srv.start()
    srv.wait(120)
    for r in reqs[:2]:
        srv.result(r["id"])
    srv.submit([dict(reqs[0], arrival=0.0)])  # read back: its id is free again
    srv.wait(120)
    srv.close()


def test_served_injected_allocation_failures():
    # Host-side fault injection: three segment allocations fail.  Those
    # requests complete with PSS_ENOMEM and leave their tenants untouched;
    # everything else equals a run of the trace without them.
    tenants, k = 4, 48
    reqs = make_requests(60, tenants, seed=7)
    srv = P.Server(tenants, k, budget_bytes=64 << 20, max_batch=6)
    srv.inject_alloc_failures(3)
    srv.submit(reqs)
    srv.start()
    srv.wait(300)
    comps = {c["id"]: c for c in srv.poll()}
    assert len(comps) == len(reqs)
    failed = {i for i, c in comps.items() if c["status"] != 0}
    assert len(failed) == 3 and all(comps[i]["status"] == P.PSS_ENOMEM for i in failed)
    res = {r["id"]: srv.result(r["id"]) for r in reqs if r["id"] not in failed}
    final = {t: srv.tenant_export(t) for t in range(tenants)}
    srv.close()
    rest = [r for r in reqs if r["id"] not in failed]
    _, res2, final2 = run_server(rest, tenants, k, budget_bytes=64 << 20, max_batch=6)
    for r in rest:
        assert ents(res[r["id"]][0]) == ents(res2[r["id"]][0]), r["id"]
        assert ents(res[r["id"]][1]) == ents(res2[r["id"]][1]), r["id"]
    for t in range(tenants):
        assert ents(final[t]) == ents(final2[t])


def test_frequent_server_matches_oracle():
    # pss_frequent_server_create: segments summarized by the Frequent batch,
    # merged into their tenant with the Frequent merge in arrival order
    tenants, k = 5, 48
    reqs = make_requests(120, tenants, seed=12)
    srv = P.Server(tenants, k, budget_bytes=64 << 20, max_batch=10, frequent=True)
    assert srv.kind == P.KIND_FREQUENT
    srv.submit(reqs)
    srv.start()
    srv.wait(300)
    comps = {c["id"]: c for c in srv.poll()}
    res = {r["id"]: srv.result(r["id"]) for r in reqs}
    final = {t: srv.tenant_export(t) for t in range(tenants)}
    srv.close()
    empty = np.zeros(0, np.uint64)
    tenant = {t: oracle.Summary(empty, empty, empty, 0, 0) for t in range(tenants)}
    for r in sorted(reqs, key=lambda r: r["arrival"]):
        x = oracle.gen_zipf(r["n"], seed=r["seed"], s=r["s"], log2u=r["log2u"], stream=r["stream_id"])
        p = P.plan_blocks(r["n"], k, 4, r["s"], frequent=True)
        seg, segq = oracle.parallel_frequent(x, k, p)
        tenant[r["tenant"]] = oracle.frequent_combine(tenant[r["tenant"]], seg, k)
        tn = tenant[r["tenant"]]
        tq = oracle.frequent_query(tn, tn.n_covered, k)
        c = comps[r["id"]]
        assert c["status"] == 0 and c["tenant_items"] == tn.n_covered
        got_seg, got_ten = res[r["id"]]
        assert ents(got_seg) == ents(segq), r["id"]
        assert ents(got_ten) == ents(tq), r["id"]
    for t in range(tenants):
        assert ents(final[t]) == ents(tenant[t])
        assert (final[t].m, final[t].n_covered) == (oracle.frequent_delta(tenant[t], k),
                                                    tenant[t].n_covered)


def test_wait_expires_before_start_then_completes():
    """The bounded wait: before the scheduler starts nothing completes, so a
    short wait returns PSS_ETIMEOUT; the server is still usable afterwards."""
    tenants, k = 2, 64
    reqs = make_requests(6, tenants, seed=9)
    srv = P.Server(tenants, k, budget_bytes=64 << 20, max_batch=4)
    try:
        srv.submit(reqs)
        with pytest.raises(P.PssError) as e:
            srv.wait(0.2)
        assert e.value.code == P.pss.PSS_ETIMEOUT
        assert srv.poll() == []
        srv.start()
        srv.wait(300)
        comps = {c["id"]: c for c in srv.poll()}
        res = {r["id"]: srv.result(r["id"]) for r in reqs}
    finally:
        srv.close()
    assert sorted(comps) == sorted(r["id"] for r in reqs)
    expect, _ = oracle_expectations(reqs, tenants, k)
    for r in reqs:
        assert comps[r["id"]]["status"] == 0
        segq, tq, _ = expect[r["id"]]
        got_seg, got_ten = res[r["id"]]
        assert ents(got_seg) == summary_entries(segq)
        assert ents(got_ten) == summary_entries(tq)
