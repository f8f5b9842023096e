#!/usr/bin/env python3
"""Benchmark of the Parallel Space Saving hot path on GB300: one JSON line.

A step is one pass of the whole path over the workload: the p block
summaries (Space Saving, Section 3), the binary combine tree (Algorithm 2)
and the k-majority query with its result read back to the host (Algorithm 1).

Default workload (the configuration the headline metric is quoted on):
n = 2^30 uint32 items drawn i.i.d. from Zipf(s = 1.1) over [0, 2^24), seed 2,
k = 2000 counters, p = 4096 equal blocks, binary merge tree, threshold n/k.
The 4 GiB input is larger than L2 (129 MB), so no flush is needed between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

On one GPU the default line also carries a `batched` object (1024 uint64
streams in one graph launch against the plain path looped over them) and a
`served` object (60 s of open-loop Poisson arrivals, p50/p99 latency), the
other two forms the metric compares (--no-batched / --no-served leave them
out; --workload batched / served print their full lines).

With --gpus N > 1 (launched by torchrun) every rank runs an independent
replica on its own GPU (the path is replicated, not sharded) and the value is
the items of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "items/s & input GB/s (% HBM peak), plain vs batched/served; p50/p99 latency"

WORKLOADS = {
    "plain": dict(
        desc="plain single stream: n=2^30 uint32 Zipf(s=1.1) over [0,2^24), seed 2; k=2000; "
             "p=4096 equal blocks; binary merge tree; query n/k",
        n=1 << 30, w=4, s=1.1, log2u=24, seed=2, k=2000, p=4096),
    "wave": dict(
        desc="one wave of the plain workload's blocks: n=304*262144 uint32 Zipf(s=1.1) over "
             "[0,2^24), seed 2; k=2000; p=304 blocks of 262144 items (the block shape of the "
             "2^30 stream); binary merge tree; query n/k",
        n=304 * 262144, w=4, s=1.1, log2u=24, seed=2, k=2000, p=304),
    "wave_k500": dict(
        desc="one wave of narrow-shape blocks: n=608*262144 uint32 Zipf(s=1.0) over [0,2^32), "
             "seed 2; k=500; p=608 blocks of 262144 items (4 CTAs of 256 threads on each of 152 "
             "SMs); binary merge tree; query n/k",
        n=608 * 262144, w=4, s=1.0, log2u=32, seed=2, k=500, p=608),
    "frequent_wave": dict(
        desc="one wave of Frequent warps at k=2000: n=1368*262144 uint32 Zipf(s=1.1) over "
             "[0,2^24), seed 2; p=1368 blocks of 262144 items (9 warps on each of 152 SMs)",
        n=1368 * 262144, w=4, s=1.1, log2u=24, seed=2, k=2000, p=1368),
    "round_k256": dict(
        desc="round-kernel shape: n=2^28 uint32 Zipf(s=1.0) over [0,2^32), seed 13; k=256; "
             "p=8192 blocks of 32768 items (one warp per block); binary merge tree; query n/k",
        n=1 << 28, w=4, s=1.0, log2u=32, seed=13, k=256, p=8192),
    "warp_k64": dict(
        desc="warp-kernel shape: n=2^27 uint32 Zipf(s=1.1) over [0,2^24), seed 2; k=64; "
             "p=4096 blocks of 32768 items (one warp per block, counters in registers); binary "
             "merge tree; query n/k",
        n=1 << 27, w=4, s=1.1, log2u=24, seed=2, k=64, p=4096),
    "small": dict(
        desc="plain single stream: n=2^20 uint32 Zipf(s=1.1) over [0,2^20), seed 1; k=100; p=8; "
             "binary merge tree; query n/k",
        n=1 << 20, w=4, s=1.1, log2u=20, seed=1, k=100, p=8),
}


# DRAM traffic of each block-summary kernel from one ncu capture of it, valid
# only for the kernel source it was measured on (the sha1 of that file) and the
# block shape it was measured at.  Traffic grows with the number of blocks, so
# a launch of p such blocks moves p times the per-block bytes.
#   ss_block_kernel: profiles/ss_block_kernel_wave_k2000.md, 304 blocks of
#     262144 u32 items, k = 2000 -> 319.19 MB read + 3.02 MB written.
#   ssr_block_kernel: profiles/ssr_block_kernel_k256.md, 8192 blocks of 32768
#     u32 items, k = 256 -> 1077.7 MB read + 32.5 MB written.
#   frequent_block_kernel: profiles/frequent_block_kernel_wave_k2000.md, 1368
#     blocks of 262144 u32 items, k = 2000 -> 1434.60 MB read + 3.76 MB written.
TRAFFIC = {
    "ss_block_kernel": {"src": "summarize.cu",
                        "sha1": "958f8314d26b6998cc5b8c223972a560bd33cbad",
                        "bytes_per_block": (319.187e6 + 3.016e6) / 304, "block_items": 262144,
                        "k": 2000, "w": 4},
    "ssr_block_kernel": {"src": "summarize_round.cu",
                         "sha1": "0e210092b09dbb8f0a1656928b774624097af347",
                         "bytes_per_block": (1077.7e6 + 32.5e6) / 8192, "block_items": 32768,
                         "k": 256, "w": 4},
    "frequent_block_kernel": {"src": "frequent.cu",
                              "sha1": "b2f35211bbd44917466a2c57c50e8e0958cfcd08",
                              "bytes_per_block": (1434.60e6 + 3.76e6) / 1368,
                              "block_items": 262144, "k": 2000, "w": 4},
}


def traffic_per_launch(kernel, n, k, p, w):
    """Measured DRAM bytes of one launch of `kernel` over p blocks of n/p
    items, or None when no capture matches this source and block shape."""
    import hashlib
    t = TRAFFIC.get(kernel)
    if t is None:
        return None
    src = os.path.join(ROOT, "paper_1606_04669_gb300", "csrc", t["src"])
    try:
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if sha != t["sha1"] or k != t["k"] or w != t["w"] or n // p != t["block_items"]:
        return None
    return t["bytes_per_block"] * p


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_info() -> dict:
    """The host the oracle runs on: logical CPUs and the CPU model."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                if key in ("model name", "hardware", "cpu model") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu_model": model or "unknown"}


def replica_aggregate(local_ms: float, local_items: int, dist=None, device="cpu"):
    """Whole-job figures of N independent replicas: the slowest rank's time
    and the items of all ranks (value = items / time).  With dist=None (one
    GPU) the local figures are returned."""
    if dist is None:
        return local_ms, local_items
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([local_items], dtype=torch.int64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(wl, budget_s: float, seed_offset: int = 0):
    """The oracle, single-threaded on a host core, over the first B blocks of
    the workload (block summaries + their combine tree + query); B is sized so
    the oracle works about budget_s seconds.  Input generation (threaded) is
    not timed."""
    import oracle
    n, k, p, w = wl["n"], wl["k"], wl["p"], wl["w"]
    threads = os.cpu_count() or 1
    lo0, hi0 = oracle.block_bounds(n, p, 0)
    x0 = oracle.gen_zipf(hi0 - lo0, seed=wl["seed"], s=wl["s"], log2u=wl["log2u"], width=w,
                         stream=seed_offset, threads=threads)
    t = time.perf_counter()
    oracle.space_saving(x0, k)
    per_block = max(time.perf_counter() - t, 1e-6)
    blocks = int(max(2, min(p, budget_s / per_block)))
    hi = oracle.block_bounds(n, p, blocks - 1)[1]
    x = oracle.gen_zipf(hi, seed=wl["seed"], s=wl["s"], log2u=wl["log2u"], width=w,
                        stream=seed_offset, threads=threads)
    t = time.perf_counter()
    levels = oracle.pss_tree(x, k, blocks)
    oracle.query(levels[-1][0], hi, k)
    dt = time.perf_counter() - t
    return {"value": hi / dt, "unit": "items/s", "cores": 1, "kind": "oracle",
            "sample": f"blocks 0..{blocks - 1} of the {p} blocks ({hi} items): block summaries, "
                      f"their binary combine tree and the query, single-threaded C++",
            "seconds": dt, "host": host_info()}


def workload_config(wl, world: int = 1) -> dict:
    """The `config` object of the plain workloads' lines (both arms)."""
    n, w = wl["n"], wl["w"]
    return {"workload": wl["desc"], "n": n, "k": wl["k"], "p": wl["p"], "item_bytes": w,
            "zipf_s": wl["s"], "universe": f"2^{wl['log2u']}", "seed": wl["seed"],
            "l2": (f"input ({n * w / 2**30:.2f} GiB) larger than L2; no flush"
                   if n * w > (256 << 20) else "input smaller than L2"),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def batched_summary(b: dict) -> dict:
    """The batched form's object on the default line."""
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "input_gbs", "hbm_frac",
            "batched_over_plain", "results_identical", "hinted", "skew_estimate",
            "gpu_launches_per_step")
    out = {key: b[key] for key in keep}
    out["plain_loop_value"] = b["plain_loop"]["value"]
    out["config"] = {key: b["config"][key] for key in ("streams", "total_items", "item_bytes",
                                                         "k_classes", "blocks", "seed")}
    out["workload"] = ("batched: 1024 uint64 streams, lengths log-uniform [1e4, 1e8], Zipf s "
                       "U[0.8, 2] over [0, 2^32), k in {64, 256, 1024, 4096}, seed 3; one graph "
                       "launch per step against the plain path looped over the streams")
    return out


def served_summary(v: dict) -> dict:
    """The served form's object on the default line."""
    keep = ("value", "unit", "latency_ms", "requests", "errors", "offered_items_per_s",
            "generator_items_per_s", "makespan_s", "gpu_launches", "clocks")
    out = {key: v[key] for key in keep}
    out["config"] = v["config"]
    out["workload"] = ("served: open-loop Poisson 2000 req/s, segments log-uniform [1e4, 1e7] "
                       "uint32, Zipf s U[1, 2] over [0, 2^24), 256 tenants at k = 1024, 16 GB "
                       "budget, seed 4; latency = completion - scheduled arrival")
    return out


def run_reference(args, wl, rank):
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    n, k, p, w = wl["n"], wl["k"], wl["p"], wl["w"]
    blocks = min(p, 8)
    hi = oracle.block_bounds(n, p, blocks - 1)[1]
    x = oracle.gen_zipf(hi, seed=wl["seed"], s=wl["s"], log2u=wl["log2u"], width=w)

    def step():
        levels = oracle.pss_tree(x, k, blocks)
        oracle.query(levels[-1][0], hi, k)

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t) / args.steps
    value = hi / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "items/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32" if w == 4 else "u64", "data": "synthetic",
        "config": workload_config(wl, 1),
        "cpu_baseline": {"value": value, "unit": "items/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: blocks 0..{blocks - 1} of {p} ({hi} items), "
                                   "block summaries + combine tree + query",
                         "host": host_info()},
        "e2e": {"value": value, "unit": "items/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


SWEEP_S = (0.5, 1.0, 1.5, 2.0, 3.0)
SWEEP_K = (500, 1000, 2000, 4000)


def run_sweep(args):
    """Skew x k sweep of the plain path: n = 2^30 uint32 over [0, 2^32),
    p = 4096, seed = 10 + 4 * i_s + i_k; one JSON line per point."""
    import torch

    import paper_1606_04669_gb300 as P
    hbm, peak_kind = peaks()
    n, p, w = 1 << 30, 4096, 4
    stream = torch.cuda.current_stream()
    x = torch.empty(n, dtype=torch.int32, device="cuda")
    # k = 8000 (the top of the paper's k sweep) runs only when named in
    # --points, with seed 30 + i_s.
    for i_s, zs in enumerate(SWEEP_S):
        for i_k, k in enumerate(SWEEP_K + (8000,)):
            named = bool(args.points) and f"{zs}:{k}" in args.points.split(",")
            if (args.points and not named) or (k == 8000 and not named):
                continue
            seed = 10 + 4 * i_s + i_k if k != 8000 else 30 + i_s
            P.gen_zipf(n, seed=seed, s=zs, log2u=32, out=x)
            torch.cuda.synchronize()

            def step():
                sm = P.summarize(x, k, p, stream=stream)
                q = sm.query(n, k, stream=stream)
                sm.close()
                return q

            for _ in range(max(args.warmup, 1)):
                q = step()
            torch.cuda.synchronize()
            P.profile_read(reset=True)
            P.profile_enable(True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                q = step()
            e1.record(stream)
            torch.cuda.synchronize()
            prof = P.profile_read(reset=True)
            P.profile_enable(False)
            ms = e0.elapsed_time(e1) / args.steps
            sum_ms = prof["summarize_ms"] / max(prof["summarize_calls"], 1)
            alg = n * w + p * k * (w + 16) + p * 24
            line = {
                "metric": METRIC, "workload": "sweep", "zipf_s": zs, "k": k, "seed": seed,
                "value": n / (ms / 1e3), "unit": "items/s", "ms_per_step": ms,
                "input_gbs": n * w / (ms / 1e3) / 1e9, "hbm_frac": n * w / (ms / 1e3) / 1e9 / hbm,
                "summarize_ms": sum_ms, "merge_tree_ms": prof["merge_ms"] / args.steps,
                "roofline": {"bound": "hbm", "achieved": alg / (sum_ms / 1e3) / 1e9, "peak": hbm,
                             "peak_kind": peak_kind, "unit": "GB/s",
                             "frac": alg / (sum_ms / 1e3) / 1e9 / hbm},
                "frequent_items": int(q.size), "steps": args.steps, "warmup": args.warmup,
                "config": {"n": n, "p": p, "universe": "2^32", "item_bytes": w},
            }
            print(json.dumps(line), flush=True)
    return 0


def run_batched(args, emit: bool = True):
    """1024 independent u64 streams (log-uniform lengths in [1e4, 1e8], Zipf s
    in [0.8, 2] over [0, 2^32), k in {64, 256, 1024, 4096}, seed 3) in one
    graph launch, against the plain path looped over the same streams
    (--kind frequent: the Frequent summary, batched and plain).  Returns the
    line (printed when emit)."""
    import torch

    import paper_1606_04669_gb300 as P
    from paper_1606_04669_gb300 import autotune
    from paper_1606_04669_gb300.gen import workloads as W
    specs = W.batched_streams(seed=3, nstreams=args.nstreams)
    stream = torch.cuda.current_stream()
    t = time.perf_counter()
    items = [P.gen_zipf(sp.n, seed=sp.seed, s=sp.s, log2u=sp.log2u, item_bytes=sp.item_bytes,
                        stream_id=sp.index) for sp in specs]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t
    ks = [sp.k for sp in specs]
    frequent = args.kind == "frequent"
    # The plan comes from the data: each stream's skew is estimated on the
    # device from its first 4096 items (no hint from the generator); the run
    # with the generator's exact s as hints is timed beside it.
    est, _ = P.estimate_skew(items)
    err = [abs(e - sp.s) for e, sp in zip(est, specs)]
    total = sum(sp.n for sp in specs)
    summarize = P.frequent if frequent else P.summarize
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(skews):
        plan = [autotune.plan_blocks(sp.n, sp.k, sk, frequent=frequent)
                for sp, sk in zip(specs, skews)]
        b = P.Batch(items, ks, ps=plan, skews=skews, frequent=frequent)
        for _ in range(max(args.warmup, 1)):
            b.run(use_graph=True)
        torch.cuda.synchronize()
        P.profile_read(reset=True)
        e0.record(stream)
        for _ in range(args.steps):
            b.run(use_graph=True, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        nl = P.profile_read(reset=True)["launches"]
        return b, plan, e0.elapsed_time(e1) / args.steps, nl

    hb, _, ms_hinted, _ = timed([sp.s for sp in specs])
    hb.close()
    batch, ps, ms_batched, launches = timed(est)
    res = batch.results()

    def plain():
        out = []
        for i, sp in enumerate(specs):
            sm = summarize(items[i], ks[i], ps[i], stream=stream)
            out.append(sm.query(sp.n, ks[i], stream=stream))
            sm.close()
        return out

    plain()
    torch.cuda.synchronize()
    e0.record(stream)
    pres = plain()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    same = all(a.item.tolist() == b.item.tolist() and a.count.tolist() == b.count.tolist()
               and a.err.tolist() == b.err.tolist() for a, b in zip(res, pres))
    hbm, _ = peaks()
    line = {
        "metric": METRIC, "workload": "batched", "summary": args.kind,
        "value": total / (ms_batched / 1e3),
        "unit": "items/s", "ms_per_step": ms_batched, "steps": args.steps, "warmup": args.warmup,
        "input_gbs": total * 8 / (ms_batched / 1e3) / 1e9,
        "hbm_frac": total * 8 / (ms_batched / 1e3) / 1e9 / hbm,
        "plain_loop": {"value": total / (ms_plain / 1e3), "ms": ms_plain},
        "batched_over_plain": ms_plain / ms_batched, "results_identical": same,
        "hinted": {"value": total / (ms_hinted / 1e3), "ms_per_step": ms_hinted,
                   "estimated_over_hinted": ms_hinted / ms_batched},
        "skew_estimate": {"source": "pss_estimate_skew: pairs of equal items among each "
                                    "stream's first 4096 items",
                          "mean_abs_err": sum(err) / len(err), "max_abs_err": max(err)},
        "gpu_launches_per_step": launches / max(args.steps, 1),
        "config": {"streams": len(specs), "total_items": total, "item_bytes": 8,
                   "k_classes": sorted(set(ks)), "blocks": sum(ps), "seed": 3,
                   "plan": "autotune.plan_blocks (block length per k and skew class) on the "
                           "estimated skews",
                   "generation_s": gen_s},
    }
    if emit:
        print(json.dumps(line), flush=True)
    batch.close()
    return line


def run_served(args, emit: bool = True):
    """Open-loop Poisson arrivals at 2000 requests/s for `duration` seconds
    (seed 4): segments of log-uniform length in [1e4, 1e7] uint32 items, Zipf
    s in [1, 2] over [0, 2^24), generated on the device at admission, for 256
    tenants whose k = 1024 summaries stay resident; 16 GB admission budget.
    Latency = completion - scheduled arrival (no coordinated omission).
    --kind frequent: Frequent (Misra-Gries) tenant summaries.  Returns the
    line (printed when emit)."""
    import numpy as np
    import torch

    import paper_1606_04669_gb300 as P
    from paper_1606_04669_gb300.gen import workloads as W
    reqs = W.served_requests(seed=4, rate=2000.0, duration=args.duration)
    k, tenants = 1024, 256
    # the device generator's own rate on this workload's shape (reported
    # separately: segments are generated at admission, inside the latency)
    g = torch.empty(1 << 28, dtype=torch.int32, device="cuda")
    P.gen_zipf(1 << 24, seed=5, s=1.5, log2u=24, out=g)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record()
    P.gen_zipf(1 << 28, seed=5, s=1.5, log2u=24, out=g)
    g1.record()
    torch.cuda.synchronize()
    gen_rate = (1 << 28) / (g0.elapsed_time(g1) / 1e3)
    del g
    frequent = args.kind == "frequent"
    srv = P.Server(tenants, k, budget_bytes=16 << 30, max_batch=256, max_inflight=4096,
                   frequent=frequent)
    # warm the kernels and the allocator pool outside the measured run
    warm = P.Server(tenants, k, budget_bytes=16 << 30, frequent=frequent)
    warm.submit([dict(id=i, arrival=0.0, tenant=i, n=100_000, s=1.5, log2u=24, seed=99,
                      stream_id=i) for i in range(8)])
    warm.start()
    warm.wait(120)
    warm.close()
    srv.submit([dict(id=r.index, arrival=r.arrival, tenant=r.tenant, n=r.n, s=r.s,
                     log2u=r.log2u, seed=r.seed, stream_id=r.index) for r in reqs])
    P.profile_read(reset=True)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    srv.start()
    srv.wait(args.duration * 20 + 120)
    clk = clocks.stop()
    comps = srv.poll()
    launches = P.profile_read(reset=True)["launches"]
    srv.close()
    lat = np.array([c["completed"] - c["arrival"] for c in comps])
    wait_q = np.array([c["admitted"] - c["arrival"] for c in comps])
    n_of = {r.index: r.n for r in reqs}
    seg_n = np.array([n_of[c["id"]] for c in comps])
    by_len = {}
    for lo, hi, name in ((1e4, 1e5, "1e4-1e5"), (1e5, 1e6, "1e5-1e6"), (1e6, 1e7 + 1, "1e6-1e7")):
        sel = (seg_n >= lo) & (seg_n < hi)
        if sel.any():
            by_len[name] = {"requests": int(sel.sum()),
                            "p50": float(np.percentile(lat[sel], 50) * 1e3),
                            "p99": float(np.percentile(lat[sel], 99) * 1e3)}
    total = sum(r.n for r in reqs)
    t_end = max(c["completed"] for c in comps)
    bad = sum(1 for c in comps if c["status"] != 0)
    line = {
        "metric": METRIC, "workload": "served", "summary": args.kind,
        "value": total / t_end, "unit": "items/s",
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                       "p99": float(np.percentile(lat, 99) * 1e3),
                       "max": float(lat.max() * 1e3),
                       "queue_p50": float(np.percentile(wait_q, 50) * 1e3),
                       "queue_p99": float(np.percentile(wait_q, 99) * 1e3),
                       "by_segment_items": by_len},
        "requests": len(comps), "errors": bad, "offered_items_per_s": total / args.duration,
        "generator_items_per_s": gen_rate,
        "makespan_s": t_end, "gpu_launches": launches, "clocks": clk,
        "config": {"rate": 2000, "duration_s": args.duration, "tenants": tenants, "k": k,
                   "segment_len": "log-uniform [1e4, 1e7]", "zipf_s": "U[1, 2]",
                   "universe": "2^24", "budget_bytes": 16 << 30, "seed": 4,
                   "segments": "generated on the device at admission (included in latency)"},
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


FREQUENT_K = (2000, 500, 64)


def run_frequent(args):
    """The Frequent (Misra-Gries) summary with its merge tree and query on the
    data of workload --base (default the plain one: n = 2^30 uint32 Zipf(1.1)
    over [0, 2^24), seed 2, p = 4096), one JSON line per k (2000, 500, 64)."""
    import numpy as np
    import torch

    import paper_1606_04669_gb300 as P
    wl = WORKLOADS[args.base]
    hbm, peak_kind = peaks()
    n, p, w = wl["n"], wl["p"], wl["w"]
    stream = torch.cuda.current_stream()
    x = P.gen_zipf(n, seed=wl["seed"], s=wl["s"], log2u=wl["log2u"], item_bytes=w)
    dcounts = P.exact_counts(x, wl["log2u"], stream=stream)
    torch.cuda.synchronize()
    points = [int(v) for v in args.points.split(",")] if args.points else FREQUENT_K
    for k in points:
        def step():
            sm = P.frequent(x, k, p, stream=stream)
            q = sm.query(n, k, stream=stream)
            sm.close()
            return q

        for _ in range(max(args.warmup, 1)):
            q = step()
        torch.cuda.synchronize()
        P.profile_read(reset=True)
        P.profile_enable(True)
        clocks = ClockSampler(0)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            q = step()
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        prof = P.profile_read(reset=True)
        P.profile_enable(False)
        ms = e0.elapsed_time(e1) / args.steps
        sum_ms = prof["summarize_ms"] / max(prof["summarize_calls"], 1)
        merge_ms = prof["merge_ms"] / max(args.steps, 1)
        # block summaries: read n*w input bytes once, write p*(k-1) entries and
        # p block headers
        alg = n * w + p * (k - 1) * (w + 16) + p * 24

        # accuracy of the candidates against exact counts (outside the timed region)
        sm = P.frequent(x, k, p, stream=stream)
        accuracy = sm.accuracy(dcounts, wl["log2u"], n, k, stream=stream)
        sm.close()
        accuracy["delta"] = int(q.err[0]) if q.size else None
        accuracy["reported_as"] = "query (count + delta) * k > n; ARE over the reported items"

        e2e = None
        if not args.no_e2e:
            hx = torch.empty(n, dtype=x.dtype, pin_memory=True)
            hx.copy_(x)
            torch.cuda.synchronize()

            def estep():
                sm = P.frequent_host(hx, k, p, stream=stream)
                qq = sm.query(n, k, stream=stream)
                sm.close()
                return qq

            for _ in range(max(args.warmup, 1)):
                qq = estep()
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            esteps = max(1, args.steps // 2)
            a0.record(stream)
            for _ in range(esteps):
                qq = estep()
            a1.record(stream)
            torch.cuda.synchronize()
            ems = a0.elapsed_time(a1) / esteps
            e2e = {"value": n / (ems / 1e3), "unit": "items/s", "ms_per_step": ems,
                   "h2d_bytes_per_step": n * w, "d2h_bytes_per_step": 8 + 24 * qq.size,
                   "api": "pss_frequent_summarize_host + pss_query (pinned host input, read "
                          "in place by the kernels over the CPU-GPU link)"}
            del hx

        cpu = None
        if not args.no_cpu:
            cpu = cpu_baseline_frequent(wl, k, args.cpu_seconds)
        line = {
            "metric": METRIC, "workload": "frequent", "k": k, "value": n / (ms / 1e3),
            "unit": "items/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "Frequent (Misra-Gries, k - 1 counters) summaries, merge tree "
                                   "and query on " + wl["desc"].split("; k=")[0],
                       "n": n, "k": k, "p": p, "item_bytes": w},
            "input_gbs": n * w / (ms / 1e3) / 1e9,
            "hbm_frac": n * w / (ms / 1e3) / 1e9 / hbm,
            "roofline": {"bound": "hbm", "kernel": "frequent_block_kernel (block summaries)",
                         "achieved": alg / (sum_ms / 1e3) / 1e9, "peak": hbm,
                         "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": alg / (sum_ms / 1e3) / 1e9 / hbm,
                         "traffic": traffic_per_launch("frequent_block_kernel", n, k, p, w),
                         "avg_launch_ms": sum_ms, "algorithmic_bytes": alg},
            "breakdown": {"summarize_ms": sum_ms, "merge_tree_ms": merge_ms},
            "accuracy": accuracy, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(prof["launches"]), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_frequent(wl, k: int, budget_s: float):
    """The Frequent oracle, single-threaded, over the first B blocks of the
    workload (block summaries + merge tree + query), B sized to about
    budget_s seconds."""
    import oracle
    n, p, w = wl["n"], wl["p"], wl["w"]
    threads = os.cpu_count() or 1
    lo0, hi0 = oracle.block_bounds(n, p, 0)
    x0 = oracle.gen_zipf(hi0 - lo0, seed=wl["seed"], s=wl["s"], log2u=wl["log2u"], width=w,
                         threads=threads)
    t = time.perf_counter()
    oracle.frequent(x0, k)
    per_block = max(time.perf_counter() - t, 1e-6)
    blocks = int(max(2, min(p, budget_s / per_block)))
    hi = oracle.block_bounds(n, p, blocks - 1)[1]
    x = oracle.gen_zipf(hi, seed=wl["seed"], s=wl["s"], log2u=wl["log2u"], width=w,
                        threads=threads)
    t = time.perf_counter()
    levels = oracle.frequent_tree(x, k, blocks)
    oracle.frequent_query(levels[-1][0], hi, k)
    dt = time.perf_counter() - t
    return {"value": hi / dt, "unit": "items/s", "cores": 1, "kind": "oracle",
            "sample": f"blocks 0..{blocks - 1} of the {p} blocks ({hi} items): Misra-Gries block "
                      f"summaries, their merge tree and the query, single-threaded C++",
            "seconds": dt, "host": host_info()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload",
                    choices=sorted(WORKLOADS) + ["sweep", "batched", "served", "frequent"],
                    default="plain")
    ap.add_argument("--duration", type=float, default=60.0, help="served: seconds of arrivals")
    ap.add_argument("--nstreams", type=int, default=1024)
    ap.add_argument("--points", default="",
                    help="sweep points to run, e.g. 0.5:500,1.1:2000; frequent: k values, e.g. 2000,64")
    ap.add_argument("--kind", choices=("space_saving", "frequent"), default="space_saving",
                    help="batched / served: the summary the streams or tenants use")
    ap.add_argument("--base", choices=sorted(WORKLOADS), default="plain",
                    help="frequent: the workload whose data, n and p it runs on")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="plain workload: leave out the batched form's object")
    ap.add_argument("--no-served", action="store_true",
                    help="plain workload: leave out the served form's object")
    args = ap.parse_args()
    if args.workload in ("sweep", "batched", "served", "frequent"):
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        rc = {"sweep": run_sweep, "batched": run_batched, "served": run_served,
              "frequent": run_frequent}[args.workload](args)
        return rc if isinstance(rc, int) else 0
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, wl, rank)

    import numpy as np
    import torch

    import paper_1606_04669_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n, k, p, w = wl["n"], wl["k"], wl["p"], wl["w"]
    x = P.gen_zipf(n, seed=wl["seed"], s=wl["s"], log2u=wl["log2u"], item_bytes=w,
                   stream_id=rank)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def step():
        sm = P.summarize(x, k, p, stream=stream)
        q = sm.query(n, k, stream=stream)
        sm.close()
        return q

    for _ in range(max(args.warmup, 0)):
        q = step()
    barrier()
    P.profile_read(reset=True)
    P.profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        q = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = P.profile_read(reset=True)
    P.profile_enable(False)
    ms, items_all = replica_aggregate(ev0.elapsed_time(ev1) / args.steps, n, dist, "cuda")
    barrier()
    value = items_all / (ms / 1e3)
    hbm, peak_kind = peaks()
    input_gbs = n * w * world / (ms / 1e3) / 1e9

    # Dominant kernel: the block summaries.  Algorithmic bytes per launch:
    # read n*w input bytes once, write p*k summary entries (item + 8-byte
    # count + 8-byte err) and p block headers.
    sum_ms = prof["summarize_ms"] / max(prof["summarize_calls"], 1)
    alg_bytes = n * w + p * k * (w + 16) + p * 24
    achieved = alg_bytes / (sum_ms / 1e3) / 1e9
    merge_ms = prof["merge_ms"] / max(args.steps, 1)
    query_ms = prof["query_ms"] / max(prof["query_calls"], 1)

    # Accuracy of the answer (the paper's Section 4 metrics), outside the
    # timed region: exact counts on the device, ARE / precision / recall.
    accuracy = None
    if wl["log2u"] <= 28:
        sm = P.summarize(x, k, p, stream=stream)
        counts = P.exact_counts(x, wl["log2u"], stream=stream)
        accuracy = sm.accuracy(counts, wl["log2u"], n, k, stream=stream)
        accuracy["reported_as"] = "query count*k > n; ARE over the reported items"
        sm.close()
        del counts

    e2e = None
    if not args.no_e2e:
        hx = torch.empty(n, dtype=x.dtype, pin_memory=True)
        hx.copy_(x)
        torch.cuda.synchronize()

        def estep():
            sm = P.summarize_host(hx, k, p, stream=stream)
            qq = sm.query(n, k, stream=stream)
            sm.close()
            return qq

        for _ in range(max(args.warmup, 1)):
            qq = estep()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        esteps = max(1, args.steps // 2)
        e0.record(stream)
        for _ in range(esteps):
            qq = estep()
        e1.record(stream)
        torch.cuda.synchronize()
        ems, eitems = replica_aggregate(e0.elapsed_time(e1) / esteps, n, dist, "cuda")
        e2e = {"value": eitems / (ems / 1e3), "unit": "items/s", "ms_per_step": ems,
               "h2d_bytes_per_step": n * w, "d2h_bytes_per_step": 8 + 24 * qq.size,
               # the host input crosses the CPU-GPU link once per step: its rate
               "link_gbs": n * w / (ems / 1e3) / 1e9,
               "api": "pss_summarize_host + pss_query (pinned host input, read in place by the "
                      "kernels over the CPU-GPU link; pss_set_host_direct(0) stages copies)"}
        del hx

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(wl, args.cpu_seconds)

    if rank == 0:
        kernel = P.plan_kernel(k, p, w)
        line = {
            "metric": METRIC, "value": value, "unit": "items/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32" if w == 4 else "u64", "data": "synthetic",
            "config": workload_config(wl, world),
            "input_gbs": input_gbs,
            "hbm_frac": input_gbs / hbm,
            "hbm_frac_nominal_8tbs": input_gbs / 8000.0,
            "roofline": {"bound": "hbm", "kernel": kernel + " (block summaries)",
                         "achieved": achieved, "peak": hbm, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic_per_launch(kernel, n, k, p, w),
                         "avg_launch_ms": sum_ms, "algorithmic_bytes": alg_bytes},
            "breakdown": {"summarize_ms": sum_ms, "merge_tree_ms": merge_ms,
                          "query_ms": query_ms,
                          "fractional_overhead": merge_ms / sum_ms if sum_ms > 0 else None},
            "frequent_items": int(q.size),
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(prof["launches"]),
            "clocks": clk,
        }
        # The batched and served forms beside the plain one (single-GPU runs:
        # the metric compares the three forms on one GPU).
        if world == 1 and args.workload == "plain":
            del x, q
            torch.cuda.empty_cache()
            if not args.no_batched:
                line["batched"] = batched_summary(run_batched(
                    argparse.Namespace(nstreams=1024, kind="space_saving",
                                       steps=min(args.steps, 5),
                                       warmup=max(1, min(args.warmup, 2))), emit=False))
                torch.cuda.empty_cache()
            if not args.no_served:
                line["served"] = served_summary(run_served(
                    argparse.Namespace(duration=args.duration, kind="space_saving"), emit=False))
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
