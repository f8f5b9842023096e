"""The benchmark's JSON line as the reference arm prints it (the oracle on the
host cores; runs without a GPU), and the host-side bookkeeping the GPU arm
uses for its roofline object."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e", "dtype", "data"):
        assert key in d, key
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "items/s" and d["higher_is_better"] is True and d["value"] > 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_traffic_record_matches_only_its_shape():
    sys.path.insert(0, ROOT)
    import bench
    t = bench.TRAFFIC["ss_block_kernel"]
    n = t["block_items"] * 4096
    # another block length, another k or another item width: no record
    assert bench.traffic_per_launch("ss_block_kernel", n // 2, t["k"], 4096, t["w"]) is None
    assert bench.traffic_per_launch("ss_block_kernel", n, t["k"] + 1, 4096, t["w"]) is None
    assert bench.traffic_per_launch("ss_block_kernel", n, t["k"], 4096, 8) is None
    assert bench.traffic_per_launch("no_such_kernel", n, t["k"], 4096, t["w"]) is None
    got = bench.traffic_per_launch("ss_block_kernel", n, t["k"], 4096, t["w"])
    # None once the kernel's source has changed since the capture; else p blocks' bytes
    assert got is None or abs(got - 4096 * t["bytes_per_block"]) < 1.0
