"""The C ABI library loads and exports every function include/*.h declares
(no compute calls: this runs without a GPU)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import paper_1606_04669_gb300 as P
from paper_1606_04669_gb300 import pss as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^[A-Za-z_][\w\s\*]*?\b(pss_\w+)\s*\(", re.M)


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(DECL.findall(text))
    return names


def test_header_declares_the_boundary():
    names = declared()
    for core in ("pss_summarize", "pss_merge", "pss_query", "pss_export", "pss_free",
                 "pss_strerror"):
        assert core in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(P.lib_path() if os.path.exists(P.lib_path()) else P.load()._name)
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert declared() <= set(binding.SIGNATURES), declared() - set(binding.SIGNATURES)


def test_strerror_without_gpu():
    lib = P.load()
    assert lib.pss_strerror(0) == b"success"
    assert lib.pss_strerror(-2).startswith(b"summaries have different k")
    assert lib.pss_abi_version() == 1


def test_planner_matches_the_autotuned_table():
    # pss_plan_blocks (host arithmetic, no device) and autotune.plan_blocks
    # read the same measured table.
    import random

    import paper_1606_04669_gb300 as P
    from paper_1606_04669_gb300 import autotune as A
    rng = random.Random(5)
    for _ in range(3000):
        n = rng.randint(0, 10 ** 10)
        k = rng.choice([2, 64, 65, 256, 257, 1024, 1025, 4096, 8000])
        s = rng.choice([0.5, 0.8, 1.1, 1.4, 1.7, 2.0, 2.7, rng.uniform(0.3, 3.0)])
        assert P.plan_blocks(n, k, 4, s) == A.plan_blocks(n, k, s), (n, k, s)
        assert P.plan_blocks(n, k, 4, s, frequent=True) == A.plan_blocks(n, k, s, frequent=True)
