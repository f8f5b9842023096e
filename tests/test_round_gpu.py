"""The round kernel (one warp per block, 32 items per round) against the
oracle: every Space Saving parity case of test_parity_gpu with every block
summary on it, bit-exact at every tree level."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_04669_gb300 as P  # noqa: E402
from tests import test_parity_gpu as T  # noqa: E402


@pytest.fixture
def round_kernel():
    prev_w = P.set_warp_kmax(0)
    prev_r = P.set_round_kmax(P.PSS_MAX_K_RESIDENT)
    yield
    P.set_round_kmax(prev_r)
    P.set_warp_kmax(prev_w)


@pytest.mark.parametrize("n,k,p,w,s,log2u,seed", [
    c for c in [
        (50_000, 64, 4, 4, 1.1, 16, 101),
        (123_457, 200, 13, 4, 0.8, 20, 102),
        (200_000, 500, 5, 4, 1.5, 32, 103),
        (300_000, 1000, 3, 4, 1.0, 32, 104),
        (100_000, 2000, 8, 8, 1.2, 32, 105),
        (80_000, 4096, 2, 4, 0.9, 24, 106),
        (80_000, 4096, 3, 8, 1.3, 40, 107),
        (60_000, 2, 9, 4, 1.1, 12, 108),
        (70_000, 333, 31, 4, 0.5, 32, 109),
        (150_000, 1024, 1, 8, 2.0, 32, 110),
        (262_144, 2000, 1, 4, 1.1, 24, 2),
        (300_000, 3, 4, 4, 0.7, 10, 111),
        (400_000, 17, 2, 8, 1.0, 14, 112),
    ]])
def test_round_random_configs(round_kernel, n, k, p, w, s, log2u, seed):
    x = oracle.gen_zipf(n, seed=seed, s=s, log2u=log2u, width=w)
    T.compare_tree(x, k, p)


def test_round_edges(round_kernel):
    T.test_edge_empty_and_tiny()
    T.test_edge_all_same_and_all_distinct()
    T.test_edge_hash_collisions()
    T.test_interleaved_hits_misses_windows()


def test_round_fuzz_small_universes(round_kernel):
    T.test_fuzz_small_universes()


def test_round_small_k_sweep(round_kernel):
    rng = np.random.default_rng(7)
    for k in (2, 3, 5, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513):
        w = 8 if k % 2 else 4
        s = 0.5 + 1.8 * rng.random()
        x = oracle.gen_zipf(30_000 + 61 * k, seed=700 + k, s=s, log2u=12 if k < 64 else 32, width=w)
        T.compare_tree(x, k, 1 + k % 5)
