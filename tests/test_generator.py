"""The seeded input generator (host side): Philox known answers, the
elementary functions, the Zipf law and the rank -> item bijection."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle


def test_philox_known_answers():
    # Published known-answer vectors of Philox4x32-10 (Salmon et al., SC 2011).
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C,
                                                          0x9B00DBD8]
    assert oracle.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert oracle.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                                [0xA4093822, 0x299F31D0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420,
                                                              0x24126EA1]


def test_log_exp_accuracy():
    rng = np.random.default_rng(1)
    for x in np.concatenate([rng.uniform(1e-6, 1e6, 500), [0.5, 1.0, 2.0, 2 ** 32, 1.5]]):
        assert abs(oracle.gen_log(float(x)) - math.log(x)) <= 4e-16 * max(1.0, abs(math.log(x)))
    for y in np.concatenate([rng.uniform(-80, 80, 500), [0.0, 1.0, -1.0, 22.2]]):
        assert abs(oracle.gen_exp(float(y)) - math.exp(y)) <= 3e-15 * math.exp(y)


def test_table_log_exp_accuracy():
    # The sampler's table-driven log and exp against the math library, over
    # wide ranges, every table cell (x = 2^e (1 + j/128 + ...)) and near 1.
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.uniform(1e-6, 1e6, 2000), np.exp(rng.uniform(-40, 44, 2000)),
                         1 + (np.arange(128) + rng.random(128)) / 128,
                         1 - rng.uniform(0, 1e-3, 200), 1 + rng.uniform(0, 1e-3, 200),
                         [0.5, 1.0, 2.0, 2 ** 32 + 0.5, 1.5, 2 ** 64]])
    for x in xs:
        ref = math.log(x)
        assert abs(oracle.gen_log_t(float(x)) - ref) <= 4e-16 * max(1.0, abs(ref)), x
    ys = np.concatenate([rng.uniform(-88, 45, 3000), np.arange(-64, 65) * math.log(2) / 64,
                         [0.0, 1.0, -1.0, 22.2, 1e-12, -1e-12]])
    for y in ys:
        ref = math.exp(y)
        assert abs(oracle.gen_exp_t(float(y)) - ref) <= 3e-15 * ref, y


@pytest.mark.parametrize("s", [0.5, 1.0, 1.1, 1.8, 3.0])
def test_zipf_law(s):
    # Chi-square goodness of fit of the ranks to P(r) ~ r^-s on [1, N].
    n_ranks, count = 64, 200_000
    r = oracle.gen_zipf_ranks(count, seed=7, s=s, n_ranks=n_ranks)
    assert r.min() >= 1 and r.max() <= n_ranks
    obs = np.bincount(r.astype(np.int64), minlength=n_ranks + 1)[1:]
    w = np.arange(1, n_ranks + 1, dtype=np.float64) ** -s
    exp = count * w / w.sum()
    keep = exp >= 5
    chi2 = float((((obs - exp) ** 2) / exp)[keep].sum())
    dof = int(keep.sum()) - 1
    # 99.99th percentile of chi-square with <= 63 dof is below 120
    assert chi2 < 120, (s, chi2, dof)


def test_zipf_large_universe_head():
    # U = 2^32 (the sweep's universe): the head frequencies follow r^-s.
    r = oracle.gen_zipf_ranks(300_000, seed=3, s=1.5, n_ranks=2 ** 32)
    c = np.bincount(np.minimum(r, 5).astype(np.int64), minlength=6)
    h = sum(i ** -1.5 for i in range(1, 200000)) + 2 * 200000 ** -0.5  # zeta(1.5) tail estimate
    p1 = 1.0 / h
    assert abs(c[1] / 300_000 - p1) < 5 * math.sqrt(p1 * (1 - p1) / 300_000)
    assert abs(c[1] / c[2] - 2 ** 1.5) < 0.1


def test_rank_to_item_bijection():
    for b in (1, 2, 7, 10, 16):
        items = {oracle.rank_to_item(r, b) for r in range(1, 2 ** b + 1)}
        assert items == set(range(2 ** b))


def test_stream_determinism_and_offsets():
    a = oracle.gen_zipf(1000, seed=9, s=1.1, log2u=20)
    b = oracle.gen_zipf(1000, seed=9, s=1.1, log2u=20)
    assert np.array_equal(a, b)
    c = oracle.gen_zipf(600, seed=9, s=1.1, log2u=20, start=400)
    assert np.array_equal(a[400:], c[:600])
    d = oracle.gen_zipf(1000, seed=9, s=1.1, log2u=20, stream=1)
    assert not np.array_equal(a, d)
    assert a.max() < 2 ** 20
    e = oracle.gen_zipf(1000, seed=9, s=1.1, log2u=32, width=8)
    assert e.dtype == np.uint64 and int(e.max()) < 2 ** 32
