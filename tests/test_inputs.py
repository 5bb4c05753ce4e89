"""Checks of the seeded input generators against their definitions (no GPU)."""
from __future__ import annotations

import numpy as np

import wc_inputs as w


def test_splitmix64_reference_values():
    # SplitMix64 with seed 0: the first outputs of Vigna's public-domain reference
    # generator (state advanced by the golden gamma before each output).
    assert [int(x) for x in w.splitmix64(0, 0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_lowbias32_is_a_bijection_on_a_slice():
    x = np.arange(1 << 20, dtype=np.uint32) * np.uint32(4093)
    assert np.unique(w.lowbias32(x)).size == x.size


def test_distinct_keys_are_distinct_and_sentinel_free():
    for f, top in ((w.distinct_u32, 0xFFFFFFFF), (w.distinct_u64, 2 ** 64 - 1)):
        k = f(123, 300_000)
        assert k.size == 300_000
        assert np.unique(k).size == k.size
        assert not np.any(k == 0) and not np.any(k == top)


def test_shuffle_index_is_a_permutation():
    for n in (1, 2, 3, 1000, 65536, 100_003):
        p = w.shuffle_index(7, n)
        assert np.array_equal(np.sort(p), np.arange(n))


def test_zipf_rank1_frequency_matches_harmonic_number():
    # P(rank 1) = 1 / H_{N,s} with H summed exactly in float64 (independent of the
    # sampler's head table and tail integral).
    N, s = 1 << 24, 1.1
    H = float(np.sum(np.arange(1, N + 1, dtype=np.float64) ** -s))
    z = w.ZipfSampler(N, s)
    assert abs(z.prob_rank1() - 1.0 / H) < 1e-5
    r = z.sample(99, 1 << 21)
    p1 = 1.0 / H
    sd = np.sqrt(p1 * (1 - p1) / r.size)
    assert abs((r == 0).mean() - p1) < 5 * sd
    # rank 2 and rank 100 follow r^-s too
    for rank in (2, 100):
        pr = rank ** -s / H
        sd = np.sqrt(pr * (1 - pr) / r.size)
        assert abs((r == rank - 1).mean() - pr) < 5 * sd
    assert r.min() >= 0 and r.max() < N


def test_zipf_tail_mass():
    # mass of ranks > 2^20 (the part drawn from the integral approximation)
    N, s = 1 << 24, 1.1
    w_all = np.arange(1, N + 1, dtype=np.float64) ** -s
    tail = w_all[1 << 20:].sum() / w_all.sum()
    r = w.ZipfSampler(N, s).sample(5, 1 << 21)
    frac = (r >= (1 << 20)).mean()
    sd = np.sqrt(tail * (1 - tail) / r.size)
    assert abs(frac - tail) < 5 * sd


def test_sv_recipe_shapes():
    d = w.sv_insert_retrieve_u32(1, 1000, 500, 500)
    assert d["queries"].size == 1000
    assert (d["q_src"] >= 0).sum() == 500
    assert np.array_equal(d["queries"][d["q_src"] >= 0], d["keys"][d["q_src"][d["q_src"] >= 0]])
    assert not np.isin(d["queries"][d["q_src"] < 0], d["keys"]).any()


def test_c_stream_fills_equal_the_numpy_definitions():
    w.build_helper()
    assert w._helper() is not None
    a = w.splitmix64(0xDEADBEEF, 17, 50_000)
    b = w.splitmix64_np(0xDEADBEEF, 17, 50_000)
    assert np.array_equal(a, b)
    hi = w.uniform_u32(5, 50_000)
    assert np.array_equal(hi, (w.splitmix64_np(5, 0, 50_000) >> np.uint64(32)).astype(np.uint32))
    x = np.arange(50_002, dtype=np.uint64).astype(np.uint32) * np.uint32(0x9E3779B9) + np.uint32(12345)
    ref = w.lowbias32(x)
    keep = ref[(ref != 0) & (ref != np.uint32(0xFFFFFFFF))][:50_000]
    assert np.array_equal(w.distinct_u32(12345, 50_000), keep)


def test_serving_trace_shape():
    tr = w.serving_trace(3, n_tables=4, log2_cap=(10, 12), n_requests=50, log2_batch=(4, 9))
    assert len(tr["requests"]) == 50 and len(tr["caps"]) == 4
    for r in tr["requests"]:
        assert r["op"] in (0, 1, 2) and r["keys"].size >= 1
        if r["op"] == 0:
            assert r["values"].size == r["keys"].size
    arr = w.poisson_arrivals(1, 1000, 1e6)
    assert (np.diff(arr.astype(np.int64)) >= 0).all()
    assert 0.5e-3 < arr[-1] / 1e9 < 2e-3  # ~1000 arrivals at 1e6/s take ~1 ms
