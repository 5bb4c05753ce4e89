"""Multi-value GPU path against the CPU oracle: exact counts and offsets, equal sorted
per-query value multisets (Sec. IV-B4); slot layout is never compared."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import wc_inputs
from tests.golden_fixtures import run_mv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wc():
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    return wc


def make_mv(wc, kb, vb, keys_cap, pool, W=0, G=None, seed=0x77):
    t = wc.MultiValueTable(kb, vb, min_capacity=keys_cap, value_pool_capacity=pool, window_width=W, seed=seed)
    if G is not None:
        for op in (wc.WC_OP_COUNT, wc.WC_OP_ERASE):
            t.set_launch(op, G)
    return t


def check_queries(t, o, q):
    offs, _ = t.count_values(q)
    eoffs, _ = o.count_values(q)
    np.testing.assert_array_equal(offs, eoffs)
    vals, _ = t.retrieve_multi(q, offs)
    evals, _ = o.retrieve_multi(q, eoffs)
    assert vals.size == evals.size == int(eoffs[-1])
    np.testing.assert_array_equal(oracle.sorted_segments(vals, offs), oracle.sorted_segments(evals, eoffs))


class _Adapter:
    def __init__(self, t):
        self.t = t

    def insert(self, k, v):
        return self.t.insert(k, v)

    def erase(self, k):
        return self.t.erase(k)

    def count_values(self, q):
        return self.t.count_values(q)

    def retrieve_multi(self, q, offs):
        return self.t.retrieve_multi(q, offs)

    def size(self):
        return self.t.size()


def test_golden_mv_worked_example_gpu(wc):
    assert run_mv("mv_ops.txt", lambda: _Adapter(make_mv(wc, 8, 4, 64, 1024))) >= 8


@pytest.mark.parametrize("W,G", [(2, 1), (2, 2), (4, 1), (4, 2), (4, 4), (8, 2), (8, 4), (8, 8)])
def test_mv_zipf_parity_every_shape(wc, W, G):
    uni, n_ins, n_abs = 1 << 14, 300_007, 1 << 12
    d = wc_inputs.mv_zipf_u64(0x57C00004 + W * 16 + G, uni, n_ins, n_abs)
    t = make_mv(wc, 8, 4, int(uni / 0.8) + 1, n_ins + 4 * uni, W, G)
    o = oracle.MultiValue(8, 4)
    t.insert(d["keys"], d["values"])
    o.insert(d["keys"], d["values"])
    assert t.size() == o.size() == n_ins
    assert t.num_keys() == o.num_keys()
    check_queries(t, o, d["queries"])


@pytest.mark.parametrize("kb,vb", [(4, 4), (4, 8), (8, 8)])
def test_mv_widths_and_repeat_inserts(wc, kb, vb):
    """Several insert calls on the same keys: buckets of later calls link to earlier
    ones (Sec. IV-C back references); erase drops every value of a key."""
    rng = np.random.default_rng(kb * 10 + vb)
    top = (1 << (8 * kb)) - 1
    universe = np.unique(rng.integers(1, min(top, 2 ** 62), 5000, dtype=np.uint64))
    t = make_mv(wc, kb, vb, 8192, 400_000)
    o = oracle.MultiValue(kb, vb)
    vmax = (1 << (8 * vb)) - 1
    for step in range(8):
        m = int(rng.integers(1, 20_000))
        ks = universe[np.minimum(rng.zipf(1.3, m), universe.size) - 1]
        vs = rng.integers(0, vmax, m, dtype=np.uint64, endpoint=True)
        t.insert(ks, vs)
        o.insert(ks, vs)
        if step == 5:
            drop = universe[:50]
            t.erase(drop)
            o.erase(drop)
        assert t.size() == o.size()
        assert t.num_keys() == o.num_keys()
        check_queries(t, o, universe)


def test_mv_paper_invariant_uniform_r(wc):
    """Sec. V-C: n keys from 1..n/r queried over 1..n return exactly n values."""
    n = 1 << 17
    for r in (1, 4, 32, 1024):
        d = wc_inputs.mv_uniform_r(500 + r, n, r)
        t = make_mv(wc, 8, 4, int(max(1, n // r) / 0.8) + 1, n + 2 * (n // r) + 64)
        t.insert(d["keys"], d["values"])
        offs, _ = t.count_values(d["queries"])
        assert int(offs[-1]) == n
        vals, _ = t.retrieve_multi(d["queries"], offs)
        np.testing.assert_array_equal(np.sort(vals), np.arange(n, dtype=np.uint32))
        seg = np.repeat(np.arange(n), np.diff(offs.astype(np.int64)))
        np.testing.assert_array_equal(d["queries"][seg], d["keys"][vals])


def test_mv_single_hot_key_spans_many_chunks(wc):
    """One key holding most of the batch: its bucket is split over many blocks."""
    n = 1 << 20
    keys = np.full(n, 12345, dtype=np.uint64)
    keys[::7] = np.arange(1, keys[::7].size + 1, dtype=np.uint64) + 100_000
    vals = np.arange(n, dtype=np.uint32)
    t = make_mv(wc, 8, 4, 1 << 18, n + (1 << 19))
    o = oracle.MultiValue(8, 4)
    t.insert(keys, vals)
    o.insert(keys, vals)
    q = np.concatenate([[12345, 7, 100_001], np.arange(100_001, 100_100)]).astype(np.uint64)
    check_queries(t, o, q)


def test_mv_sentinels_empty_and_pool_exhaustion(wc):
    t = make_mv(wc, 8, 4, 4096, 64)
    f = t.insert(np.array([0, 2 ** 64 - 1, 5], dtype=np.uint64), np.array([1, 2, 4], dtype=np.uint32))
    assert f == wc.WC_FLAG_INVALID_KEY
    offs, f = t.count_values(np.array([0, 5, 6], dtype=np.uint64))
    assert list(offs) == [0, 0, 1, 1] and f == wc.WC_FLAG_INVALID_KEY
    offs, _ = t.count_values(np.array([], dtype=np.uint64))
    assert list(offs) == [0]
    # the pool holds 64 values: a batch of 1000 cannot fit -> flagged, nothing corrupt
    f = t.insert(np.arange(1, 1001, dtype=np.uint64), np.arange(1000, dtype=np.uint32))
    assert f & wc.WC_FLAG_POOL_EXHAUSTED
    q = np.arange(1, 1001, dtype=np.uint64)
    offs, _ = t.count_values(q)
    vals, _ = t.retrieve_multi(q, offs)
    stored = np.repeat(q, np.diff(offs.astype(np.int64)))
    np.testing.assert_array_equal(vals.astype(np.uint64), stored - 1)  # value = key - 1
    # buckets are reserved per block of key-store slots: blocks that fit keep their values
    assert t.size() == int(offs[-1]) < 1001


def test_mv_u32_keys_full_mix(wc):
    d = wc_inputs.mv_zipf_u64(99, 1 << 12, 1 << 16, 1 << 10)
    keys32 = (d["keys"] & np.uint64(0x7FFFFFFF)).astype(np.uint32) | np.uint32(1)
    q32 = (d["queries"] & np.uint64(0x7FFFFFFF)).astype(np.uint32) | np.uint32(1)
    t = make_mv(wc, 4, 4, 8192, 1 << 17)
    o = oracle.MultiValue(4, 4)
    t.insert(keys32, d["values"])
    o.insert(keys32, d["values"])
    check_queries(t, o, q32)
    assert t.size() == o.size()


def test_mv_region_split_insert_parity(wc):
    """A key store above 64 MiB and a batch of >= 2^20 pairs take the region-split insert;
    counts and value multisets still equal the oracle's, also on a repeat insert."""
    uni, n = 1 << 22, 1 << 21
    d = wc_inputs.mv_zipf_u64(0x5B117, uni, n, 1 << 16)
    t = make_mv(wc, 8, 4, 5_000_000, 2 * n + 4 * uni)
    assert t.info["table_bytes"] > (64 << 20)
    o = oracle.MultiValue(8, 4)
    for rep in range(2):
        t.insert(d["keys"], d["values"])
        o.insert(d["keys"], d["values"])
        assert t.size() == o.size() == (rep + 1) * n
        assert t.num_keys() == o.num_keys()
    q = d["queries"][wc_inputs.shuffle_index(3, d["queries"].size)[:200_000]]
    check_queries(t, o, q)


# ---- bucket growth strategy (Sec. IV-C) ---------------------------------------------------

def bucket_sizes(s0, lam, upto):
    """s_0 = s0, s_i = ceil(lambda * s_{i-1}) (a product within 1e-9 of an integer counts as
    that integer), until the sizes hold `upto` values."""
    import math
    sizes, total = [], 0
    s = s0
    while total < upto:
        sizes.append(s)
        total += s
        x = lam * s
        s = max(s, math.ceil(x - 1e-9 * x))
    return sizes


def pool_elements(count, s0, lam, vb):
    """Pool elements a key with `count` values occupies: its buckets 0..b, each holding
    its values plus (all but the first) an 8-byte back reference, in whole 8-byte words."""
    if count == 0:
        return 0
    used = 0
    for i, s in enumerate(bucket_sizes(s0, lam, count)):
        e = s + (8 // vb if i else 0)
        used += (e + 1) & ~1 if vb == 4 else e
    return used


def test_growth_paper_example_buckets_1_2_4(wc):
    """Fig. 4 / Sec. IV-C: s0 = 1 and lambda = 2 give buckets of 1, 2 and 4 values for six
    values; the seventh fills the last bucket, the eighth opens a bucket of 8."""
    assert bucket_sizes(1, 2.0, 6) == [1, 2, 4]
    t = wc.MultiValueTable(4, 4, min_capacity=64, value_pool_capacity=1024, bucket_first_size=1, bucket_growth=2.0)
    o = oracle.MultiValue(4, 4)
    for vals in ([1, 2], [3], [4, 5, 6]):  # three calls: appends go into the last bucket first
        k = np.full(len(vals), 42, np.uint32)
        t.insert(k, np.array(vals, np.uint32))
        o.insert(k, np.array(vals, np.uint32))
    check_queries(t, o, np.array([42, 7], np.uint32))
    assert t.pool_used() == pool_elements(6, 1, 2.0, 4) == 2 + 4 + 6
    t.insert(np.array([42], np.uint32), np.array([7], np.uint32))
    assert t.pool_used() == pool_elements(7, 1, 2.0, 4) == 12
    t.insert(np.array([42], np.uint32), np.array([8], np.uint32))
    assert t.pool_used() == pool_elements(8, 1, 2.0, 4) == 12 + 10
    o.insert(np.array([42, 42], np.uint32), np.array([7, 8], np.uint32))
    check_queries(t, o, np.array([42], np.uint32))
    assert run_mv("mv_ops.txt", lambda: _Adapter(wc.MultiValueTable(8, 4, min_capacity=64, value_pool_capacity=1024,
                                                                    bucket_first_size=1, bucket_growth=2.0))) >= 8


@pytest.mark.parametrize("kb,vb", [(4, 4), (8, 8)])
@pytest.mark.parametrize("s0,lam", [(1, 1.1), (1, 2.0), (3, 1.5), (4, 1.0), (1, 1.0)])
def test_growth_repeat_inserts_and_pool_accounting(wc, kb, vb, s0, lam):
    """Growth strategy over repeated insert calls (each call first fills the key's last
    bucket) with erases in between: counts and value multisets equal the oracle's, and the
    pool holds exactly the buckets the growth formula gives each key's final count."""
    rng = np.random.default_rng(int(s0 * 100 + lam * 10) + kb)
    universe = np.unique(rng.integers(1, 2 ** 31 - 1, 4000, dtype=np.uint64))
    if kb == 4:
        universe = universe.astype(np.uint32)
    t = wc.MultiValueTable(kb, vb, min_capacity=8192, value_pool_capacity=3_000_000, bucket_first_size=s0,
                           bucket_growth=lam)
    o = oracle.MultiValue(kb, vb)
    counts, pool = {}, 0
    vmax = (1 << (8 * vb)) - 1
    for step in range(8):
        m = int(rng.integers(1, 30_000))
        ks = universe[np.minimum(rng.zipf(1.4, m), universe.size) - 1]
        vs = rng.integers(0, vmax, m, dtype=np.uint64, endpoint=True)
        if vb == 4:
            vs = vs.astype(np.uint32)
        assert t.insert(ks, vs) == 0
        o.insert(ks, vs)
        u, c = np.unique(ks, return_counts=True)
        for k, n in zip(u.tolist(), c.tolist()):
            counts[k] = counts.get(k, 0) + n
        if step == 4:
            drop = universe[:300]
            t.erase(drop)
            o.erase(drop)
            for k in drop.tolist():
                pool += pool_elements(counts.pop(k, 0), s0, lam, vb)  # erased buckets stay allocated
        assert t.size() == o.size()
        check_queries(t, o, universe)
    expect = pool + sum(pool_elements(n, s0, lam, vb) for n in counts.values())
    assert t.pool_used() == expect


def test_growth_uniform_r_invariant_and_snapshot(wc):
    """Sec. V-C invariant with the paper's default growth (lambda = 1.1, s0 = 1), then a
    snapshot restored into a table of the same growth parameters (and refused by another)."""
    n = 1 << 17
    for r in (1, 16, 256):
        d = wc_inputs.mv_uniform_r(900 + r, n, r)
        t = wc.MultiValueTable(8, 4, min_capacity=int(max(1, n // r) / 0.8) + 1, value_pool_capacity=4 * n,
                               bucket_first_size=1, bucket_growth=1.1)
        t.insert(d["keys"][: n // 2], d["values"][: n // 2])
        t.insert(d["keys"][n // 2:], d["values"][n // 2:])
        offs, _ = t.count_values(d["queries"])
        assert int(offs[-1]) == n
        vals, _ = t.retrieve_multi(d["queries"], offs)
        np.testing.assert_array_equal(np.sort(vals), np.arange(n, dtype=np.uint32))
        seg = np.repeat(np.arange(n), np.diff(offs.astype(np.int64)))
        np.testing.assert_array_equal(d["queries"][seg], d["keys"][vals])
    snap = wc.api.wc_table_snapshot(t.handle)
    kw = dict(min_capacity=int(max(1, n // 256) / 0.8) + 1, value_pool_capacity=4 * n, bucket_first_size=1)
    u = wc.MultiValueTable(8, 4, bucket_growth=1.1, **kw)
    wc.api.wc_table_restore(u.handle, snap)
    offs2, _ = u.count_values(d["queries"])
    np.testing.assert_array_equal(offs2, offs)
    other = wc.MultiValueTable(8, 4, bucket_growth=1.2, **kw)  # held: a freed handle must not be passed
    with pytest.raises(wc.WcError):
        wc.api.wc_table_restore(other.handle, snap)


def test_growth_parameters_are_validated(wc):
    for kw in (dict(bucket_first_size=1, bucket_growth=0.9), dict(bucket_first_size=1, bucket_growth=1.0001)):
        with pytest.raises(wc.WcError):
            wc.MultiValueTable(8, 4, min_capacity=64, value_pool_capacity=64, **kw)
    with pytest.raises(wc.WcError):  # single-value tables have no buckets
        wc.SingleValueTable(4, 4, min_capacity=64, bucket_first_size=1, bucket_growth=2.0)


def test_mv_full_key_store_keeps_whole_keys(wc):
    """More distinct keys than key-store slots, spread over many tiles: PROBE_LIMIT is
    raised and a key is either stored with every one of its values (those of all tiles
    it occurs in) or not at all; the key count and the size agree with what is stored."""
    t = make_mv(wc, 8, 4, 64, 1 << 16)
    cap = t.capacity
    rng = np.random.default_rng(5)
    uni = np.arange(1, 4 * cap + 1, dtype=np.uint64) * np.uint64(0x9E3779B1)
    keys = uni[rng.integers(0, uni.size, 20000)]
    vals = np.arange(keys.size, dtype=np.uint32)
    o = oracle.MultiValue(8, 4)
    o.insert(keys, vals)
    f = t.insert(keys, vals)
    assert f & wc.WC_FLAG_PROBE_LIMIT
    offs, _ = t.count_values(uni)
    got = np.diff(offs.astype(np.int64))
    want, _ = o.count_values(uni)
    want = np.diff(want.astype(np.int64))
    stored = got > 0
    np.testing.assert_array_equal(got[stored], want[stored])
    assert 0 < stored.sum() <= cap and t.num_keys() == stored.sum()
    assert t.size() == int(offs[-1]) == int(want[stored].sum())
    q = uni[stored]
    qo, _ = t.count_values(q)
    v, _ = t.retrieve_multi(q, qo)
    eo, _ = o.count_values(q)
    ev, _ = o.retrieve_multi(q, eo)
    np.testing.assert_array_equal(qo, eo)
    np.testing.assert_array_equal(oracle.sorted_segments(v, qo), oracle.sorted_segments(ev, eo))
