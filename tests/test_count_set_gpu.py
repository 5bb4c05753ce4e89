"""Counting tables, hash sets and Bloom filters (Sec. IV's CountingHashTable, HashSet and
BloomFilter) against their CPU oracles, element by element."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import wc_inputs

pytestmark = pytest.mark.gpu

COUNT_SHAPES = [(4, 4, 1), (4, 4, 2), (4, 8, 1), (4, 8, 2), (4, 16, 2), (4, 16, 4), (4, 32, 4), (4, 32, 8),
                (8, 2, 1), (8, 4, 1), (8, 4, 2), (8, 8, 2), (8, 8, 4), (8, 16, 4), (8, 16, 8)]


@pytest.fixture(scope="module")
def wc():
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    return wc


def zipf_keys(seed, kb, universe, n):
    d = wc_inputs.mv_zipf_u64(seed, universe, n, 1 << 10)
    if kb == 4:
        return ((d["keys"] & np.uint64(0x7FFFFFFF)) | np.uint64(1)).astype(np.uint32), \
            ((d["queries"] & np.uint64(0x7FFFFFFF)) | np.uint64(1)).astype(np.uint32)
    return d["keys"], d["queries"]


def check_counts(t, o, q):
    out, found, _ = t.retrieve(q)
    eo, ef, _ = o.retrieve(q)
    np.testing.assert_array_equal(found, ef)
    np.testing.assert_array_equal(out, eo)


# ---- counting tables ---------------------------------------------------------------------

@pytest.mark.parametrize("kb,W,G", COUNT_SHAPES)
def test_counting_parity_every_shape(wc, kb, W, G):
    """Zipf keys (a hot key is incremented by thousands of threads at once): unit-weight
    and weighted inserts, erase, re-insert; counts equal the oracle's."""
    keys, q = zipf_keys(0xC0 + kb * 64 + W + G, kb, 1 << 12, 150_001)
    t = wc.CountingTable(kb, min_capacity=1 << 13, window_width=W)
    t.set_launch(wc.WC_OP_INSERT, G)
    o = oracle.Counting(kb)
    assert t.insert(keys) == o.insert(keys) == 0
    check_counts(t, o, q)
    w = wc_inputs.uniform_u32(5, keys.size) if kb == 4 else wc_inputs.uniform_u64(5, keys.size)
    assert t.insert(keys, w) == o.insert(keys, w) == 0  # weighted, wrapping at the width
    check_counts(t, o, q)
    drop = np.unique(keys)[::5]
    t.erase(drop)
    o.erase(drop)
    t.insert(keys[:10_000])
    o.insert(keys[:10_000])
    check_counts(t, o, q)
    assert t.size() == o.size()


@pytest.mark.parametrize("kb", [4, 8])
def test_counting_region_split_unit_and_weighted(wc, kb):
    """Tables above 64 MiB with batches of >= 2^18 keys take the region-split insert; with
    no weights the split fills them with ones."""
    keys, q = zipf_keys(0xC1 + kb, kb, 1 << 20, 1 << 21)
    t = wc.CountingTable(kb, min_capacity=12_000_000 if kb == 4 else 6_000_000, options=wc.WC_OPT_OVERFLOW_BITS)
    assert t.info["table_bytes"] > (64 << 20)
    o = oracle.Counting(kb)
    t.insert(keys)
    o.insert(keys)
    # region-split inserts set exactly the overflow bits the stored keys' walks imply
    info = t.info
    bits = wc.api.wc_table_dump_overflow_bits(t.handle).view(np.uint8)[:info["windows"]]
    expect = oracle.overflow_bits_of(wc.api.wc_table_dump_slots(t.handle), info["windows"], info["window_width"],
                                     info["slot_bytes"], 0x5EED_C0DE, key_bytes=kb)
    np.testing.assert_array_equal(bits, expect)
    w = wc_inputs.uniform_u32(6, keys.size) if kb == 4 else wc_inputs.uniform_u64(6, keys.size)
    t.insert(keys, w)
    o.insert(keys, w)
    check_counts(t, o, q)
    assert t.size() == o.size()


def test_counting_sentinels_and_unsupported_calls(wc):
    t = wc.CountingTable(4, min_capacity=1000)
    assert t.insert(np.array([0, 0xFFFFFFFF, 7, 7], np.uint32)) == wc.WC_FLAG_INVALID_KEY  # no DUPLICATE
    out, found, _ = t.retrieve(np.array([7, 8], np.uint32))
    assert list(out) == [2, 0xFFFFFFFF] and list(found) == [1, 0]
    import torch
    offs = torch.empty(3, dtype=torch.int64, device="cuda")
    with pytest.raises(wc.WcError):
        wc.wc_count_values(t.handle, t.keys_dev(np.array([7, 8], np.uint32)), offs)


# ---- hash sets -----------------------------------------------------------------------------

SET_SHAPES = [(4, 8, 1), (4, 8, 2), (4, 16, 1), (4, 16, 2), (4, 16, 4), (4, 32, 4), (4, 32, 8),
              (8, 4, 1), (8, 4, 2), (8, 8, 1), (8, 8, 2), (8, 16, 2), (8, 16, 4), (8, 32, 4), (8, 32, 8)]


def check_set(t, o, q):
    found, _ = t.contains(q)
    ef, _ = o.contains(q)
    np.testing.assert_array_equal(found, ef)


@pytest.mark.parametrize("opt", [0, 1])
@pytest.mark.parametrize("kb,W,G", SET_SHAPES)
def test_hash_set_parity_every_shape(wc, kb, W, G, opt):
    """Key-only slots: inserts with repeats (DUPLICATE_KEY), membership, erase and
    re-insert over tombstones, at load 0.9; the slot dump passes the invariant checker."""
    n = 120_001
    keys = wc_inputs.distinct_u32(0x5E7 + W, n) if kb == 4 else wc_inputs.distinct_u64(0x5E7 + W, n)
    other = wc_inputs.distinct_u32(0x5E8 + W, n) if kb == 4 else wc_inputs.distinct_u64(0x5E8 + W, n)
    q = np.concatenate([keys, other[~np.isin(other, keys)]])
    t = wc.HashSetTable(kb, min_capacity=int(n / 0.9), window_width=W, seed=0x5E7, options=opt)
    for op in (wc.WC_OP_INSERT, wc.WC_OP_RETRIEVE, wc.WC_OP_ERASE):
        t.set_launch(op, G)
    o = oracle.HashSet(kb)
    assert t.insert(keys) == o.insert(keys) == 0
    assert t.insert(keys[:1000]) == o.insert(keys[:1000]) == oracle.FLAG_DUPLICATE_KEY
    check_set(t, o, q)
    t.erase(keys[::2])
    o.erase(keys[::2])
    check_set(t, o, q)
    assert t.insert(keys[::4]) == o.insert(keys[::4]) == 0
    check_set(t, o, q)
    assert t.size() == o.size()
    info = t.info
    bits = wc.api.wc_table_dump_overflow_bits(t.handle) if opt else None
    r = oracle.check_slots(wc.api.wc_table_dump_slots(t.handle), info["windows"], info["window_width"],
                           info["slot_bytes"], 0x5E7, True, bits, key_bytes=kb)
    assert r == {"live": o.size(), "dups": 0, "unreachable": 0}


@pytest.mark.parametrize("kb", [4, 8])
def test_hash_set_region_split_and_sentinels(wc, kb):
    n = 1 << 21
    keys = wc_inputs.distinct_u32(0x5E9, n) if kb == 4 else wc_inputs.distinct_u64(0x5E9, n)
    t = wc.HashSetTable(kb, min_capacity=24_000_000 if kb == 4 else 12_000_000)
    assert t.info["table_bytes"] > (64 << 20)
    o = oracle.HashSet(kb)
    assert t.insert(keys) == o.insert(keys) == 0
    assert t.size() == n
    q = np.concatenate([keys[::7], (wc_inputs.distinct_u32(0x5EA, 1 << 18) if kb == 4
                                    else wc_inputs.distinct_u64(0x5EA, 1 << 18))])
    check_set(t, o, q)
    top = (1 << (8 * kb)) - 1
    assert t.insert(np.array([0, top, 5], dtype=np.uint64)) == wc.WC_FLAG_INVALID_KEY
    found, f = t.contains(np.array([0, top, 5], dtype=np.uint64))
    assert list(found) == [0, 0, 1] and f == wc.WC_FLAG_INVALID_KEY
    import torch
    with pytest.raises(wc.WcError):  # no values in a set
        k = t.keys_dev(np.array([5], dtype=np.uint64))
        wc.wc_retrieve(t.handle, k, torch.empty_like(k), None)


# ---- Bloom filters -------------------------------------------------------------------------

def bloom_fp_formula(n, bits, k):
    """Blocked-filter false-positive rate: average over blocks (Poisson key counts with mean
    256 n / bits) of (1 - (1 - 1/256)^(k x))^k."""
    import math
    lam = 256.0 * n / bits
    p, total, x = math.exp(-lam), 0.0, 0
    while x < lam + 20 * math.sqrt(lam + 1) + 20:
        total += p * (1.0 - (1.0 - 1.0 / 256) ** (k * x)) ** k
        x += 1
        p *= lam / x
    return total


@pytest.mark.parametrize("kb,k,bpk", [(4, 8, 10), (8, 4, 8), (4, 1, 16), (8, 16, 24), (4, 7, 12)])
def test_bloom_filter_parity_and_false_positive_rate(wc, kb, k, bpk):
    """The filter sets exactly the bits of the documented definition (membership equals
    the oracle's bit for bit), never reports an inserted key absent, and its false-positive
    rate on absent keys matches the blocked-filter formula."""
    n = 200_003
    keys = wc_inputs.distinct_u32(0xB1 + k, n) if kb == 4 else wc_inputs.distinct_u64(0xB1 + k, n)
    absent = wc_inputs.distinct_u32(0xB2 + k, 400_000) if kb == 4 else wc_inputs.distinct_u64(0xB2 + k, 400_000)
    absent = absent[~np.isin(absent, keys)]
    t = wc.BloomFilterTable(kb, bits=n * bpk, k=k, seed=0xB100)
    assert t.info["window_width"] == k
    blocks = t.info["windows"]
    o = oracle.BloomFilter(kb, blocks, k, 0xB100)
    half = n // 2
    assert t.insert(keys[:half]) == o.insert(keys[:half]) == 0
    assert t.insert(keys[half:]) == o.insert(keys[half:]) == 0
    assert t.size() == n
    q = np.concatenate([keys, absent])
    found, _ = t.contains(q)
    ef, _ = o.contains(q)
    np.testing.assert_array_equal(found, ef)
    assert found[:n].all()  # no false negatives
    fp = found[n:].mean()
    expect = bloom_fp_formula(n, blocks * 256, k)
    assert abs(fp - expect) <= 0.1 * expect + 3 * np.sqrt(expect / absent.size), (fp, expect)


def test_bloom_filter_calls_and_sentinels(wc):
    t = wc.BloomFilterTable(8, bits=1 << 16, k=6)
    top = 2 ** 64 - 1
    assert t.insert(np.array([0, top, 9], dtype=np.uint64)) == wc.WC_FLAG_INVALID_KEY
    found, f = t.contains(np.array([0, top, 9], dtype=np.uint64))
    assert list(found) == [0, 0, 1] and f == wc.WC_FLAG_INVALID_KEY
    with pytest.raises(wc.WcError):  # bits are shared between keys: no erase
        t.erase(np.array([9], dtype=np.uint64))
    with pytest.raises(wc.WcError):
        wc.BloomFilterTable(4, bits=1024, k=17)
    t.clear()
    found, _ = t.contains(np.array([9], dtype=np.uint64))
    assert list(found) == [0]
