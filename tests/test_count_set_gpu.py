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
