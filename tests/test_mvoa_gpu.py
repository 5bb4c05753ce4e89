"""Open-addressing multi-value table (WC_MULTI_VALUE_OA) against the CPU oracle: exact
counts and offsets, equal sorted per-query value multisets (Sec. IV-B4), erase of every
copy (Sec. IV-B5) and the Sec. V-C uniform-r invariant.  Slot positions are never
compared: which slot a pair lands in depends on the order concurrent inserts claim them."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import wc_inputs
from tests.golden_fixtures import run_mv

pytestmark = pytest.mark.gpu

P32_SHAPES = [(4, 1), (4, 2), (8, 1), (8, 2), (16, 2), (16, 4), (32, 4), (32, 8)]
P64_SHAPES = [(2, 1), (4, 1), (4, 2), (8, 2), (8, 4), (16, 4), (16, 8)]


@pytest.fixture(scope="module")
def wc():
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    return wc


def make_oa(wc, kb, cap, W=0, G=None, seed=0x0A0A):
    t = wc.MultiValueOATable(kb, kb, min_capacity=cap, window_width=W, seed=seed)
    if G is not None:
        for op in (wc.WC_OP_INSERT, wc.WC_OP_RETRIEVE, wc.WC_OP_COUNT, wc.WC_OP_ERASE):
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


@pytest.mark.parametrize("kb", [4, 8])
def test_golden_mv_worked_example_oa(wc, kb):
    from tests.test_mv_gpu import _Adapter
    assert run_mv("mv_ops.txt", lambda: _Adapter(make_oa(wc, kb, 256))) >= 8


def _zipf_case(seed, kb, uni, n_ins, n_abs):
    d = wc_inputs.mv_zipf_u64(seed, uni, n_ins, n_abs)
    if kb == 4:
        for f in ("keys", "queries"):
            d[f] = ((d[f] & np.uint64(0x7FFFFFFF)) | np.uint64(1)).astype(np.uint32)
        d["values"] = d["values"].astype(np.uint32)
    else:
        d["values"] = d["values"].astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    return d


@pytest.mark.parametrize("kb,W,G", [(4,) + s for s in P32_SHAPES] + [(8,) + s for s in P64_SHAPES])
def test_oa_zipf_parity_every_shape(wc, kb, W, G):
    """Zipf multiplicities (a few keys with thousands of copies, most with one), all
    four operations on the shape; 100k pairs at load ~0.8 span many tiles and a ragged
    tail of the last warp's range."""
    n_ins = 100_003
    d = _zipf_case(0x0A5E + kb * 131 + W * 7 + G, kb, 1 << 13, n_ins, 1 << 11)
    t = make_oa(wc, kb, int(n_ins / 0.8), W, G)
    o = oracle.MultiValue(kb, kb)
    assert t.insert(d["keys"], d["values"]) == 0
    o.insert(d["keys"], d["values"])
    assert t.size() == o.size() == n_ins
    assert t.num_keys() == o.num_keys()
    check_queries(t, o, d["queries"])
    drop = np.unique(d["keys"])[::3]
    t.erase(drop)
    o.erase(drop)
    assert t.size() == o.size()
    assert t.num_keys() == o.num_keys()
    check_queries(t, o, d["queries"])


@pytest.mark.parametrize("kb", [4, 8])
def test_oa_random_ops_reuse_tombstones(wc, kb):
    """Interleaved inserts and erases: erased copies leave tombstones that later inserts
    take again (Sec. IV-B5); every step matches the oracle."""
    rng = np.random.default_rng(0x70B + kb)
    top = (1 << 31) - 2 if kb == 4 else 2 ** 62
    universe = np.unique(rng.integers(1, top, 3000, dtype=np.uint64))
    if kb == 4:
        universe = universe.astype(np.uint32)
    t = make_oa(wc, kb, 60_000)
    o = oracle.MultiValue(kb, kb)
    vmax = (1 << (8 * kb)) - 1
    for step in range(12):
        m = int(rng.integers(1, 6000))
        ks = universe[np.minimum(rng.zipf(1.5, m), universe.size) - 1]
        vs = rng.integers(0, vmax, m, dtype=np.uint64, endpoint=True)
        if kb == 4:
            vs = vs.astype(np.uint32)
        t.insert(ks, vs)
        o.insert(ks, vs)
        if step % 3 == 2:
            drop = universe[rng.integers(0, universe.size, 400)]
            t.erase(drop)
            o.erase(drop)
        assert t.size() == o.size()
        assert t.num_keys() == o.num_keys()
        check_queries(t, o, universe)


@pytest.mark.parametrize("kb", [4, 8])
def test_oa_paper_invariant_uniform_r(wc, kb):
    """Sec. V-C: n keys from 1..n/r inserted at load 0.8, queried over 1..n, return
    exactly n values, each under the key it was inserted with."""
    n = 1 << 17
    for r in (1, 2, 8, 32, 256):
        d = wc_inputs.mv_uniform_r(700 + r, n, r)
        keys = d["keys"].astype(np.uint32) if kb == 4 else d["keys"]
        q = d["queries"].astype(np.uint32) if kb == 4 else d["queries"]
        vals_in = d["values"] if kb == 4 else d["values"].astype(np.uint64)
        t = make_oa(wc, kb, int(n / 0.8))
        assert t.insert(keys, vals_in) == 0
        assert t.size() == n
        offs, _ = t.count_values(q)
        assert int(offs[-1]) == n
        vals, _ = t.retrieve_multi(q, offs)
        np.testing.assert_array_equal(np.sort(vals.astype(np.int64)), np.arange(n))
        seg = np.repeat(np.arange(n), np.diff(offs.astype(np.int64)))
        np.testing.assert_array_equal(q[seg], keys[vals.astype(np.int64)])
        t.close()


def test_oa_hot_key_spans_many_windows(wc):
    """One key with 4096 copies occupies 512 windows of W = 8; every copy is counted and
    copied by the window-parallel walk."""
    n_hot = 4096
    keys = np.concatenate([np.full(n_hot, 777, dtype=np.uint32), np.arange(1000, 9000, dtype=np.uint32)])
    vals = np.arange(keys.size, dtype=np.uint32)
    t = make_oa(wc, 4, 16_384, W=8)
    o = oracle.MultiValue(4, 4)
    t.insert(keys, vals)
    o.insert(keys, vals)
    check_queries(t, o, np.array([777, 1000, 5, 8999, 777], dtype=np.uint32))
    assert t.num_keys() == o.num_keys() == 8001


def test_oa_sentinels_empty_overfull_and_unsupported(wc):
    t = make_oa(wc, 8, 64, W=8)
    f = t.insert(np.array([0, 2 ** 64 - 1, 5], dtype=np.uint64), np.array([1, 2, 4], dtype=np.uint64))
    assert f == wc.WC_FLAG_INVALID_KEY
    offs, f = t.count_values(np.array([0, 5, 6, 2 ** 64 - 1], dtype=np.uint64))
    assert list(offs) == [0, 0, 1, 1, 1] and f == wc.WC_FLAG_INVALID_KEY
    offs, _ = t.count_values(np.array([], dtype=np.uint64))
    assert list(offs) == [0]
    # 88 slots (p = 11 windows of 8): 100 more pairs cannot all fit
    cap = t.capacity
    assert cap == 88
    ks = np.arange(10, 110, dtype=np.uint64)
    f = t.insert(ks, ks * np.uint64(3))
    assert f & wc.WC_FLAG_PROBE_LIMIT
    assert t.size() == cap
    q = np.concatenate([[5], ks]).astype(np.uint64)
    offs, _ = t.count_values(q)
    assert int(offs[-1]) == cap
    vals, _ = t.retrieve_multi(q, offs)
    stored = np.repeat(q, np.diff(offs.astype(np.int64)))
    np.testing.assert_array_equal(vals[1:], stored[1:] * np.uint64(3))
    assert abs(t.load_factor() - 1.0) < 1e-12
    # single-value retrieve does not exist for a multi-value table
    with pytest.raises(RuntimeError):
        from paper_2009_07914_gb300 import api
        import torch
        k = torch.ones(4, dtype=torch.int64, device="cuda")
        api.wc_retrieve(t.handle, k, torch.empty_like(k), None)
    # erase everything: the table is empty again, tombstones remain claimable
    t.erase(q)
    assert t.size() == 0 and t.num_keys() == 0
    f = t.insert(ks[:60], ks[:60])
    assert f == 0 and t.size() == 60


@pytest.mark.parametrize("kb", [4, 8])
def test_oa_region_split_insert_parity(wc, kb):
    """A table above 64 MiB and a batch of >= 2^18 pairs take the region-split insert
    (automatically; a small table is forced onto it with 1 MiB regions); counts and
    value multisets still equal the oracle's, also on a repeat insert."""
    uni, n = 1 << 19, 1 << 21
    d = _zipf_case(0x5B11A + kb, kb, uni, n, 1 << 14)
    t = make_oa(wc, kb, 12_000_000 if kb == 4 else 6_000_000)
    assert t.info["table_bytes"] > (64 << 20)
    o = oracle.MultiValue(kb, kb)
    for rep in range(2):
        assert t.insert(d["keys"], d["values"]) == 0
        o.insert(d["keys"], d["values"])
        assert t.size() == o.size() == (rep + 1) * n
    assert t.num_keys() == o.num_keys()
    q = d["queries"][wc_inputs.shuffle_index(5, d["queries"].size)[:100_000]]
    check_queries(t, o, q)
    small = make_oa(wc, kb, 150_000)
    small.set_launch(wc.WC_OP_INSERT, small.info["window_width"] // (4 if kb == 4 else 2) or 1,
                     scheme=wc.WC_SCHEME_BLOCKED, region_mib=1)
    o2 = oracle.MultiValue(kb, kb)
    m = 100_000
    assert small.insert(d["keys"][:m], d["values"][:m]) == 0
    o2.insert(d["keys"][:m], d["values"][:m])
    assert small.size() == m
    check_queries(small, o2, q[:20_000])
