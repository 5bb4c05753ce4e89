"""Host copies of GPU tables: slot dumps checked by the slot-dump invariant checker (no
key twice in a single-value table or key store, no live key behind a window holding an
empty slot on its own sequence), snapshots restored into a fresh table, the folded status
check, and the out-of-memory paths through the allocation-failure hook."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import wc_inputs

pytestmark = pytest.mark.gpu

SEED = 0x5EED


@pytest.fixture(scope="module")
def wc():
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    return wc


def checked(wc, t, unique):
    info = t.info
    dump = wc.api.wc_table_dump_slots(t.handle)
    assert dump.size == info["table_bytes"]
    r = oracle.check_slots(dump, info["windows"], info["window_width"], info["slot_bytes"], SEED, unique)
    if info["options"] & 1:  # overflow bits: lookups also stop at a window whose bit is clear
        bits = wc.api.wc_table_dump_overflow_bits(t.handle)
        rb = oracle.check_slots(dump, info["windows"], info["window_width"], info["slot_bytes"], SEED, unique, bits)
        assert rb == r
    return r


@pytest.mark.parametrize("opt", [0, 1])
@pytest.mark.parametrize("kb,W", [(4, 4), (4, 8), (4, 32), (8, 2), (8, 4), (8, 16)])
def test_single_value_dump_invariants_after_inserts_erases_reinserts(wc, kb, W, opt):
    n = 60_000
    keys = wc_inputs.distinct_u32(11, n) if kb == 4 else wc_inputs.distinct_u64(11, n)
    vals = keys.copy()
    t = wc.SingleValueTable(kb, kb, min_capacity=int(n / 0.9), window_width=W, seed=SEED, options=opt)
    t.insert(keys, vals)
    t.erase(keys[::3])
    t.insert(keys[::6], vals[::6])  # half of the erased keys come back, over tombstones
    r = checked(wc, t, True)
    assert r["dups"] == 0 and r["unreachable"] == 0
    assert r["live"] == t.size() == n - len(keys[::3]) + len(keys[::6])


@pytest.mark.parametrize("kb", [4, 8])
def test_oa_multi_value_dump_invariants(wc, kb):
    d = wc_inputs.mv_zipf_u64(21, 1 << 12, 80_000, 16)
    keys = d["keys"] if kb == 8 else ((d["keys"] & np.uint64(0x7FFFFFFF)) | np.uint64(1)).astype(np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32 if kb == 4 else np.uint64)
    t = wc.MultiValueOATable(kb, kb, min_capacity=100_000, seed=SEED)
    t.insert(keys, vals)
    t.erase(np.unique(keys)[::4])
    t.insert(keys[:20_000], vals[:20_000])
    r = checked(wc, t, False)
    assert r["unreachable"] == 0 and r["live"] == t.size()


def test_bucket_multi_value_key_store_dump_invariants(wc):
    d = wc_inputs.mv_zipf_u64(22, 1 << 14, 200_000, 16)
    t = wc.MultiValueTable(8, 4, min_capacity=int((1 << 14) / 0.8), value_pool_capacity=1 << 19, seed=SEED)
    t.insert(d["keys"], d["values"])
    t.erase(np.unique(d["keys"])[::5])
    r = checked(wc, t, True)
    assert r["dups"] == 0 and r["unreachable"] == 0 and r["live"] == t.num_keys()


def test_snapshot_restore_single_value(wc):
    n = 50_000
    d = wc_inputs.sv_insert_retrieve_u32(31, n, n // 2, n // 2)
    t = wc.SingleValueTable(4, 4, min_capacity=int(n / 0.8), seed=SEED)
    t.insert(d["keys"], d["values"])
    before = t.retrieve(d["queries"])
    snap = wc.api.wc_table_snapshot(t.handle)
    assert snap.size == wc.api.wc_table_snapshot_bytes(t.handle)
    t.erase(d["keys"][: n // 2])
    t.insert(wc_inputs.distinct_u32(32, 1000) | np.uint32(1 << 31), np.zeros(1000, np.uint32))
    u = wc.SingleValueTable(4, 4, min_capacity=int(n / 0.8), seed=SEED)
    wc.api.wc_table_restore(u.handle, snap)
    after = u.retrieve(d["queries"])
    assert u.size() == n
    np.testing.assert_array_equal(after[0], before[0])
    np.testing.assert_array_equal(after[1], before[1])
    # a table of another geometry or seed refuses the snapshot and is left unchanged
    for other in (wc.SingleValueTable(4, 4, min_capacity=n, seed=SEED),
                  wc.SingleValueTable(4, 4, min_capacity=int(n / 0.8), seed=SEED + 1)):
        with pytest.raises(wc.WcError):
            wc.api.wc_table_restore(other.handle, snap)
        assert other.size() == 0


def test_snapshot_restore_bucket_multi_value(wc):
    d = wc_inputs.mv_zipf_u64(33, 1 << 12, 100_000, 1 << 8)
    kw = dict(min_capacity=int((1 << 12) / 0.8), value_pool_capacity=1 << 18, seed=SEED)
    t = wc.MultiValueTable(8, 4, **kw)
    t.insert(d["keys"], d["values"])
    offs, _ = t.count_values(d["queries"])
    vals, _ = t.retrieve_multi(d["queries"], offs)
    snap = wc.api.wc_table_snapshot(t.handle)
    t.insert(d["keys"][:5000], d["values"][:5000])  # diverge after the snapshot
    u = wc.MultiValueTable(8, 4, **kw)
    wc.api.wc_table_restore(u.handle, snap)
    offs2, _ = u.count_values(d["queries"])
    np.testing.assert_array_equal(offs2, offs)
    vals2, _ = u.retrieve_multi(d["queries"], offs2)
    np.testing.assert_array_equal(oracle.sorted_segments(vals2, offs2), oracle.sorted_segments(vals, offs))
    assert u.size() == 100_000
    # the restored table keeps working: further inserts append after the restored pool
    u.insert(d["keys"][:5000], d["values"][:5000])
    offs3, _ = u.count_values(d["queries"])
    assert int(offs3[-1]) == 105_000


def test_check_status_folds_flags(wc):
    t = wc.SingleValueTable(4, 4, min_capacity=64, window_width=8, seed=SEED)
    code, flags = wc.api.wc_check_status(t.handle)
    assert (code, flags) == (0, 0)
    k = np.arange(1, 50, dtype=np.uint32)
    wc.api.wc_insert(t.handle, t.keys_dev(np.concatenate([k, k[:3]])), t.values_dev(np.zeros(52, np.uint32)))
    code, flags = wc.api.wc_check_status(t.handle)
    assert code == 0 and flags == wc.WC_FLAG_DUPLICATE_KEY  # a warning, not an error
    wc.api.wc_insert(t.handle, t.keys_dev(np.arange(100, 300, dtype=np.uint32)),
                     t.values_dev(np.zeros(200, np.uint32)))
    code, flags = wc.api.wc_check_status(t.handle)
    assert code == 3 and flags & wc.WC_FLAG_PROBE_LIMIT  # WC_ERR_FULL
    assert wc.api.wc_check_status(t.handle) == (0, 0)  # cleared


def test_injected_allocation_failures(wc):
    api = wc.api
    api.wc_debug_fail_allocations(1)
    with pytest.raises(wc.WcError) as e:
        wc.SingleValueTable(4, 4, min_capacity=1000)
    assert e.value.code == 2  # WC_ERR_OUT_OF_MEMORY
    t = wc.SingleValueTable(4, 4, min_capacity=40_000_000, seed=SEED, options=1)  # next create works
    n = 1 << 20
    keys = wc_inputs.distinct_u32(41, n)
    # the region-split insert's scratch allocation fails: error, table untouched
    api.wc_debug_fail_allocations(1)
    with pytest.raises(wc.WcError) as e:
        api.wc_insert(t.handle, t.keys_dev(keys), t.values_dev(keys))
    assert e.value.code == 2
    assert t.size() == 0
    api.wc_debug_fail_allocations(0)
    t.insert(keys, keys)
    assert t.size() == n
    r = checked(wc, t, True)
    assert r["live"] == n and r["dups"] == 0 and r["unreachable"] == 0
