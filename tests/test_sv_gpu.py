"""Single-value GPU path against the CPU oracle, element by element (calls go through the
C ABI via the ctypes binding).  Sizes span many warps' ranges with ragged tails."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import wc_inputs
from tests.golden_fixtures import run_sv

pytestmark = pytest.mark.gpu

W_G_P32 = [(4, 1), (4, 2), (4, 4), (8, 1), (8, 2), (8, 4), (8, 8), (16, 1), (16, 2), (16, 4), (16, 8), (16, 16),
           (32, 4), (32, 8), (32, 16), (32, 32)]
W_G_P64 = [(2, 1), (2, 2), (4, 1), (4, 2), (4, 4), (8, 1), (8, 2), (8, 4), (8, 8), (16, 4), (16, 8), (16, 16)]


@pytest.fixture(scope="module")
def wc():
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    return wc


def make_sv(wc, kb, vb, cap, W=0, G=None, seed=0x1234, scheme=0, region_mib=0, options=0):
    t = wc.SingleValueTable(kb, vb, min_capacity=cap, window_width=W, seed=seed, options=options)
    if G is not None:
        for op in (wc.WC_OP_INSERT, wc.WC_OP_RETRIEVE, wc.WC_OP_ERASE):
            t.set_launch(op, G)
    if scheme:
        g = G if G is not None else wc.wc_table_get_launch(t.handle, wc.WC_OP_INSERT)["group_size"]
        t.set_launch(wc.WC_OP_INSERT, g, scheme=scheme, region_mib=region_mib)
    return t


def check_retrieve(t, o, keys):
    out, found, flags = t.retrieve(keys)
    eo, ef, efl = o.retrieve(keys)
    np.testing.assert_array_equal(found, ef)
    np.testing.assert_array_equal(out, eo)
    assert flags == efl


class _Adapter:
    """Oracle-shaped wrapper over a GPU table for the golden fixtures."""

    def __init__(self, t):
        self.t = t

    def insert(self, k, v):
        return self.t.insert(k, v)

    def erase(self, k):
        return self.t.erase(k)

    def retrieve(self, k):
        return self.t.retrieve(k)

    def size(self):
        return self.t.size()


def test_golden_sv_worked_example_gpu(wc):
    assert run_sv("sv_ops.txt", lambda: _Adapter(make_sv(wc, 4, 4, 64))) >= 10


@pytest.mark.parametrize("W,G", W_G_P32)
def test_sv_u32_parity_every_shape(wc, W, G):
    n = 100_003
    d = wc_inputs.sv_insert_retrieve_u32(0x57C00001 + W * 64 + G, n, n // 2, 50_001)
    t = make_sv(wc, 4, 4, int(n / 0.9) + 1, W, G)
    o = oracle.SingleValue(4, 4)
    assert t.insert(d["keys"], d["values"]) == o.insert(d["keys"], d["values"]) == 0
    assert t.size() == o.size() == n
    check_retrieve(t, o, d["queries"])
    # erase a seeded half, retrieve everything again
    drop = d["keys"][wc_inputs.shuffle_index(3, n)[: n // 2]]
    assert t.erase(drop) == o.erase(drop)
    assert t.size() == o.size()
    check_retrieve(t, o, d["queries"])
    # re-insert the erased keys with new values: tombstones are reused, nothing doubles
    newv = wc_inputs.uniform_u32(77, drop.size)
    assert t.insert(drop, newv) == o.insert(drop, newv)
    assert t.size() == o.size() == n
    check_retrieve(t, o, np.concatenate([d["keys"], d["queries"]]))
    # overwrite present keys: duplicate warning, new values
    upd = d["keys"][:1000]
    v2 = wc_inputs.uniform_u32(78, 1000)
    assert t.insert(upd, v2) == o.insert(upd, v2) == oracle.FLAG_DUPLICATE_KEY
    check_retrieve(t, o, d["keys"])
    assert t.size() == n


@pytest.mark.parametrize("W,G", W_G_P64)
def test_sv_u64_parity_every_shape(wc, W, G):
    n = 60_001
    keys = wc_inputs.distinct_u64(0x57C00003 + W * 64 + G, n + 30_000)
    vals = wc_inputs.uniform_u64(5, n)
    t = make_sv(wc, 8, 8, int(n / 0.9) + 1, W, G)
    o = oracle.SingleValue(8, 8)
    assert t.insert(keys[:n], vals) == o.insert(keys[:n], vals) == 0
    q = keys[wc_inputs.shuffle_index(9, keys.size)]
    check_retrieve(t, o, q)
    drop = keys[: n // 3]
    t.erase(drop)
    o.erase(drop)
    assert t.size() == o.size()
    check_retrieve(t, o, q)
    t.insert(drop, vals[: n // 3] ^ np.uint64(0xABCDEF))
    o.insert(drop, vals[: n // 3] ^ np.uint64(0xABCDEF))
    check_retrieve(t, o, q)
    assert t.size() == o.size() == n


@pytest.mark.parametrize("opt", [0, 1])
@pytest.mark.parametrize("kb", [4, 8])
def test_sv_random_op_sequences(wc, kb, opt):
    """Small key universe: heavy reuse of tombstones, duplicates inside batches (with and
    without overflow bits)."""
    rng = np.random.default_rng(kb)
    top = (1 << (8 * kb)) - 1
    universe = np.unique(rng.integers(1, min(top, 2 ** 62), 3000, dtype=np.uint64))
    t = make_sv(wc, kb, kb, 4096, options=opt)
    o = oracle.SingleValue(kb, kb)
    for step in range(40):
        m = int(rng.integers(1, 2000))
        ks = np.unique(universe[rng.integers(0, universe.size, m)])  # unique inside a batch
        rng.shuffle(ks)
        if step % 3 == 2:
            assert t.erase(ks) == o.erase(ks)
        else:
            vs = rng.integers(0, top, ks.size, dtype=np.uint64, endpoint=True)
            assert t.insert(ks, vs) == o.insert(ks, vs)
        assert t.size() == o.size()
        check_retrieve(t, o, universe)


def test_duplicates_inside_one_batch_store_one_of_their_values(wc):
    keys = np.array([5, 9, 5, 5, 9, 11] * 1000, dtype=np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32)
    t = make_sv(wc, 4, 4, 1024)
    flags = t.insert(keys, vals)
    assert flags & wc.WC_FLAG_DUPLICATE_KEY
    assert t.size() == 3
    out, found, _ = t.retrieve(np.array([5, 9, 11], dtype=np.uint32))
    assert found.all()
    for k, v in zip((5, 9, 11), out):
        assert int(v) in set(vals[keys == k].tolist())


def test_sentinels_and_empty_batches(wc):
    t = make_sv(wc, 4, 4, 1024)
    assert t.insert(np.array([], dtype=np.uint32), np.array([], dtype=np.uint32)) == 0
    f = t.insert(np.array([0, 0xFFFFFFFF, 7], dtype=np.uint32), np.array([1, 2, 3], dtype=np.uint32))
    assert f == wc.WC_FLAG_INVALID_KEY
    assert t.size() == 1
    out, found, f = t.retrieve(np.array([0, 7, 0xFFFFFFFF], dtype=np.uint32))
    assert list(found) == [0, 1, 0] and int(out[1]) == 3 and int(out[0]) == 0xFFFFFFFF
    assert f == wc.WC_FLAG_INVALID_KEY


@pytest.mark.parametrize("kb", [4, 8])
def test_overfull_table_reports_probe_limit_without_hanging(wc, kb):
    t = make_sv(wc, kb, kb, 64)  # 64 slots requested -> a few windows
    cap = t.capacity
    keys = (wc_inputs.distinct_u32(1, cap + 50) if kb == 4 else wc_inputs.distinct_u64(1, cap + 50))
    flags = t.insert(keys, keys)
    assert flags & wc.WC_FLAG_PROBE_LIMIT
    assert t.size() == cap  # every slot filled, the rest rejected
    out, found, _ = t.retrieve(keys)
    assert int(found.sum()) == cap
    assert (out[found == 1] == keys[found == 1]).all()


def test_load_factor_and_clear(wc):
    n = 50_000
    d = wc_inputs.sv_insert_retrieve_u32(21, n, 0, 0)
    t = make_sv(wc, 4, 4, int(n / 0.8))
    t.insert(d["keys"], d["values"])
    assert abs(t.load_factor() - n / t.capacity) < 1e-12
    t.clear()
    assert t.size() == 0
    _, found, _ = t.retrieve(d["keys"])
    assert not found.any()


@pytest.mark.parametrize("W", [4, 8, 16, 32])
def test_window_counts_within_uniform_hashing_bound(wc, W):
    """Hash quality (not parity): a full table at alpha = 0.9 answers every query; the
    table's retrieve finds all keys -- probing never gives up early."""
    n = 200_000
    d = wc_inputs.sv_insert_retrieve_u32(31 + W, n, n, n)
    t = make_sv(wc, 4, 4, int(n / 0.9) + 1, W)
    assert t.insert(d["keys"], d["values"]) == 0
    out, found, _ = t.retrieve(d["queries"])
    assert int(found.sum()) == n


@pytest.mark.parametrize("kb,W,G", [(4, 4, 1), (4, 8, 2), (4, 16, 4), (4, 32, 8), (8, 4, 2), (8, 8, 4)])
def test_blocked_insert_scheme_parity(wc, kb, W, G):
    """Region-split (blocked) inserts give the same table contents as the oracle,
    including tombstone reuse after erases and duplicate overwrites."""
    n = 1_000_003
    if kb == 4:
        d = wc_inputs.sv_insert_retrieve_u32(0xB10C + W + G, n, n // 2, 300_000)
        keys, vals, q = d["keys"], d["values"], d["queries"]
    else:
        allk = wc_inputs.distinct_u64(0xB10C + W + G, n + 300_000)
        keys, vals = allk[:n], wc_inputs.uniform_u64(3, n)
        q = allk[wc_inputs.shuffle_index(4, allk.size)]
    t = make_sv(wc, kb, kb, int(n / 0.9) + 1, W, G, scheme=wc.WC_SCHEME_BLOCKED, region_mib=1)
    o = oracle.SingleValue(kb, kb)
    assert t.insert(keys, vals) == o.insert(keys, vals) == 0
    assert t.size() == n
    check_retrieve(t, o, q)
    drop = keys[: n // 3]
    t.erase(drop)
    o.erase(drop)
    back = np.concatenate([drop[::2], keys[n // 3: n // 3 + 1000]])  # re-insert + overwrite
    bv = (vals[: back.size] ^ 0x5A).astype(vals.dtype)
    assert t.insert(back, bv) == o.insert(back, bv) == oracle.FLAG_DUPLICATE_KEY
    assert t.size() == o.size()
    check_retrieve(t, o, q)


def test_blocked_insert_auto_scheme_on_large_table(wc):
    """AUTO picks the blocked scheme for big batches into tables above 64 MiB."""
    n = 1 << 23
    d = wc_inputs.sv_insert_retrieve_u32(0xA070, n, 1 << 20, 1 << 20)
    t = make_sv(wc, 4, 4, int(n / 0.9) + 1)
    assert t.info["table_bytes"] > (64 << 20)
    assert t.insert(d["keys"], d["values"]) == 0
    assert t.size() == n
    out, found, _ = t.retrieve(d["queries"])
    pres = d["q_src"] >= 0
    assert found[pres].all() and not found[~pres].any()
    np.testing.assert_array_equal(out[pres], d["values"][d["q_src"][pres]])


@pytest.mark.parametrize("kb,W,G", [(4, 4, 1), (4, 8, 2), (4, 16, 4), (4, 32, 8), (8, 2, 1), (8, 4, 2), (8, 8, 4)])
def test_blocked_retrieve_scheme_parity(wc, kb, W, G):
    """Region-split (blocked) retrieve: split by table region, probe in region order,
    split the results by output position, place them -- same values and found mask as
    the oracle, with absent keys, repeated queries, sentinels and a ragged tail; also
    without a found mask and for batches of 1 and 0 queries."""
    n = 700_001
    if kb == 4:
        d = wc_inputs.sv_insert_retrieve_u32(0xB10D + W + G, n, n // 2, 400_000)
        keys, vals, q = d["keys"], d["values"], d["queries"]
    else:
        allk = wc_inputs.distinct_u64(0xB10D + W + G, n + 400_000)
        keys, vals = allk[:n], wc_inputs.uniform_u64(5, n)
        q = allk[wc_inputs.shuffle_index(6, allk.size)]
    q = np.concatenate([q, q[:5000], np.array([0, 2 ** (8 * kb) - 1] * 3, dtype=q.dtype)])
    t = make_sv(wc, kb, kb, int(n / 0.9) + 1, W, G)
    t.set_launch(wc.WC_OP_RETRIEVE, G, scheme=wc.WC_SCHEME_BLOCKED, region_mib=1)
    o = oracle.SingleValue(kb, kb)
    t.insert(keys, vals)
    o.insert(keys, vals)
    check_retrieve(t, o, q)
    t.erase(keys[::4])
    o.erase(keys[::4])
    check_retrieve(t, o, q)
    # without the found mask
    import torch
    qd = t.keys_dev(q)
    out = torch.empty(q.size, dtype=torch.int32 if kb == 4 else torch.int64, device=qd.device)
    wc.wc_retrieve(t.handle, qd, out, None)
    assert wc.wc_get_status(t.handle, True) == oracle.FLAG_INVALID_KEY  # the sentinel queries
    eo, _, _ = o.retrieve(q)
    np.testing.assert_array_equal(out.cpu().numpy().view(eo.dtype), eo)
    for m in (1, 0):
        check_retrieve(t, o, q[:m])


def assert_exact_overflow_bits(wc, t, seed, kb):
    """After inserts alone, the table's overflow bits are exactly the tag bits of the
    windows each stored key walked past (derived from the slot dump by the oracle)."""
    info = t.info
    p = info["windows"]
    bits = wc.wc_table_dump_overflow_bits(t.handle).view(np.uint8)[:p]
    expect = oracle.overflow_bits_of(wc.api.wc_table_dump_slots(t.handle), p, info["window_width"],
                                     info["slot_bytes"], seed, key_bytes=kb)
    np.testing.assert_array_equal(bits, expect)
    assert np.count_nonzero(bits) > p // 10  # high load: many windows were walked past


@pytest.mark.parametrize("kb,W,G", [(4, 4, 1), (4, 8, 2), (4, 16, 4), (4, 32, 8), (8, 2, 1), (8, 4, 2), (8, 8, 4),
                                    (8, 16, 8)])
def test_overflow_bits_parity(wc, kb, W, G):
    """WC_OPT_OVERFLOW_BITS: lookups and erases that stop at a window with a clear overflow
    bit give the oracle's results at load 0.95, through erases (tombstones), re-inserts,
    overwrites and the blocked insert and retrieve schemes; the bits exist only on request
    and only for single-value tables."""
    n = 400_003
    if kb == 4:
        d = wc_inputs.sv_insert_retrieve_u32(0x0F1 + W + G, n, n // 2, 300_000)
        keys, vals, q = d["keys"], d["values"], d["queries"]
    else:
        allk = wc_inputs.distinct_u64(0x0F1 + W + G, n + 300_000)
        keys, vals = allk[:n], wc_inputs.uniform_u64(7, n)
        q = allk[wc_inputs.shuffle_index(8, allk.size)]
    t = make_sv(wc, kb, kb, int(n / 0.95) + 1, W, G, options=wc.WC_OPT_OVERFLOW_BITS)
    assert t.info["options"] == wc.WC_OPT_OVERFLOW_BITS
    o = oracle.SingleValue(kb, kb)
    assert t.insert(keys, vals) == o.insert(keys, vals) == 0
    check_retrieve(t, o, q)
    assert_exact_overflow_bits(wc, t, 0x1234, kb)
    drop = keys[: n // 2]
    assert t.erase(drop) == o.erase(drop)
    assert t.erase(drop[:1000]) == o.erase(drop[:1000])  # absent now: stops early, no-op
    assert t.size() == o.size()
    check_retrieve(t, o, q)
    back = np.concatenate([drop[::3], keys[n // 2: n // 2 + 5000]])
    bv = (vals[: back.size] ^ 0x33).astype(vals.dtype)
    assert t.insert(back, bv) == o.insert(back, bv)
    check_retrieve(t, o, q)
    for op in (wc.WC_OP_INSERT, wc.WC_OP_RETRIEVE):
        t.set_launch(op, G, scheme=wc.WC_SCHEME_BLOCKED, region_mib=1)
    more = q[~np.isin(q, keys)][:20_000]
    assert t.insert(more, more) == o.insert(more, more)
    check_retrieve(t, o, q)
    assert t.size() == o.size()


def test_overflow_bits_only_for_single_value_tables(wc):
    with pytest.raises(wc.WcError):
        wc.MultiValueTable(8, 4, min_capacity=1000, value_pool_capacity=1000, options=wc.WC_OPT_OVERFLOW_BITS)
    with pytest.raises(wc.WcError):
        wc.SingleValueTable(4, 4, min_capacity=1000, options=4)  # no such option
    t = wc.SingleValueTable(4, 4, min_capacity=1000)
    with pytest.raises(wc.WcError):
        wc.wc_table_dump_overflow_bits(t.handle)


SOA_SHAPES = [(4, 8, 1), (4, 8, 2), (4, 16, 1), (4, 16, 2), (4, 16, 4), (4, 32, 4), (4, 32, 8),
              (8, 4, 1), (8, 4, 2), (8, 8, 1), (8, 8, 2), (8, 16, 2), (8, 16, 4), (8, 32, 4), (8, 32, 8)]


@pytest.mark.parametrize("kb,W,G", SOA_SHAPES)
def test_soa_layout_parity_every_shape(wc, kb, W, G):
    """WC_OPT_SOA (keys and values in two arrays, Sec. IV-A): inserts with overwrites,
    lookups with absent keys and sentinels, erase and re-insert over tombstones, the
    blocked insert and retrieve schemes and overflow bits -- the oracle's results, and the
    key array passes the slot-dump invariant checker."""
    n = 300_007
    if kb == 4:
        d = wc_inputs.sv_insert_retrieve_u32(0x50A + W + G, n, n // 2, 200_000)
        keys, vals, q = d["keys"], d["values"], d["queries"]
    else:
        allk = wc_inputs.distinct_u64(0x50A + W + G, n + 200_000)
        keys, vals = allk[:n], wc_inputs.uniform_u64(9, n)
        q = allk[wc_inputs.shuffle_index(10, allk.size)]
    q = np.concatenate([q, np.array([0, 2 ** (8 * kb) - 1], dtype=q.dtype)])
    opts = wc.WC_OPT_SOA | (wc.WC_OPT_OVERFLOW_BITS if G % 2 == 0 else 0)
    t = make_sv(wc, kb, kb, int(n / 0.9) + 1, W, G, options=opts, seed=0x50A)
    assert t.info["slot_bytes"] == kb
    o = oracle.SingleValue(kb, kb)
    assert t.insert(keys, vals) == o.insert(keys, vals) == 0
    check_retrieve(t, o, q)
    over = (vals[:5000] ^ 0x77).astype(vals.dtype)
    assert t.insert(keys[:5000], over) == o.insert(keys[:5000], over) == oracle.FLAG_DUPLICATE_KEY
    t.erase(keys[5000::3])
    o.erase(keys[5000::3])
    check_retrieve(t, o, q)
    for op in (wc.WC_OP_INSERT, wc.WC_OP_RETRIEVE):
        t.set_launch(op, G, scheme=wc.WC_SCHEME_BLOCKED, region_mib=1)
    back = keys[5000::6]
    bv = (vals[5000::6] ^ 0x99).astype(vals.dtype)
    assert t.insert(back, bv) == o.insert(back, bv) == 0
    check_retrieve(t, o, q)
    assert t.size() == o.size()
    info = t.info
    bits = wc.wc_table_dump_overflow_bits(t.handle) if opts & wc.WC_OPT_OVERFLOW_BITS else None
    r = oracle.check_slots(wc.wc_table_dump_slots(t.handle), info["windows"], info["window_width"], kb, 0x50A, True,
                           bits, key_bytes=kb)
    assert r == {"live": o.size(), "dups": 0, "unreachable": 0}


def test_soa_tables_are_refused_where_the_packed_layout_is_required(wc):
    t = wc.SingleValueTable(4, 4, min_capacity=4096, options=wc.WC_OPT_SOA)
    with pytest.raises(wc.WcError):
        wc.wc_table_device_view(t.handle)
    k = t.keys_dev(np.arange(1, 100, dtype=np.uint32))
    with pytest.raises(wc.WcError):
        wc.wc_insert_noalloc(t.handle, k, k)
    with pytest.raises(wc.WcError):  # struct-of-arrays is a single-value layout
        wc.CountingTable(4, min_capacity=1000, options=wc.WC_OPT_SOA)


def dedup_queries(keys, absent, m, seed):
    """m queries dense in repeats: a hot set of 48 keys (every 32-query block holds many
    equal keys), uniform draws over all keys, absent keys, runs of one key, and sentinels."""
    u = wc_inputs.uniform_u64(seed, m)
    q = keys[(u % np.uint64(48)).astype(np.int64)].copy()
    sel = (u >> np.uint64(8)) % np.uint64(4)
    wide = keys[((u >> np.uint64(16)) % np.uint64(keys.size)).astype(np.int64)]
    q[sel == 1] = wide[sel == 1]
    q[sel == 2] = absent[((u >> np.uint64(24)) % np.uint64(absent.size)).astype(np.int64)][sel == 2]
    q[100:160] = keys[7]  # a run across two blocks
    top = keys.dtype.type(~keys.dtype.type(0))
    q[5::97] = 0
    q[11::101] = top
    return q


@pytest.mark.parametrize("kb,W,G", [(4, 8, 2), (4, 8, 1), (4, 16, 4), (4, 32, 8), (8, 4, 2), (8, 8, 4), (8, 2, 1)])
@pytest.mark.parametrize("opt", [0, 1])
def test_dedup_scheme_parity(wc, kb, W, G, opt):
    """WC_SCHEME_DEDUP (one probe per group of equal queries in a warp's 32-query block,
    the result written to every position of the group): values, found flags and status
    equal the oracle's on query streams full of repeats, absent keys and sentinels, for
    retrieve with and without the found mask and for wc_contains; batch sizes that end
    inside a block."""
    import torch
    n = 200_003
    keys = wc_inputs.distinct_u32(0xDD00 + W, n) if kb == 4 else wc_inputs.distinct_u64(0xDD00 + W, n)
    vals = (wc_inputs.uniform_u32(0xDE01, n) if kb == 4 else wc_inputs.uniform_u64(0xDE01, n)).astype(keys.dtype)
    other = wc_inputs.distinct_u32(0xDE02, 50_000) if kb == 4 else wc_inputs.distinct_u64(0xDE02, 50_000)
    absent = other[~np.isin(other, keys)]
    assert absent.size > 40_000
    t = make_sv(wc, kb, kb, int(n / 0.9) + 1, W, G, options=opt)
    t.set_launch(wc.WC_OP_RETRIEVE, G, scheme=wc.WC_SCHEME_DEDUP)
    assert wc.wc_table_get_launch(t.handle, wc.WC_OP_RETRIEVE)["scheme"] == wc.WC_SCHEME_DEDUP
    o = oracle.SingleValue(kb, kb)
    assert t.insert(keys, vals) == o.insert(keys, vals) == 0
    q = dedup_queries(keys, absent, 300_017, 0xDD3 + W)
    eo, ef, eflags = o.retrieve(q)
    out, found, flags = t.retrieve(q)
    assert flags == eflags == oracle.FLAG_INVALID_KEY
    np.testing.assert_array_equal(found, ef)
    np.testing.assert_array_equal(out, eo)
    qd = t.keys_dev(q)
    vo = torch.empty_like(qd)
    wc.wc_retrieve(t.handle, qd, vo, None)  # values only
    np.testing.assert_array_equal(vo.cpu().numpy().view(eo.dtype), eo)
    fm = torch.empty(q.size, dtype=torch.uint8, device="cuda")
    wc.api.wc_contains(t.handle, qd, fm)  # membership only
    np.testing.assert_array_equal(fm.cpu().numpy(), ef)
    wc.wc_get_status(t.handle, True)
    for m in (1, 31, 33, 65, 0):
        eo, ef, _ = o.retrieve(q[:m])
        out, found, _ = t.retrieve(q[:m])
        np.testing.assert_array_equal(found, ef)
        np.testing.assert_array_equal(out, eo)


def test_dedup_scheme_counting_set_and_refusals(wc):
    """The grouped lookup serves counting tables (counts) and hash sets (membership) too;
    it is refused for inserts and erases and for tables without a single-slot lookup."""
    d = wc_inputs.mv_zipf_u64(0xDD4, 1 << 12, 150_001, 1 << 10)
    keys, q = d["keys"], d["queries"]
    c = wc.CountingTable(8, min_capacity=1 << 13)
    c.set_launch(wc.WC_OP_RETRIEVE, 2, scheme=wc.WC_SCHEME_DEDUP)
    oc = oracle.Counting(8)
    c.insert(keys)
    oc.insert(keys)
    qq = np.concatenate([keys[:100_000], q])
    out, found, _ = c.retrieve(qq)
    eo, ef, _ = oc.retrieve(qq)
    np.testing.assert_array_equal(found, ef)
    np.testing.assert_array_equal(out, eo)
    st = wc.HashSetTable(8, min_capacity=1 << 13)
    st.set_launch(wc.WC_OP_RETRIEVE, 2, scheme=wc.WC_SCHEME_DEDUP)
    os_ = oracle.HashSet(8)
    st.insert(keys)
    os_.insert(keys)
    found, _ = st.contains(qq)
    ef, _ = os_.contains(qq)
    np.testing.assert_array_equal(found, ef)
    for op in (wc.WC_OP_INSERT, wc.WC_OP_ERASE):
        with pytest.raises(wc.WcError):
            c.set_launch(op, 2, scheme=wc.WC_SCHEME_DEDUP)
    mv = wc.MultiValueOATable(4, 4, min_capacity=1 << 12)
    with pytest.raises(wc.WcError):
        mv.set_launch(wc.WC_OP_RETRIEVE, 2, scheme=wc.WC_SCHEME_DEDUP)


def test_l2_persist_carveout_is_given_back(wc):
    """Tables created with l2_persist raise the context's persisting-L2 carve-out; the
    limit found before the first of them comes back when the last one is destroyed."""
    import ctypes
    rt = ctypes.CDLL("libcudart.so.13")  # the runtime instance libwc.so is linked against
    limit_persisting_l2 = 0x06  # cudaLimitPersistingL2CacheSize

    def limit():
        v = ctypes.c_size_t(0)
        assert rt.cudaDeviceGetLimit(ctypes.byref(v), limit_persisting_l2) == 0
        return v.value

    # start from no carve-out (a limit of this process's context only), so that the
    # tables have something to raise
    assert rt.cudaDeviceSetLimit(limit_persisting_l2, ctypes.c_size_t(0)) == 0
    before = limit()
    assert before == 0
    a = wc.SingleValueTable(4, 4, min_capacity=1 << 20, l2_persist=True)
    b = wc.SingleValueTable(4, 4, min_capacity=1 << 19, l2_persist=True)
    raised = limit()
    assert raised > before
    o = oracle.SingleValue(4, 4)
    keys = wc_inputs.distinct_u32(0xC0FE, 1 << 18)
    vals = wc_inputs.uniform_u32(0xC0FF, 1 << 18)
    assert a.insert(keys, vals) == o.insert(keys, vals) == 0
    check_retrieve(a, o, keys)
    a.close()
    assert limit() == raised  # b still holds it
    b.close()
    assert limit() == before


# shapes where lookups keep two keys per group in flight (up to 32 bytes of window per lane)
KIF2_P32 = [(W, G) for W, G in W_G_P32 if W // G <= 4]
KIF2_P64 = [(W, G) for W, G in W_G_P64 if W // G <= 2]


@pytest.mark.parametrize("opt", [0, 1], ids=["plain", "overflow_bits"])
@pytest.mark.parametrize("kb,W,G", [(4,) + x for x in KIF2_P32] + [(8,) + x for x in KIF2_P64])
def test_retrieve_two_keys_per_group_in_flight(wc, kb, W, G, opt):
    """Lookups with keys_in_flight = 2 against the oracle, element by element: present and
    absent keys, sentinels, after erases (tombstones walked past) and re-inserts; a batch
    with a ragged tail that does not fill the warps' ranges evenly."""
    n = 70_001
    if kb == 4:
        keys = wc_inputs.distinct_u32(0x2F17 + W * 64 + G, n + 35_000)
        vals = wc_inputs.uniform_u32(6, n)
    else:
        keys = wc_inputs.distinct_u64(0x2F17 + W * 64 + G, n + 35_000)
        vals = wc_inputs.uniform_u64(6, n)
    t = make_sv(wc, kb, kb, int(n / 0.92) + 1, W, G, options=opt)
    t.set_launch(wc.WC_OP_RETRIEVE, G, keys_in_flight=2)
    assert wc.wc_table_get_launch(t.handle, wc.WC_OP_RETRIEVE)["keys_in_flight"] == 2
    o = oracle.SingleValue(kb, kb)
    assert t.insert(keys[:n], vals) == o.insert(keys[:n], vals) == 0
    q = keys[wc_inputs.shuffle_index(11, keys.size)]
    q = np.concatenate([q, np.array([0, 0, (1 << (8 * kb)) - 1], dtype=q.dtype), q[:17]])
    check_retrieve(t, o, q)
    drop = keys[: n // 3]
    assert t.erase(drop) == o.erase(drop)
    check_retrieve(t, o, q)
    assert t.insert(drop[::2], vals[: n // 3: 2]) == o.insert(drop[::2], vals[: n // 3: 2])
    check_retrieve(t, o, q)
    assert t.size() == o.size()
