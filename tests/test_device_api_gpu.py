"""Device-side API (include/wc_device_api.cuh) from a user's program: per-element inserts,
lookups and erases in user kernels, for_each / for_all with device lambdas, and a fused
producer kernel.  Each direction is crossed with the bulk calls -- keys inserted by user
kernels are found by wc_retrieve, keys inserted by wc_insert are found by user kernels --
and every result is compared with the CPU oracle; the tables' slot dumps pass the
invariant checker."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import wc_inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SEED = 0xD1CE


@pytest.fixture(scope="module")
def env(tmp_path_factory):
    from paper_2009_07914_gb300 import build
    build.build()
    import torch

    import paper_2009_07914_gb300 as wc
    out = str(tmp_path_factory.mktemp("devapi") / "libwcuser.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           "--extended-lambda", "-shared", "-Xcompiler", "-fPIC", "-cudart", "shared",
                           "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "device_api", "user_kernels.cu"), "-o", out])
    lib = ctypes.CDLL(out)
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    V = ctypes.POINTER(wc._binding.WcDeviceView)
    lib.wcu_insert.argtypes = [V, vp, vp, u64, vp]
    lib.wcu_insert_uncounted.argtypes = [V, vp, vp, u64, vp]
    lib.wcu_retrieve.argtypes = [V, vp, u64, vp, vp]
    lib.wcu_erase.argtypes = [V, vp, u64, vp]
    lib.wcu_fused_insert.argtypes = [V, u64, u32, vp]
    lib.wcu_for_each.argtypes = [V, vp, u64, vp, vp]
    lib.wcu_for_all.argtypes = [V, vp]
    lib.wcu_mv_append.argtypes = [V, vp, vp, u64, vp]
    lib.wcu_mv_append_uncounted.argtypes = [V, vp, vp, u64, vp]
    lib.wcu_set_op.argtypes = [V, ctypes.c_int, vp, u64, vp, vp]
    lib.wcu_group_op.argtypes = [V, ctypes.c_int, ctypes.c_int, vp, vp, u64, vp, vp, vp]
    lib.wcu_count_add.argtypes = [V, vp, vp, u64, vp]
    lib.wcu_count_get.argtypes = [V, vp, u64, vp, vp]
    lib.wcu_poke_u64.argtypes = [vp, u64]
    return wc, torch, lib


def dev(torch, a, width):
    from paper_2009_07914_gb300.table import to_device
    return to_device(a, width, torch.device("cuda", 0))


def host(t, width):
    from paper_2009_07914_gb300.table import to_numpy
    return to_numpy(t, width)


def check_dump(wc, t, opt):
    info = t.info
    bits = wc.api.wc_table_dump_overflow_bits(t.handle) if opt else None
    r = oracle.check_slots(wc.api.wc_table_dump_slots(t.handle), info["windows"], info["window_width"],
                           info["slot_bytes"], SEED, True, bits)
    assert r["dups"] == 0 and r["unreachable"] == 0
    return r


@pytest.mark.parametrize("opt", [0, 1])
@pytest.mark.parametrize("kb,W", [(4, 8), (4, 32), (8, 4), (8, 2)])
def test_device_ops_interoperate_with_bulk_calls(env, kb, W, opt):
    wc, torch, lib = env
    n = 200_003
    keys = wc_inputs.distinct_u32(71 + W, n) if kb == 4 else wc_inputs.distinct_u64(71 + W, n)
    vals = (wc_inputs.uniform_u32(72, n) if kb == 4 else wc_inputs.uniform_u64(72, n)).astype(keys.dtype)
    batch_k = np.concatenate([keys, keys[:5000], np.array([0, keys.dtype.type(~keys.dtype.type(0))], keys.dtype)])
    batch_v = np.concatenate([vals, vals[:5000] ^ keys.dtype.type(0x5A), np.zeros(2, keys.dtype)])
    absent = (wc_inputs.distinct_u32(7300 + W, n) | np.uint32(1 << 31)) if kb == 4 else wc_inputs.distinct_u64(7300 + W, n)
    absent = absent[~np.isin(absent, keys)]
    queries = np.concatenate([keys, absent[:100_000]])
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")

    # user-kernel inserts -> bulk retrieve
    a = wc.SingleValueTable(kb, kb, min_capacity=int(n / 0.9), window_width=W, seed=SEED, options=opt)
    va = wc.api.wc_table_device_view(a.handle)
    assert lib.wcu_insert(ctypes.byref(va), dev(torch, batch_k, kb).data_ptr(), dev(torch, batch_v, kb).data_ptr(),
                          batch_k.size, flags.data_ptr()) == 0
    o = oracle.SingleValue(kb, kb)
    of = o.insert(batch_k, batch_v)
    assert int(flags.item()) == of == oracle.FLAG_DUPLICATE_KEY | oracle.FLAG_INVALID_KEY
    assert a.status(clear=True) == of
    assert a.size() == o.size() == n
    out, found, _ = a.retrieve(queries)
    eo, ef, _ = o.retrieve(queries)
    np.testing.assert_array_equal(found, ef)
    # a key inserted twice in one batch keeps one of its two values
    dup = np.isin(queries, keys[:5000])
    np.testing.assert_array_equal(out[~dup], eo[~dup])
    ok = (out[dup] == eo[dup]) | (out[dup] == (eo[dup] ^ keys.dtype.type(0x5A)))
    assert ok.all()
    check_dump(wc, a, opt)

    # bulk insert -> user-kernel retrieve, erase, for_each, for_all
    b = wc.SingleValueTable(kb, kb, min_capacity=int(n / 0.9), window_width=W, seed=SEED, options=opt)
    b.insert(keys, vals)
    o2 = oracle.SingleValue(kb, kb)
    o2.insert(keys, vals)
    vb = wc.api.wc_table_device_view(b.handle)
    qd = dev(torch, queries, kb)
    outd = torch.empty_like(qd)
    foundd = torch.empty(queries.size, dtype=torch.uint8, device="cuda")
    assert lib.wcu_retrieve(ctypes.byref(vb), qd.data_ptr(), queries.size, outd.data_ptr(), foundd.data_ptr()) == 0
    eo, ef, _ = o2.retrieve(queries)
    np.testing.assert_array_equal(foundd.cpu().numpy(), ef)
    np.testing.assert_array_equal(host(outd, kb)[ef == 1], eo[ef == 1])
    drop = np.concatenate([keys[::4], absent[:1000]])
    erased = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert lib.wcu_erase(ctypes.byref(vb), dev(torch, drop, kb).data_ptr(), drop.size, erased.data_ptr()) == 0
    o2.erase(drop)
    assert int(erased.item()) == keys[::4].size and b.size() == o2.size()
    out, found, _ = b.retrieve(queries)
    eo, ef, _ = o2.retrieve(queries)
    np.testing.assert_array_equal(found, ef)
    np.testing.assert_array_equal(out, eo)
    check_dump(wc, b, opt)
    sums = torch.zeros(2, dtype=torch.int64, device="cuda")
    fmask = torch.zeros(queries.size, dtype=torch.uint8, device="cuda")
    assert lib.wcu_for_each(ctypes.byref(vb), qd.data_ptr(), queries.size, sums.data_ptr(), fmask.data_ptr()) == 0
    np.testing.assert_array_equal(fmask.cpu().numpy(), ef)
    s = sums.cpu().numpy().view(np.uint64)
    assert int(s[1]) == int(ef.sum())
    assert int(s[0]) == int(eo[ef == 1].astype(np.uint64).sum(dtype=np.uint64))
    alls = torch.zeros(3, dtype=torch.int64, device="cuda")
    assert lib.wcu_for_all(ctypes.byref(vb), alls.data_ptr()) == 0
    live = keys[~np.isin(keys, drop)]
    lv = vals[~np.isin(keys, drop)]
    a3 = alls.cpu().numpy().view(np.uint64)
    assert int(a3[0]) == live.size
    assert int(a3[1]) == int(live.astype(np.uint64).sum(dtype=np.uint64))
    assert int(a3[2]) == int(lv.astype(np.uint64).sum(dtype=np.uint64))


def test_fused_producer_kernel_and_full_table(env):
    """A user kernel that produces its keys and inserts them directly (no batch in device
    memory); the bulk retrieve finds every produced key with its index as value.  A table
    too small for the stream reports PROBE_LIMIT without hanging."""
    wc, torch, lib = env
    n, seed = 1 << 20, 0x1234567
    t = wc.SingleValueTable(4, 4, min_capacity=int(n / 0.85), seed=SEED, options=wc.WC_OPT_OVERFLOW_BITS)
    v = wc.api.wc_table_device_view(t.handle)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.wcu_fused_insert(ctypes.byref(v), n, seed, flags.data_ptr()) == 0
    idx = np.arange(n, dtype=np.uint64)
    k = ((idx * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)).astype(np.uint32) ^ np.uint32(seed)
    valid = (k != 0) & (k != 0xFFFFFFFF)
    assert t.size() == int(valid.sum())
    out, found, _ = t.retrieve(k[valid])
    assert found.all()
    np.testing.assert_array_equal(out, idx[valid].astype(np.uint32))
    check_dump(wc, t, 1)
    small = wc.SingleValueTable(4, 4, min_capacity=1000, seed=SEED)
    vs = wc.api.wc_table_device_view(small.handle)
    flags.zero_()
    assert lib.wcu_fused_insert(ctypes.byref(vs), 5000, seed, flags.data_ptr()) == 0
    assert int(flags.item()) & wc.WC_FLAG_PROBE_LIMIT
    assert small.size() == small.capacity
    mv = wc.MultiValueTable(8, 4, min_capacity=64, value_pool_capacity=64)
    with pytest.raises(wc.WcError):  # bucket multi-value tables have no device view
        wc.api.wc_table_device_view(mv.handle)


def test_library_device_api_probe(env):
    """wc_bench_device_api (the library's own fused producer over the device API) stores
    exactly the produced pairs, and its lookup pass adds up their values."""
    wc, torch, lib = env
    from paper_2009_07914_gb300.roofline import wc_bench_device_api
    n, seed = 300_001, 0xBEEF
    t = wc.SingleValueTable(4, 4, min_capacity=int(n / 0.9), seed=SEED, options=wc.WC_OPT_OVERFLOW_BITS)
    wc_bench_device_api(t.handle, 0, n, seed)
    idx = np.arange(n, dtype=np.uint64)
    k = ((idx * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)).astype(np.uint32) ^ np.uint32(seed)
    valid = (k != 0) & (k != 0xFFFFFFFF)
    assert t.size() == int(valid.sum())
    out, found, _ = t.retrieve(k)
    np.testing.assert_array_equal(found, valid.astype(np.uint8))
    np.testing.assert_array_equal(out[valid], idx[valid].astype(np.uint32))
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    wc_bench_device_api(t.handle, 1, n, seed, sink)
    assert int(sink.item()) == int(idx[valid].sum())
    check_dump(wc, t, 1)



# ---- per-element appends to a bucket multi-value table (Sec. IV-C) -----------------------

def _mv_view(wc, t, wait_ns=0):
    v = wc._binding.WcDeviceView()
    wc._binding.check(wc._binding.lib().wc_table_device_view(t.handle, ctypes.byref(v)), "wc_table_device_view")
    v.wait_ns = wait_ns
    return v


def _mv_check(t, o, queries):
    offs, _ = t.count_values(queries)
    eoffs, _ = o.count_values(queries)
    np.testing.assert_array_equal(offs, eoffs)
    vals, _ = t.retrieve_multi(queries, offs)
    evals, _ = o.retrieve_multi(queries, eoffs)
    np.testing.assert_array_equal(oracle.sorted_segments(vals, offs), oracle.sorted_segments(evals, eoffs))


@pytest.mark.parametrize("kb,vb", [(4, 4), (8, 4), (8, 8)])
@pytest.mark.parametrize("s0,lam", [(1, 1.1), (4, 1.0), (1, 2.0)])
@pytest.mark.parametrize("counted", [True, False], ids=["append", "append_uncounted"])
def test_device_appends_build_the_bucket_lists(env, kb, vb, s0, lam, counted):
    """Concurrent per-element appends of hot keys (2^18 values over 1000 keys, every key's
    copies spread over the launch) against the multiset oracle, then a bulk insert into
    the same lists and appends again: counts, offsets and sorted values per key equal the
    oracle's; the size counts every value, the key count every distinct key (with
    append_uncounted, once each thread has added its counts)."""
    wc, torch, lib = env
    n, nk = 1 << 18, 1000
    kdt = np.uint32 if kb == 4 else np.uint64
    vdt = np.uint32 if vb == 4 else np.uint64
    uni = (wc_inputs.distinct_u32(0xB1 + kb, nk) if kb == 4 else wc_inputs.distinct_u64(0xB1 + kb, nk)).astype(kdt)
    absent = uni[: nk // 4] ^ kdt(0x5A5A5A5A)
    absent = absent[~np.isin(absent, uni) & (absent != 0)]
    rng = np.random.default_rng(kb * 8 + vb)
    t = wc.MultiValueTable(kb, vb, min_capacity=2 * nk, value_pool_capacity=8 * n, bucket_first_size=s0,
                           bucket_growth=lam)
    o = oracle.MultiValue(kb, vb)
    v = _mv_view(wc, t)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    for rnd in range(2):
        keys = uni[rng.integers(0, nk, n)]
        vals = rng.integers(0, 1 << (8 * vb - 1), n, dtype=np.uint64).astype(vdt)
        dk, dv = dev(torch, keys, kb), dev(torch, vals, vb)
        fn = lib.wcu_mv_append if counted else lib.wcu_mv_append_uncounted
        assert fn(ctypes.byref(v), dk.data_ptr(), dv.data_ptr(), n, flags.data_ptr()) == 0
        o.insert(keys, vals)
        assert int(flags.item()) == 0 and t.status(clear=True) == 0
        assert t.size() == o.size() and t.num_keys() == nk
        _mv_check(t, o, np.concatenate([uni, absent]))
        if rnd == 0:  # a bulk insert fills the lists' last buckets and adds more
            bk = uni[rng.integers(0, nk, 5000)]
            bv = rng.integers(0, 1 << (8 * vb - 1), 5000, dtype=np.uint64).astype(vdt)
            t.insert(bk, bv)
            o.insert(bk, bv)
            _mv_check(t, o, uni)


def test_device_appends_stop_at_a_full_pool(env):
    """A pool too small for the appends: POOL_EXHAUSTED is raised and what was stored is
    consistent -- every key's values are a sub-multiset of its appended ones, and the
    counts add up to the size."""
    wc, torch, lib = env
    n, nk = 50_000, 300
    uni = wc_inputs.distinct_u32(0xC4, nk)
    rng = np.random.default_rng(9)
    keys = uni[rng.integers(0, nk, n)]
    vals = np.arange(n, dtype=np.uint32)
    t = wc.MultiValueTable(4, 4, min_capacity=2 * nk, value_pool_capacity=n // 2, bucket_first_size=2,
                           bucket_growth=1.5)
    v = _mv_view(wc, t)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    dk, dv = dev(torch, keys, 4), dev(torch, vals, 4)
    assert lib.wcu_mv_append(ctypes.byref(v), dk.data_ptr(), dv.data_ptr(), n, flags.data_ptr()) == 0
    assert int(flags.item()) & wc.WC_FLAG_POOL_EXHAUSTED
    assert t.status(clear=True) & wc.WC_FLAG_POOL_EXHAUSTED
    offs, _ = t.count_values(uni)
    got, _ = t.retrieve_multi(uni, offs)
    assert int(offs[-1]) == t.size() < n
    for i in range(nk):
        seg = got[offs[i]:offs[i + 1]]
        mine = vals[keys == uni[i]]
        assert np.isin(seg, mine).all() and np.unique(seg).size == seg.size


def test_device_append_wait_is_bounded(env):
    """A list handle left blocked (its blocked bit set from the host, as if the thread
    making its next bucket had stopped): an append to that key waits at most wait_ns, then
    returns QUEUE_TIMEOUT and sets it in the status word -- the kernel ends; appends of other
    keys are unaffected.  Clearing the bit lets appends of the key go on."""
    wc, torch, lib = env
    t = wc.MultiValueTable(8, 4, min_capacity=64, value_pool_capacity=1024, bucket_first_size=1, bucket_growth=1.0)
    v = _mv_view(wc, t, wait_ns=2_000_000)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    k = np.array([0x1234567, 0x7654321], dtype=np.uint64)
    one = np.array([7, 8], dtype=np.uint32)
    assert lib.wcu_mv_append(ctypes.byref(v), dev(torch, k, 8).data_ptr(), dev(torch, one, 4).data_ptr(), 2,
                             flags.data_ptr()) == 0
    assert int(flags.item()) == 0
    dump = wc.api.wc_table_dump_slots(t.handle).view(np.uint64).reshape(-1, 2)
    idx = int(np.nonzero(dump[:, 0] == k[0])[0][0])
    handle = int(dump[idx, 1])
    addr = v.slots + idx * 16 + 8
    assert lib.wcu_poke_u64(addr, handle | (1 << 63)) == 0
    k2 = np.array([k[0], k[1]], dtype=np.uint64)
    assert lib.wcu_mv_append(ctypes.byref(v), dev(torch, k2, 8).data_ptr(), dev(torch, one, 4).data_ptr(), 2,
                             flags.data_ptr()) == 0
    assert int(flags.item()) == wc.WC_FLAG_QUEUE_TIMEOUT
    assert t.status(clear=True) == wc.WC_FLAG_QUEUE_TIMEOUT
    assert lib.wcu_poke_u64(addr, handle) == 0
    flags.zero_()
    assert lib.wcu_mv_append(ctypes.byref(v), dev(torch, k[:1], 8).data_ptr(), dev(torch, one[1:], 4).data_ptr(), 1,
                             flags.data_ptr()) == 0
    assert int(flags.item()) == 0
    offs, _ = t.count_values(k)
    got, _ = t.retrieve_multi(k, offs)
    assert list(np.diff(offs)) == [2, 2]
    assert sorted(got[:2].tolist()) == [7, 8] and sorted(got[2:].tolist()) == [8, 8]



# ---- hash sets and counting tables from user kernels (Sec. IV: HashSet, CountingHashTable) --

def _view(wc, t):
    v = wc._binding.WcDeviceView()
    wc._binding.check(wc._binding.lib().wc_table_device_view(t.handle, ctypes.byref(v)), "wc_table_device_view")
    return v


@pytest.mark.parametrize("opt", [0, 1], ids=["plain", "overflow_bits"])
@pytest.mark.parametrize("kb,W", [(4, 8), (4, 32), (8, 4), (8, 16)])
def test_device_set_ops_match_the_oracle(env, kb, W, opt):
    """Set inserts from a user kernel (duplicates inside the batch and of stored keys),
    membership and erase by user kernels and by the bulk calls, crossed: every answer
    equals the oracle's set; the slot dump has no duplicate and no unreachable key."""
    wc, torch, lib = env
    n = 60_000
    allk = wc_inputs.distinct_u32(0x5E7 + W, 2 * n) if kb == 4 else wc_inputs.distinct_u64(0x5E7 + W, 2 * n)
    keys = np.concatenate([allk[:n], allk[: n // 10]])  # the tail repeats stored keys
    rng = np.random.default_rng(W)
    rng.shuffle(keys)
    t = wc.HashSetTable(kb, min_capacity=int(n / 0.85), window_width=W, seed=SEED, options=opt)
    v = _view(wc, t)
    o = oracle.HashSet(kb)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(keys.size, dtype=torch.uint8, device="cuda")
    assert lib.wcu_set_op(ctypes.byref(v), 0, dev(torch, keys, kb).data_ptr(), keys.size, out.data_ptr(),
                          flags.data_ptr()) == 0
    assert int(flags.item()) == o.insert(keys) == wc.WC_FLAG_DUPLICATE_KEY
    assert int(out.sum().item()) == n and t.size() == o.size() == n
    q = allk[wc_inputs.shuffle_index(3, allk.size)]
    qo = torch.empty(q.size, dtype=torch.uint8, device="cuda")
    assert lib.wcu_set_op(ctypes.byref(v), 1, dev(torch, q, kb).data_ptr(), q.size, qo.data_ptr(),
                          flags.data_ptr()) == 0
    ef, _ = o.contains(q)
    np.testing.assert_array_equal(qo.cpu().numpy(), ef)
    np.testing.assert_array_equal(t.contains(q)[0], ef)  # the bulk call sees the user kernel's keys
    drop = allk[: n // 3]
    eo = torch.empty(drop.size, dtype=torch.uint8, device="cuda")
    assert lib.wcu_set_op(ctypes.byref(v), 2, dev(torch, drop, kb).data_ptr(), drop.size, eo.data_ptr(),
                          flags.data_ptr()) == 0
    assert int(eo.sum().item()) == drop.size
    o.erase(drop)
    t.insert(allk[n: n + 1000])  # bulk inserts, seen by the user kernel's lookups
    o.insert(allk[n: n + 1000])
    assert lib.wcu_set_op(ctypes.byref(v), 1, dev(torch, q, kb).data_ptr(), q.size, qo.data_ptr(),
                          flags.data_ptr()) == 0
    ef, _ = o.contains(q)
    np.testing.assert_array_equal(qo.cpu().numpy(), ef)
    assert t.size() == o.size()
    info = t.info
    r = oracle.check_slots(wc.api.wc_table_dump_slots(t.handle), info["windows"], info["window_width"],
                           info["slot_bytes"], SEED, True,
                           wc.api.wc_table_dump_overflow_bits(t.handle) if opt else None, key_bytes=kb)
    assert r["dups"] == 0 and r["unreachable"] == 0 and r["live"] == o.size()


@pytest.mark.parametrize("kb,W", [(4, 8), (4, 16), (8, 4), (8, 8)])
def test_device_count_add_matches_the_oracle(env, kb, W):
    """Counting-table adds from a user kernel: 2^18 skewed occurrences with weights (and a
    second launch without), crossed with bulk inserts and lookups; every count equals the
    oracle's sum of weights per key (wrapping at the key width)."""
    wc, torch, lib = env
    n, nk = 1 << 18, 3000
    kdt = np.uint32 if kb == 4 else np.uint64
    uni = (wc_inputs.distinct_u32(0xC0 + W, 2 * nk) if kb == 4 else wc_inputs.distinct_u64(0xC0 + W, 2 * nk))
    rng = np.random.default_rng(kb * 16 + W)
    ranks = np.minimum(rng.zipf(1.3, n) - 1, nk - 1)
    keys = uni[ranks].astype(kdt)
    wts = rng.integers(0, 1000, n, dtype=np.uint64).astype(kdt)
    t = wc.CountingTable(kb, min_capacity=int(nk / 0.8), window_width=W, seed=SEED)
    v = _view(wc, t)
    o = oracle.Counting(kb)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.wcu_count_add(ctypes.byref(v), dev(torch, keys, kb).data_ptr(), dev(torch, wts, kb).data_ptr(), n,
                             flags.data_ptr()) == 0
    o.insert(keys, wts)
    assert lib.wcu_count_add(ctypes.byref(v), dev(torch, keys[: n // 2], kb).data_ptr(), None, n // 2,
                             flags.data_ptr()) == 0
    o.insert(keys[: n // 2])
    t.insert(keys[: 5000])  # bulk occurrences of the same keys
    o.insert(keys[: 5000])
    assert int(flags.item()) == 0 and t.size() == o.size()
    q = uni  # half of them never occur
    out = torch.empty(q.size, dtype=torch.int32 if kb == 4 else torch.int64, device="cuda")
    found = torch.empty(q.size, dtype=torch.uint8, device="cuda")
    assert lib.wcu_count_get(ctypes.byref(v), dev(torch, q, kb).data_ptr(), q.size, out.data_ptr(),
                             found.data_ptr()) == 0
    eo, ef, _ = o.retrieve(q)
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(host(out, kb)[ef == 1], eo[ef == 1])
    bo, bf, _ = t.retrieve(q)  # the bulk lookup reads the same counts
    np.testing.assert_array_equal(bf, ef)
    np.testing.assert_array_equal(bo[ef == 1], eo[ef == 1])



# ---- group-cooperative device operations (a tile of G threads per key, Sec. IV-B2) ------

@pytest.mark.parametrize("opt", [0, 1], ids=["plain", "overflow_bits"])
@pytest.mark.parametrize("kb,W,G", [(4, 8, 1), (4, 8, 2), (4, 8, 4), (4, 16, 4), (4, 32, 8), (8, 4, 2), (8, 8, 4),
                                    (8, 2, 2)])
def test_group_device_ops_match_the_oracle(env, kb, W, G, opt):
    """Tiles of G threads insert (with repeats of stored keys, after erases that leave
    tombstones) and look up keys together; crossed with the bulk calls; every value and
    found bit equals the oracle's and the slot dump passes the invariant checker."""
    wc, torch, lib = env
    n = 50_000
    allk = wc_inputs.distinct_u32(0x6A + W * 8 + G, 2 * n) if kb == 4 else wc_inputs.distinct_u64(0x6A + W * 8 + G,
                                                                                                 2 * n)
    vals = (wc_inputs.uniform_u32(G, 2 * n) if kb == 4 else wc_inputs.uniform_u64(G, 2 * n))
    t = wc.SingleValueTable(kb, kb, min_capacity=int(n / 0.9) + 1, window_width=W, seed=SEED, options=opt)
    o = oracle.SingleValue(kb, kb)
    v = _view(wc, t)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    wdt = torch.int32 if kb == 4 else torch.int64

    def ins(k, x):
        assert lib.wcu_group_op(ctypes.byref(v), 0, G, dev(torch, k, kb).data_ptr(), dev(torch, x, kb).data_ptr(),
                                k.size, None, None, flags.data_ptr()) == 0

    def look(k):
        out = torch.empty(k.size, dtype=wdt, device="cuda")
        fnd = torch.empty(k.size, dtype=torch.uint8, device="cuda")
        assert lib.wcu_group_op(ctypes.byref(v), 1, G, dev(torch, k, kb).data_ptr(), None, k.size, out.data_ptr(),
                                fnd.data_ptr(), flags.data_ptr()) == 0
        return host(out, kb), fnd.cpu().numpy()

    ins(allk[:n], vals[:n])
    o.insert(allk[:n], vals[:n])
    assert int(flags.item()) == 0 and t.size() == o.size() == n
    q = allk[wc_inputs.shuffle_index(5, allk.size)]
    go, gf = look(q)
    eo, ef, _ = o.retrieve(q)
    np.testing.assert_array_equal(gf, ef)
    np.testing.assert_array_equal(go[ef == 1], eo[ef == 1])
    bo, bf, _ = t.retrieve(q)  # the bulk lookup finds the group inserts
    np.testing.assert_array_equal(bf, ef)
    np.testing.assert_array_equal(bo, eo)
    drop = allk[: n // 3]
    t.erase(drop)
    o.erase(drop)
    again = np.concatenate([drop[::2], allk[n // 2: n // 2 + 300]])  # tombstones reused, duplicates
    ins(again, vals[n: n + again.size])
    o.insert(again, vals[n: n + again.size])
    assert int(flags.item()) == wc.WC_FLAG_DUPLICATE_KEY and t.size() == o.size()
    go, gf = look(q)
    eo, ef, _ = o.retrieve(q)
    np.testing.assert_array_equal(gf, ef)
    np.testing.assert_array_equal(go[ef == 1], eo[ef == 1])
    info = t.info
    r = oracle.check_slots(wc.api.wc_table_dump_slots(t.handle), info["windows"], info["window_width"],
                           info["slot_bytes"], SEED, True, wc.api.wc_table_dump_overflow_bits(t.handle) if opt else None)
    assert r["dups"] == 0 and r["unreachable"] == 0 and r["live"] == o.size()


@pytest.mark.parametrize("kb", [4, 8])
def test_uncounted_inserts_add_their_size_once(env, kb):
    """insert_uncounted in a grid-stride kernel that adds its count of new keys to the size
    once per thread: the same table, flags and size as the oracle's, duplicates and
    sentinels included."""
    wc, torch, lib = env
    n = 40000
    keys = wc_inputs.distinct_u32(31 + kb, n) if kb == 4 else wc_inputs.distinct_u64(31 + kb, n)
    vals = (np.arange(n, dtype=np.uint64) * 7 + 3).astype(keys.dtype)
    batch_k = np.concatenate([keys, keys[:3000], np.array([0], dtype=keys.dtype)])
    batch_v = np.concatenate([vals, vals[:3000], np.array([1], dtype=keys.dtype)])
    t = wc.SingleValueTable(kb, kb, min_capacity=int(n / 0.9), window_width=8 if kb == 4 else 4, seed=SEED,
                            options=wc.WC_OPT_OVERFLOW_BITS)
    v = wc.api.wc_table_device_view(t.handle)
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.wcu_insert_uncounted(ctypes.byref(v), dev(torch, batch_k, kb).data_ptr(),
                                    dev(torch, batch_v, kb).data_ptr(), batch_k.size, flags.data_ptr()) == 0
    o = oracle.SingleValue(kb, kb)
    of = o.insert(batch_k, batch_v)
    assert int(flags.item()) == of
    assert t.size() == o.size() == n
    out, found, _ = t.retrieve(keys[3000:])
    eo, ef, _ = o.retrieve(keys[3000:])
    np.testing.assert_array_equal(found, ef)
    np.testing.assert_array_equal(out, eo)
    t.close()
