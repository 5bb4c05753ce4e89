"""Host-buffer calls (wc_insert_host, wc_retrieve_host): batches larger than one staging
chunk, ragged tails, pinned and pageable buffers, counting tables and sets, against the
CPU oracle or, for batches too large for it, against the inserted pairs themselves."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import wc_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2009_07914_gb300 import build
    build.build()
    import torch

    import paper_2009_07914_gb300 as wc
    return wc, torch


def pinned(torch, a):
    return torch.from_numpy(a.view(np.int32 if a.itemsize == 4 else np.int64)).pin_memory()


@pytest.mark.parametrize("pin", [True, False])
@pytest.mark.parametrize("kb", [4, 8])
def test_host_calls_match_oracle(env, kb, pin):
    wc, torch = env
    n = 300_007
    keys = wc_inputs.distinct_u32(0x4057 + kb, n) if kb == 4 else wc_inputs.distinct_u64(0x4057 + kb, n)
    vals = (wc_inputs.uniform_u32(0x4058, n) if kb == 4 else wc_inputs.uniform_u64(0x4058, n)).astype(keys.dtype)
    other = wc_inputs.distinct_u32(0x4059, n) if kb == 4 else wc_inputs.distinct_u64(0x4059, n)
    q = np.concatenate([keys[::3], other[~np.isin(other, keys)][:200_000], np.zeros(3, keys.dtype)])
    t = wc.SingleValueTable(kb, kb, min_capacity=int(n / 0.9), options=wc.WC_OPT_OVERFLOW_BITS)
    o = oracle.SingleValue(kb, kb)
    hk, hv, hq = (pinned(torch, a) if pin else a for a in (keys, vals, q))
    wc.api.wc_insert_host(t.handle, hk, hv)
    torch.cuda.synchronize()
    assert o.insert(keys, vals) == 0 and t.size() == o.size()
    ho = np.empty_like(q)
    hf = np.empty(q.size, np.uint8)
    if pin:
        ho_t, hf_t = pinned(torch, ho), torch.empty(q.size, dtype=torch.uint8).pin_memory()
        wc.api.wc_retrieve_host(t.handle, hq, ho_t, hf_t)
        torch.cuda.synchronize()
        ho, hf = ho_t.numpy().view(keys.dtype), hf_t.numpy()
    else:
        wc.api.wc_retrieve_host(t.handle, hq, ho, hf)
        torch.cuda.synchronize()
    eo, ef, _ = o.retrieve(q)
    np.testing.assert_array_equal(hf, ef)
    np.testing.assert_array_equal(ho[ef == 1], eo[ef == 1])
    assert t.status(clear=True) == oracle.FLAG_INVALID_KEY  # the zero queries


def test_multi_chunk_batches(env):
    """2^25 + 4097 distinct pairs (two insert chunks: 2^23, then the ragged rest) and
    2^25 + 12345 queries (five retrieve chunks, around the ring of three staging buffers):
    every present key returns its own value."""
    wc, torch = env
    n = (1 << 25) + 4097
    keys = wc_inputs.distinct_u32(0x4060, n)
    vals = wc_inputs.uniform_u32(0x4061, n)
    t = wc.SingleValueTable(4, 4, min_capacity=int(n / 0.85), options=wc.WC_OPT_OVERFLOW_BITS)
    hk, hv = pinned(torch, keys), pinned(torch, vals)
    wc.api.wc_insert_host(t.handle, hk, hv)
    torch.cuda.synchronize()
    assert t.size() == n and t.status(clear=True) == 0
    m = (1 << 25) + 12345
    sel = wc_inputs.uniform_u64(0x4062, m) % np.uint64(n)
    q = keys[sel]
    q[::5] = 0xFFFFFFFF  # invalid key: not found
    hq = pinned(torch, q)
    ho = torch.empty(m, dtype=torch.int32).pin_memory()
    hf = torch.empty(m, dtype=torch.uint8).pin_memory()
    ho.fill_(-1)
    wc.api.wc_retrieve_host(t.handle, hq, ho, hf)
    torch.cuda.synchronize()
    f = hf.numpy()
    expect = np.ones(m, np.uint8)
    expect[::5] = 0
    np.testing.assert_array_equal(f, expect)
    np.testing.assert_array_equal(ho.numpy().view(np.uint32)[f == 1], vals[sel][f == 1])
    # the same table, queried through the device call, agrees
    out, found, _ = t.retrieve(q[:100_000])
    np.testing.assert_array_equal(found, f[:100_000])
    np.testing.assert_array_equal(out[found == 1], ho.numpy().view(np.uint32)[:100_000][found == 1])


def test_counting_and_set_host_inserts(env):
    wc, torch = env
    d = wc_inputs.mv_zipf_u64(0x4063, 1 << 14, 400_001, 1 << 10)
    keys = d["keys"]
    c = wc.CountingTable(8, min_capacity=1 << 15)
    oc = oracle.Counting(8)
    wc.api.wc_insert_host(c.handle, pinned(torch, keys), None)
    wc.api.wc_insert_host(c.handle, keys[:1000], None)  # pageable, unit weights
    torch.cuda.synchronize()
    oc.insert(keys)
    oc.insert(keys[:1000])
    q = np.unique(keys)[:5000]
    ho, hf = np.empty(q.size, np.uint64), np.empty(q.size, np.uint8)
    wc.api.wc_retrieve_host(c.handle, q, ho, hf)
    torch.cuda.synchronize()
    eo, ef, _ = oc.retrieve(q)
    np.testing.assert_array_equal(hf, ef)
    np.testing.assert_array_equal(ho, eo)
    s = wc.HashSetTable(8, min_capacity=1 << 15)
    wc.api.wc_insert_host(s.handle, keys, None)
    torch.cuda.synchronize()
    assert s.size() == np.unique(keys).size
    with pytest.raises(wc.WcError):  # sets have no values to retrieve
        wc.api.wc_retrieve_host(s.handle, q, ho, hf)


def test_host_calls_refuse_device_pointers(env):
    wc, torch = env
    t = wc.SingleValueTable(4, 4, min_capacity=1000)
    dk = torch.ones(10, dtype=torch.int32, device="cuda")
    with pytest.raises(wc.WcError):
        wc.api.wc_insert_host(t.handle, dk.data_ptr(), dk.data_ptr(), 10)
    with pytest.raises(ValueError):
        wc.api.wc_insert_host(t.handle, dk, dk)
    wc.api.wc_insert_host(t.handle, np.arange(1, 11, dtype=np.uint32), np.arange(10, dtype=np.uint32), 0)
    assert t.size() == 0


@pytest.mark.parametrize("kb", [4, 8])
def test_host_calls_struct_of_arrays_and_overflow_bits(env, kb):
    """The host calls serve every single-value layout: struct-of-arrays slots and tables
    with overflow bits give the oracle's results."""
    wc, torch = env
    n = 250_001
    keys = wc_inputs.distinct_u32(0x4070 + kb, n) if kb == 4 else wc_inputs.distinct_u64(0x4070 + kb, n)
    vals = (wc_inputs.uniform_u32(0x4071, n) if kb == 4 else wc_inputs.uniform_u64(0x4071, n)).astype(keys.dtype)
    other = wc_inputs.distinct_u32(0x4072, 100_000) if kb == 4 else wc_inputs.distinct_u64(0x4072, 100_000)
    q = np.concatenate([keys[::2], other[~np.isin(other, keys)]])
    o = oracle.SingleValue(kb, kb)
    o.insert(keys, vals)
    eo, ef, _ = o.retrieve(q)
    for opt in (wc.WC_OPT_SOA, wc.WC_OPT_OVERFLOW_BITS, wc.WC_OPT_SOA | wc.WC_OPT_OVERFLOW_BITS):
        t = wc.SingleValueTable(kb, kb, min_capacity=int(n / 0.9), options=opt)
        wc.api.wc_insert_host(t.handle, pinned(torch, keys), pinned(torch, vals))
        ho, hf = np.empty_like(q), np.empty(q.size, np.uint8)
        wc.api.wc_retrieve_host(t.handle, q, ho, hf)
        torch.cuda.synchronize()
        assert t.size() == n
        np.testing.assert_array_equal(hf, ef)
        np.testing.assert_array_equal(ho[ef == 1], eo[ef == 1])
