"""wc_insert_noalloc -- the insert for callers that cannot allocate device memory during
the call (memory budgeted up front, a device owned by another allocator) -- stores what
wc_insert stores and what the oracle's plain map holds: on two calls in a row into the same
table (the second also overwriting keys of the first), every key and as many absent keys
are retrieved and compared exactly with a table filled by wc_insert and with the oracle;
with overflow bits, the slot dump passes the oracle's reachability check and the dumped
bits equal the ones the oracle derives from it.  Also: a batch of exactly the documented
maximum, a batch one larger (refused), and keys in pageable host memory (refused on the
host, before anything runs on the GPU).  Collected last (file name) so that a failure here
stops a `-x` run only after every other test has run; runs alone in a fresh process too."""
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
    from paper_2009_07914_gb300 import api
    from paper_2009_07914_gb300.table import to_device
    return wc, api, torch, to_device


def _keys_values(kb, n, seed):
    if kb == 4:
        return wc_inputs.distinct_u32(seed, n), wc_inputs.uniform_u32(seed + 1, n)
    return wc_inputs.distinct_u64(seed, n), wc_inputs.uniform_u64(seed + 1, n)


def _check_layout(api, t, seed, bits_on):
    info = api.wc_table_get_info(t.handle)
    dump = api.wc_table_dump_slots(t.handle)
    bits = api.wc_table_dump_overflow_bits(t.handle) if bits_on else None
    r = oracle.check_slots(dump, info["windows"], info["window_width"], info["slot_bytes"], seed, True, bits)
    assert r["dups"] == 0 and r["unreachable"] == 0
    if bits_on:
        expect = oracle.overflow_bits_of(dump, info["windows"], info["window_width"], info["slot_bytes"], seed)
        assert np.array_equal(bits.view(np.uint8)[:info["windows"]], expect)
    return r["live"]


@pytest.mark.parametrize("kb", [4, 8])
@pytest.mark.parametrize("bits", [False, True], ids=["plain", "overflow_bits"])
def test_noalloc_insert_matches_wc_insert_and_oracle_on_two_calls(env, kb, bits):
    wc, api, torch, to_device = env
    dev = torch.device("cuda", 0)
    n1, n2, na = 700_001, 300_007, 200_000
    allk, allv = _keys_values(kb, n1 + n2 + na, 0x40A1)
    k1, k2 = allk[:n1], allk[n1:n1 + n2]
    v1, v2 = allv[:n1], allv[n1:n1 + n2]
    # the second call also overwrites some keys of the first (duplicate path)
    k2 = np.concatenate([k2, k1[:5000]])
    v2 = np.concatenate([v2, v2[:5000] ^ v2.dtype.type(0x77)])
    queries = allk[wc_inputs.shuffle_index(9, allk.size)]
    cap = int((n1 + n2) / 0.9) + 1
    opts = wc.WC_OPT_OVERFLOW_BITS if bits else 0
    ref = wc.SingleValueTable(kb, kb, min_capacity=cap, seed=0xAB, options=opts)
    tst = wc.SingleValueTable(kb, kb, min_capacity=cap, seed=0xAB, options=opts)
    orc = oracle.SingleValue(kb, kb)
    q = to_device(queries, kb, dev)
    for ks, vs in ((k1, v1), (k2, v2)):
        dk, dv = to_device(ks, kb, dev), to_device(vs, kb, dev)
        api.wc_insert(ref.handle, dk, dv)
        api.wc_insert_noalloc(tst.handle, dk, dv)
        flags = orc.insert(ks, vs)
        torch.cuda.synchronize()
        assert tst.status(clear=True) == ref.status(clear=True) == flags
        assert tst.size() == ref.size() == orc.size()
        ro, rf, _ = ref.retrieve(q)
        to, tf, _ = tst.retrieve(q)
        eo, ef, _ = orc.retrieve(queries)
        np.testing.assert_array_equal(tf, rf)
        np.testing.assert_array_equal(to, ro)
        np.testing.assert_array_equal(tf, ef)
        np.testing.assert_array_equal(to, eo)
        assert _check_layout(api, tst, 0xAB, bits) == orc.size()
    assert tst.size() == n1 + n2
    ref.close()
    tst.close()


def test_noalloc_insert_at_the_maximum_batch(env):
    """Exactly the documented maximum of 4+4-byte pairs, where the split values end at the
    end of the fixed buffer; then a second, small call into the same table."""
    wc, api, torch, to_device = env
    dev = torch.device("cuda", 0)
    limit = (api.WC_NOALLOC_SCRATCH_BYTES - 512) // 8
    assert limit == 2_097_088
    ks, vs = _keys_values(4, limit + 1000, 0x51)
    t = wc.SingleValueTable(4, 4, min_capacity=int(limit / 0.9) + 1, seed=0x77,
                            options=wc.WC_OPT_OVERFLOW_BITS)
    orc = oracle.SingleValue(4, 4)
    for a, b in ((0, limit), (limit, limit + 1000)):
        api.wc_insert_noalloc(t.handle, to_device(ks[a:b], 4, dev), to_device(vs[a:b], 4, dev))
        assert t.status(clear=True) == orc.insert(ks[a:b], vs[a:b]) == 0
        out, found, _ = t.retrieve(ks)
        eo, ef, _ = orc.retrieve(ks)
        np.testing.assert_array_equal(found, ef)
        np.testing.assert_array_equal(out, eo)
    assert t.size() == limit + 1000
    assert _check_layout(api, t, 0x77, True) == limit + 1000
    t.close()


def test_noalloc_insert_refuses_what_it_cannot_take(env):
    """A batch one pair beyond the buffer, and keys and values in pageable host memory
    (which the GPU cannot reach): WC_ERR_INVALID_ARG from the host, table unchanged."""
    wc, api, torch, to_device = env
    t = wc.SingleValueTable(4, 4, min_capacity=1 << 23)
    limit = (api.WC_NOALLOC_SCRATCH_BYTES - 512) // 8
    big = torch.zeros(limit + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(wc.WcError) as e:
        api.wc_insert_noalloc(t.handle, big, big)
    assert e.value.code == 1  # WC_ERR_INVALID_ARG
    host = torch.arange(1, 1025, dtype=torch.int32)  # pageable CPU memory
    dev_vals = torch.ones(1024, dtype=torch.int32, device="cuda")
    # raw addresses, so that the C ABI itself (not the Python binding) sees the host buffer
    with pytest.raises(wc.WcError) as e:
        api.wc_insert_noalloc(t.handle, host.data_ptr(), dev_vals, n=1024)
    assert e.value.code == 1
    with pytest.raises(wc.WcError) as e:
        api.wc_insert_noalloc(t.handle, dev_vals, host.data_ptr(), n=1024)
    assert e.value.code == 1
    assert t.size() == 0 and t.status() == 0
    t.close()
