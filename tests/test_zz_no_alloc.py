"""wc_insert_noalloc -- the insert for callers that cannot allocate device memory during
the call -- gives the same table as wc_insert (compared through retrieves of every key
and of absent keys, exact), on two calls in a row into the same table, and rejects a
batch larger than its fixed buffer.  Collected last (file name) so that a failure here
stops a `-x` run only after every other test has run."""
from __future__ import annotations

import numpy as np
import pytest

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


@pytest.mark.parametrize("kb", [4, 8])
def test_noalloc_insert_matches_wc_insert_on_two_calls(env, kb):
    wc, api, torch, to_device = env
    dev = torch.device("cuda", 0)
    n1, n2, na = 700_001, 300_007, 200_000
    if kb == 4:
        allk = wc_inputs.distinct_u32(0x40A1, n1 + n2 + na)
        v1, v2 = wc_inputs.uniform_u32(1, n1), wc_inputs.uniform_u32(2, n2)
    else:
        allk = wc_inputs.distinct_u64(0x40A1, n1 + n2 + na)
        v1, v2 = wc_inputs.uniform_u64(1, n1), wc_inputs.uniform_u64(2, n2)
    k1, k2 = allk[:n1], allk[n1:n1 + n2]
    # the second call also overwrites some keys of the first (duplicate path)
    k2 = np.concatenate([k2, k1[:5000]])
    v2 = np.concatenate([v2, v2[:5000] ^ v2.dtype.type(0x77)])
    queries = allk[wc_inputs.shuffle_index(9, allk.size)]
    cap = int((n1 + n2) / 0.9) + 1
    ref = wc.SingleValueTable(kb, kb, min_capacity=cap, seed=0xAB)
    tst = wc.SingleValueTable(kb, kb, min_capacity=cap, seed=0xAB)
    q = to_device(queries, kb, dev)
    for ks, vs in ((k1, v1), (k2, v2)):
        dk, dv = to_device(ks, kb, dev), to_device(vs, kb, dev)
        api.wc_insert(ref.handle, dk, dv)
        api.wc_insert_noalloc(tst.handle, dk, dv)
        torch.cuda.synchronize()
        assert ref.status(clear=True) == tst.status(clear=True)
        assert ref.size() == tst.size()
        ro, rf, _ = ref.retrieve(q)
        to, tf, _ = tst.retrieve(q)
        np.testing.assert_array_equal(tf, rf)
        np.testing.assert_array_equal(to, ro)
    assert tst.size() == n1 + n2
    ref.close()
    tst.close()


def test_noalloc_insert_rejects_batches_beyond_its_buffer(env):
    wc, api, torch, to_device = env
    t = wc.SingleValueTable(4, 4, min_capacity=1 << 23)
    limit = (api.WC_NOALLOC_SCRATCH_BYTES - 512) // 8
    big = torch.zeros(limit + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(wc.WcError) as e:
        api.wc_insert_noalloc(t.handle, big, big)
    assert e.value.code == 1  # WC_ERR_INVALID_ARG
    assert t.size() == 0
    t.close()
