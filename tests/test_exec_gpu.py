"""Batched executor (one persistent kernel for many tables' bulk operations) against the
CPU oracle applied in submission order."""
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
    from paper_2009_07914_gb300 import serve
    return wc, serve, torch


def _oracle_apply(oracles, trace):
    expect = []
    for r in trace["requests"]:
        o = oracles[r["table"]]
        if r["op"] == 0:
            o.insert(r["keys"], r["values"])
            expect.append(None)
        elif r["op"] == 2:
            o.erase(r["keys"])
            expect.append(None)
        else:
            out, found, _ = o.retrieve(r["keys"])
            expect.append((out, found))
    return expect


def _oracles(trace):
    os_ = []
    for k, v in zip(trace["prefill_keys"], trace["prefill_vals"]):
        o = oracle.SingleValue(4, 4)
        o.insert(k, v)
        os_.append(o)
    return os_


@pytest.mark.parametrize("W", [4, 8, 16])
def test_executor_matches_oracle_in_submission_order(env, W):
    wc, serve, torch = env
    tr = wc_inputs.serving_trace(11 + W, n_tables=6, log2_cap=(10, 17), n_requests=80, log2_batch=(0, 14))
    dt = serve.DeviceTrace(tr, window_width=W)
    dt.reset()
    ex = serve.wc_executor_create(0, W, max_items=64, tile_keys=1024)
    works = dt.works()
    tickets = [serve.wc_executor_submit(ex, works[i:i + 17]) for i in range(0, len(works), 17)]
    serve.wc_executor_wait(ex, tickets[-1])
    assert all(serve.wc_executor_query(ex, t) for t in tickets)
    last = works[(len(tickets) - 1) * 17:]
    assert all(serve.wc_executor_query_item(ex, tickets[-1], j) for j in range(len(last)))
    assert serve.wc_executor_get_status(ex) == 0
    expect = _oracle_apply(_oracles(tr), tr)
    for got, exp in zip(dt.retrieve_results(), expect):
        if exp is None:
            continue
        np.testing.assert_array_equal(got[1], exp[1])
        np.testing.assert_array_equal(got[0], exp[0])
    ors = _oracles(tr)
    _oracle_apply(ors, tr)
    assert dt.sizes() == [o.size() for o in ors]
    serve.wc_executor_destroy(ex)
    dt.close()


def test_executor_bounded_wait_reports_timeout(env):
    """A dependency that never completes (test hook) makes the waiting tiles give up
    after the deadline: the kernel returns and the status word says so."""
    wc, serve, torch = env
    from paper_2009_07914_gb300.table import to_device
    dev = torch.device("cuda", 0)
    t = wc.SingleValueTable(4, 4, min_capacity=4096, window_width=8)
    keys = to_device(wc_inputs.distinct_u32(3, 1000), 4, dev)
    vals = to_device(wc_inputs.uniform_u32(4, 1000), 4, dev)
    out = torch.empty(1000, dtype=torch.int32, device=dev)
    ex = serve.wc_executor_create(0, 8, max_items=8, tile_keys=256, timeout_ns=50_000_000, test_stall=True)
    tk = serve.wc_executor_submit(ex, [serve.work(0, t.handle, keys, vals),
                                       serve.work(1, t.handle, keys, values_out=out)])
    serve.wc_executor_wait(ex, tk)
    assert serve.wc_executor_get_status(ex, clear=True) & wc.WC_FLAG_QUEUE_TIMEOUT
    assert t.status(clear=True) & wc.WC_FLAG_QUEUE_TIMEOUT
    # the executor stays usable after a timeout
    serve.wc_executor_destroy(ex)
    ex = serve.wc_executor_create(0, 8, max_items=8, tile_keys=256)
    tk = serve.wc_executor_submit(ex, [serve.work(1, t.handle, keys, values_out=out)])
    serve.wc_executor_wait(ex, tk)
    assert serve.wc_executor_get_status(ex) == 0
    serve.wc_executor_destroy(ex)
    t.close()


def test_executor_rejects_tables_it_cannot_serve(env):
    wc, serve, torch = env
    from paper_2009_07914_gb300._binding import WcError
    t64 = wc.SingleValueTable(8, 8, min_capacity=1024)
    t4 = wc.SingleValueTable(4, 4, min_capacity=1024, window_width=4)
    k = torch.ones(4, dtype=torch.int64, device="cuda")
    ex = serve.wc_executor_create(0, 8, max_items=8)
    for t in (t64, t4):
        with pytest.raises(WcError) as e:
            serve.wc_executor_submit(ex, [serve.work(2, t.handle, k)])
        assert e.value.code == 6
    assert serve.wc_executor_submit(ex, []) >= 0
    serve.wc_executor_destroy(ex)
