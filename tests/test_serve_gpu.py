"""Serving loop: admission by HBM budget, continuous batching into the batched executor,
per-call baseline.  Every request's result must be the same served in the mix (either
mode) as run alone in arrival order (the CPU oracle applied one request at a time)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import wc_inputs
from tests.test_exec_gpu import _oracle_apply, _oracles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2009_07914_gb300 import build
    build.build()
    import torch

    from paper_2009_07914_gb300 import serve
    return serve, torch


@pytest.mark.parametrize("mode,solo", [(0, 0), (0, 2000), (1, 0)])
def test_results_equal_alone_and_in_the_mix(env, mode, solo):
    serve, torch = env
    tr = wc_inputs.serving_trace(77, n_tables=8, log2_cap=(12, 18), n_requests=120, log2_batch=(6, 14))
    dt = serve.DeviceTrace(tr, window_width=8)
    dt.reset()
    arr = wc_inputs.poisson_arrivals(5, len(tr["requests"]), rate_per_s=20_000.0)
    ex = serve.wc_executor_create(0, 8, max_items=64, tile_keys=1024) if mode == 0 else None
    reqs = dt.requests(arr)
    tim, st = serve.wc_serve_run(ex, reqs, mode, hbm_budget_bytes=1 << 30, max_batch_items=64, max_inflight=2,
                                 solo_min_keys=solo)
    assert st["keys"] == sum(r["keys"].size for r in tr["requests"])
    assert (tim["completed_ns"] >= tim["launched_ns"]).all() and (tim["launched_ns"] >= tim["admitted_ns"]).all()
    assert (tim["admitted_ns"] >= arr).all()
    expect = _oracle_apply(_oracles(tr), tr)
    for got, exp in zip(dt.retrieve_results(), expect):
        if exp is not None:
            np.testing.assert_array_equal(got[1], exp[1])
            np.testing.assert_array_equal(got[0], exp[0])
    ors = _oracles(tr)
    _oracle_apply(ors, tr)
    assert dt.sizes() == [o.size() for o in ors]
    if mode == 0:
        # all requests at once: the device is never idle with one request waiting, so the
        # executor coalesces them; the results stay those of the oracle
        dt.reset()
        reqs = dt.requests(np.zeros(len(tr["requests"]), dtype=np.uint64))
        tim, st = serve.wc_serve_run(ex, reqs, mode, hbm_budget_bytes=1 << 30, max_batch_items=64, max_inflight=2,
                                     solo_min_keys=solo)
        assert st["launches"] < len(reqs)  # requests were coalesced
        for got, exp in zip(dt.retrieve_results(), expect):
            if exp is not None:
                np.testing.assert_array_equal(got[1], exp[1])
                np.testing.assert_array_equal(got[0], exp[0])
        serve.wc_executor_destroy(ex)
    dt.close()


def test_admission_respects_the_hbm_budget(env):
    serve, torch = env
    tr = wc_inputs.serving_trace(78, n_tables=4, log2_cap=(12, 16), n_requests=40, log2_batch=(8, 12))
    dt = serve.DeviceTrace(tr, window_width=8)
    dt.reset()
    reqs = dt.requests(np.zeros(len(tr["requests"]), dtype=np.uint64))  # all arrive at once
    biggest = max(r.io_bytes for r in reqs)
    from paper_2009_07914_gb300 import api
    resident = sum(i["device_bytes"] + i["work_bytes"] for i in map(api.wc_table_get_info, dt.tables))
    budget = resident + 2 * biggest
    ex = serve.wc_executor_create(0, 8, max_items=64, tile_keys=1024)
    # the tables alone do not fit in a budget of their own size minus one byte
    with pytest.raises(Exception):
        serve.wc_serve_run(ex, reqs, 0, hbm_budget_bytes=resident - 1, max_batch_items=64, max_inflight=2)
    tim, st = serve.wc_serve_run(ex, reqs, 0, hbm_budget_bytes=budget, max_batch_items=64, max_inflight=2)
    assert st["resident_bytes"] == resident
    assert resident < st["peak_admitted_bytes"] <= budget
    assert st["launches"] >= 2
    # admission is in arrival order
    order = np.argsort(tim["admitted_ns"], kind="stable")
    assert (np.diff(tim["admitted_ns"][order]) >= 0).all()
    expect = _oracle_apply(_oracles(tr), tr)
    for got, exp in zip(dt.retrieve_results(), expect):
        if exp is not None:
            np.testing.assert_array_equal(got[0], exp[0])
    serve.wc_executor_destroy(ex)
    dt.close()


def _sharded_oracles(trace):
    os_ = []
    for k, v in zip(trace["prefill_keys"], trace["prefill_vals"]):
        o = oracle.ShardedSingleValue(4, 4)
        o.insert(k, v)
        os_.append(o)
    return os_


@pytest.mark.slow
def test_served_workload_at_its_own_scale(env):
    """The batched + served workload at its own scale: 64 tables of capacity 2^U(16, 26)
    pre-filled to load U(0, 0.6), 160 requests of 2^U(log2 1000, 24) keys (insert /
    retrieve / erase 60 / 35 / 5, inserts clamped to load 0.9).  Served three times from
    the same start -- batched with Poisson arrivals, batched closed loop, per call with
    Poisson arrivals -- every retrieve result (values and found masks) and every table
    size equals the oracle's with the requests applied one at a time in arrival order."""
    serve, torch = env
    tr = wc_inputs.serving_trace(0x57C00005, n_tables=64, n_requests=160)
    nreq = len(tr["requests"])
    assert max(r["keys"].size for r in tr["requests"]) > (1 << 22)
    ors = _sharded_oracles(tr)
    expect = _oracle_apply(ors, tr)
    sizes = [o.size() for o in ors]
    del ors
    dt = serve.DeviceTrace(tr, window_width=8)
    ex = serve.wc_executor_create(0, 8, max_items=1024, tile_keys=4096)
    poisson = wc_inputs.poisson_arrivals(0x5E5, nreq, rate_per_s=10_000.0)
    from paper_2009_07914_gb300 import api
    for mode, arr in ((0, poisson), (0, np.zeros(nreq, dtype=np.uint64)), (1, poisson)):
        dt.reset()
        # after the pre-fill, which may have grown the tables' scratch
        resident = sum(i["device_bytes"] + i["work_bytes"] for i in map(api.wc_table_get_info, dt.tables))
        # the tables' own bytes plus 1 GiB for the requests' buffers: binds when they queue
        tim, st = serve.wc_serve_run(ex if mode == 0 else None, dt.requests(arr), mode,
                                     hbm_budget_bytes=resident + (1 << 30), max_batch_keys=1 << 26,
                                     max_batch_items=1024, max_inflight=2)
        assert st["peak_admitted_bytes"] <= resident + (1 << 30)
        assert st["keys"] == sum(r["keys"].size for r in tr["requests"])
        assert (tim["completed_ns"] >= tim["launched_ns"]).all() and (tim["admitted_ns"] >= arr).all()
        for i, (got, exp) in enumerate(zip(dt.retrieve_results(), expect)):
            if exp is not None:
                np.testing.assert_array_equal(got[1], exp[1], err_msg="found mask of request %d" % i)
                np.testing.assert_array_equal(got[0], exp[0], err_msg="values of request %d" % i)
        assert dt.sizes() == sizes
        if mode == 0:
            assert serve.wc_executor_get_status(ex, clear=True) == 0
            if not arr.any():
                assert st["launches"] < nreq  # all at once: requests were coalesced
    serve.wc_executor_destroy(ex)
    dt.close()
