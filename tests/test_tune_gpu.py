"""Autotuner: picks valid launch shapes, caches them, and the tuned table still matches
the oracle."""
from __future__ import annotations

import json

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_tune_table_sets_valid_shapes_and_keeps_parity(tmp_path, monkeypatch):
    from paper_2009_07914_gb300 import build
    build.build()
    monkeypatch.setenv("WC_TUNE_CACHE", str(tmp_path / "cache.json"))
    from paper_2009_07914_gb300 import api, tune
    from paper_2009_07914_gb300.table import to_numpy
    n = 1 << 16
    keys, values, queries = tune.sample(4, n)
    h = api.wc_table_create(0, 4, 4, int(n / 0.9) + 1, 8, 0, 0x5EED, 0)
    best = tune.tune_table(h, keys, values, queries, reps=1)
    for op, code in (("insert", 0), ("retrieve", 1), ("erase", 2)):
        lc = api.wc_table_get_launch(h, code)
        assert lc["group_size"] == best[op]["group"] and lc["group_size"] in tune.SHAPES[8][8]
    cache = json.load(open(tmp_path / "cache.json"))
    assert len(cache) == 3
    # second call is served from the cache
    again = tune.tune_table(h, keys, values, queries, reps=1)
    assert all(v.get("cached") for v in again.values())
    o = oracle.SingleValue(4, 4)
    o.insert(to_numpy(keys, 4), to_numpy(values, 4))
    import torch
    out = torch.empty(queries.numel(), dtype=torch.int32, device="cuda")
    found = torch.empty(queries.numel(), dtype=torch.uint8, device="cuda")
    api.wc_retrieve(h, queries, out, found)
    eo, ef, _ = o.retrieve(to_numpy(queries, 4))
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(to_numpy(out, 4), eo)
    api.wc_table_destroy(h)


def test_recommend_window_returns_a_valid_width():
    from paper_2009_07914_gb300 import tune
    best = tune.recommend_window(4, 4, 1 << 14, 0.9, reps=1, use_cache=False)
    assert best["W"] in (4, 8, 16, 32)


@pytest.mark.parametrize("W", [4, 8, 16])
def test_executor_runs_the_tuned_lane_shapes(tmp_path, monkeypatch, W):
    """tune.executor_groups picks lanes per key from the executor's instantiated sets; an
    executor built with them (and one with every other valid pair of the width) serves a
    mixed batch with the oracle's results."""
    monkeypatch.setenv("WC_TUNE_CACHE", str(tmp_path / "cache.json"))
    import wc_inputs
    from paper_2009_07914_gb300 import serve, tune
    from tests.test_exec_gpu import _oracle_apply, _oracles
    g = tune.executor_groups(W, n=1 << 14, reps=1)
    gi_set, gr_set = tune.EXEC_SHAPES[W]
    assert g["group_insert"] in gi_set and g["group_retrieve"] in gr_set
    pairs = {(g["group_insert"], g["group_retrieve"])} | {(i, r) for i in gi_set for r in gr_set}
    tr = wc_inputs.serving_trace(90 + W, n_tables=4, log2_cap=(10, 15), n_requests=40, log2_batch=(0, 12))
    expect = _oracle_apply(_oracles(tr), tr)
    for gi, gr in sorted(pairs):
        dt = serve.DeviceTrace(tr, window_width=W)
        dt.reset()
        ex = serve.wc_executor_create(0, W, max_items=64, tile_keys=1024, group_insert=gi, group_retrieve=gr)
        works = dt.works()
        t = serve.wc_executor_submit(ex, works)
        serve.wc_executor_wait(ex, t)
        assert serve.wc_executor_get_status(ex) == 0
        for got, exp in zip(dt.retrieve_results(), expect):
            if exp is not None:
                np.testing.assert_array_equal(got[1], exp[1])
                np.testing.assert_array_equal(got[0], exp[0])
        serve.wc_executor_destroy(ex)
        dt.close()
    with pytest.raises(Exception):
        serve.wc_executor_create(0, W, group_insert=8, group_retrieve=8)
