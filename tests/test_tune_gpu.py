"""Autotuner: picks valid launch shapes, caches them, and the tuned table still matches
the oracle."""
from __future__ import annotations

import json

import numpy as np
import pytest

import oracle
import wc_inputs

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


# ---- the library's own autotuner (include/wc_tune.h) and window_width = 0 ------------------

SIZES = {(0, 4, 4): 8, (0, 8, 8): 16, (4, 4, 4): 8, (4, 8, 8): 16, (3, 4, 0): 4, (3, 8, 0): 8}  # slot bytes
WIDTHS = {4: (8, 16, 32), 8: (4, 8, 16), 16: (2, 4, 8)}


def test_native_autotune_picks_valid_shapes_and_caches():
    """wc_autotune times every window width and group size on its own sample: the choice
    is a valid shape of an allowed width, a second call with the cache is answered from it
    unchanged, and a table of the chosen width accepts the shapes."""
    from paper_2009_07914_gb300 import build
    build.build()
    from paper_2009_07914_gb300 import api
    a = api.wc_autotune(0, 4, 4, load=0.9, sample_keys=1 << 16, use_cache=False)
    assert a["from_cache"] == 0 and a["window_width"] in WIDTHS[8]
    assert a["candidates"] >= 3 * 3 and all(ms > 0 for ms in a["ms"]) and a["sample_keys"] == 1 << 16
    b = api.wc_autotune(0, 4, 4, load=0.9, sample_keys=1 << 16, use_cache=True)
    c = api.wc_autotune(0, 4, 4, load=0.9, sample_keys=1 << 16, use_cache=True)
    assert b["from_cache"] == 0 and c["from_cache"] == 1
    assert {k: v for k, v in c.items() if k != "from_cache"} == {k: v for k, v in b.items() if k != "from_cache"}
    h = api.wc_table_create(0, 4, 4, 1 << 12, a["window_width"], 0, 0x5EED, 0)
    api.wc_table_apply_tuning(h, a)
    for op in range(3):
        assert api.wc_table_get_launch(h, op) == a["launch"][op]
    api.wc_table_destroy(h)
    # a fixed width is kept; unsupported kinds and bad arguments are refused
    f = api.wc_autotune(0, 8, 8, window_width=4, load=0.8, sample_keys=1 << 14, use_cache=False)
    assert f["window_width"] == 4
    for bad in (dict(kind=1), dict(load=1.0), dict(sample_keys=100), dict(options=2)):
        args = dict(kind=0, key_bytes=4, value_bytes=4, load=0.9, sample_keys=1 << 14, use_cache=False)
        args.update(bad)
        with pytest.raises(Exception):
            api.wc_autotune(**args)
    h = api.wc_table_create(0, 4, 4, 1 << 12, 16, 0, 0x5EED, 0)
    with pytest.raises(Exception):  # a tuning for another window width
        api.wc_table_apply_tuning(h, dict(a, window_width=8 if a["window_width"] != 8 else 4))
    api.wc_table_destroy(h)


@pytest.mark.parametrize("kind,kb,vb", sorted(SIZES))
def test_window_zero_tables_are_tuned_and_match_the_oracle(kind, kb, vb):
    """window_width = 0: the table takes the width and shapes of the cached tuning for its
    kind and widths (small tables: a 2^20-key sample at load 0.9), and the tuned table
    gives the oracle's results for insert, lookup and erase."""
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    from paper_2009_07914_gb300 import api
    n = 30000
    seed = 7000 + 10 * kind + kb
    keys = (wc_inputs.distinct_u32(seed, 2 * n) if kb == 4 else wc_inputs.distinct_u64(seed, 2 * n))
    ins, absent = keys[:n], keys[n:]
    q = np.concatenate([ins[::2], absent[: n // 2]])
    if kind == 3:
        t = wc.HashSetTable(kb, min_capacity=int(n / 0.85))
        o = oracle.HashSet(kb)
    elif kind == 4:
        t = wc.CountingTable(kb, min_capacity=int(n / 0.85))
        o = oracle.Counting(kb)
    else:
        t = wc.SingleValueTable(kb, vb, min_capacity=int(n / 0.85))
        o = oracle.SingleValue(kb, vb)
    tu = api.wc_autotune(kind, kb, vb, load=0.9, sample_keys=1 << 20, use_cache=True)
    assert tu["from_cache"] == 1  # the create above tuned and cached it
    assert t.info["window_width"] == tu["window_width"] in WIDTHS[SIZES[(kind, kb, vb)]]
    for op in range(3):
        assert api.wc_table_get_launch(t.handle, op) == tu["launch"][op]
    if kind == 3:
        assert t.insert(ins) == 0
        o.insert(ins)
        got, _ = t.contains(q)
        np.testing.assert_array_equal(got, o.contains(q)[0])
        t.erase(ins[: n // 3])
        o.erase(ins[: n // 3])
        got, _ = t.contains(q)
        np.testing.assert_array_equal(got, o.contains(q)[0])
    else:
        vals = (np.arange(n, dtype=np.uint64) * 2654435761 + 1).astype(np.uint32 if vb == 4 else np.uint64)
        if kind == 4:
            t.insert(ins, vals)
            o.insert(ins, vals)
        else:
            assert t.insert(ins, vals) == 0
            o.insert(ins, vals)
        out, found, _ = t.retrieve(q)
        eo, ef, _ = o.retrieve(q)
        np.testing.assert_array_equal(found, ef)
        np.testing.assert_array_equal(out, eo)
        t.erase(ins[: n // 3])
        o.erase(ins[: n // 3])
        out, found, _ = t.retrieve(q)
        eo, ef, _ = o.retrieve(q)
        np.testing.assert_array_equal(found, ef)
        np.testing.assert_array_equal(out, eo)
    assert t.size() == o.size()
    t.close()


def test_window_zero_without_tuning_is_the_64_byte_window(monkeypatch):
    """WC_AUTOTUNE=0: window_width = 0 gives W = 64 / slot bytes and the fixed default shapes,
    and bucket multi-value tables are never tuned."""
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    monkeypatch.setenv("WC_AUTOTUNE", "0")
    for (kind, kb, vb), sb in sorted(SIZES.items()):
        t = (wc.HashSetTable(kb, min_capacity=4096) if kind == 3 else
             wc.CountingTable(kb, min_capacity=4096) if kind == 4 else
             wc.SingleValueTable(kb, vb, min_capacity=4096))
        assert t.info["window_width"] == 64 // sb
        t.close()
    monkeypatch.delenv("WC_AUTOTUNE")
    m = wc.MultiValueTable(4, 4, min_capacity=4096, value_pool_capacity=1 << 14)
    assert m.info["window_width"] == 4
    m.close()
