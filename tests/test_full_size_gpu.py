"""Parity at the benchmark sizes, in the launch configuration bench.py times (default
shapes and schemes): every output is checked through properties that hold at any size
(found masks and values against the generator's bookkeeping, exact per-key counts and
value multisets), and a sampled subset against the CPU oracle."""
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
    from paper_2009_07914_gb300.table import to_device, to_numpy
    return wc, api, torch, to_device, to_numpy


def _sample(n, k, seed):
    return wc_inputs.shuffle_index(seed, n)[:k]


@pytest.fixture(scope="module")
def sv27():
    """The 2^27-pair workload of the single-value load sweep, generated once per module."""
    n = 1 << 27
    return n, wc_inputs.sv_insert_retrieve_u32(0x57C00002, n, n // 2, n // 2)


# (target load, table options): the bench's table (overflow bits) at every load of the
# paper's density sweep (Sec. V-A), and the plain table at the headline load.
SWEEP = [(0.9, 0), (0.9, 1), (0.5, 1), (0.8, 1), (0.95, 1), (0.99, 1)]


@pytest.mark.parametrize("alpha,opts", SWEEP, ids=["a%.2f-o%d" % x for x in SWEEP])
def test_sv_u32_2e27_load_sweep(env, sv27, alpha, opts):
    """2^27 unique uint32 pairs inserted at target load alpha, then 2^26 present + 2^26
    absent queries, in the bench's launch configuration (opts = 1: overflow bits, as
    bench.py times it).  Checked: no status flag (in particular no PROBE_LIMIT) and the
    exact size; found mask and values of every query against the generator's bookkeeping;
    a sample against the oracle; with the bits, the whole slot dump passes the
    reachability check and the dumped bits equal the ones the oracle derives from it;
    then an erase of 2^20 keys."""
    wc, api, torch, to_device, to_numpy = env
    n, d = sv27
    dev = torch.device("cuda", 0)
    keys, vals, q = (to_device(d[k], 4, dev) for k in ("keys", "values", "queries"))
    h = api.wc_table_create(0, 4, 4, int(np.ceil(n / alpha)), 0, 0, 0x5EEDC0DE, 0, options=opts)
    info = api.wc_table_get_info(h)
    assert n / info["capacity"] <= alpha and n / info["capacity"] > alpha - 0.001
    api.wc_insert(h, keys, vals)
    del keys, vals
    assert api.wc_get_status(h, True) == 0, "status flags after the insert"
    assert api.wc_size(h) == n
    if opts:
        dump = api.wc_table_dump_slots(h)
        bits = api.wc_table_dump_overflow_bits(h)
        r = oracle.check_slots(dump, info["windows"], info["window_width"], info["slot_bytes"], 0x5EEDC0DE, False,
                               bits)
        assert r == {"live": n, "dups": 0, "unreachable": 0}
        expect = oracle.overflow_bits_of(dump, info["windows"], info["window_width"], info["slot_bytes"], 0x5EEDC0DE)
        assert np.array_equal(bits.view(np.uint8)[:info["windows"]], expect)
        del dump, bits, expect
    out = torch.empty(n, dtype=torch.int32, device=dev)
    found = torch.empty(n, dtype=torch.uint8, device=dev)
    api.wc_retrieve(h, q, out, found)
    assert api.wc_get_status(h, True) == 0
    f = found.cpu().numpy()
    o = to_numpy(out, 4)
    pres = d["q_src"] >= 0
    assert np.array_equal(f, pres.astype(np.uint8))
    assert np.array_equal(o[pres], d["values"][d["q_src"][pres]])
    assert (o[~pres] == 0xFFFFFFFF).all()
    # oracle on a sample: the pairs behind 2^16 sampled queries
    idx = _sample(n, 1 << 16, 1)
    src = d["q_src"][idx]
    orc = oracle.SingleValue(4, 4)
    orc.insert(d["keys"][src[src >= 0]], d["values"][src[src >= 0]])
    eo, ef, _ = orc.retrieve(d["queries"][idx])
    assert np.array_equal(f[idx], ef) and np.array_equal(o[idx], eo)
    # erase 2^20 present keys, everything else unchanged
    drop = d["keys"][_sample(n, 1 << 20, 2)]
    api.wc_erase(h, to_device(drop, 4, dev))
    assert api.wc_size(h) == n - (1 << 20)
    api.wc_retrieve(h, to_device(drop, 4, dev), out, found, n=drop.size)
    assert not found[: drop.size].any().item()
    api.wc_retrieve(h, q, out, found)
    keep = np.ones(n, dtype=bool)
    keep[_sample(n, 1 << 20, 2)] = False  # positions of the erased keys in d["keys"]
    still = pres.copy()
    still[pres] = keep[d["q_src"][pres]]
    assert np.array_equal(found.cpu().numpy(), still.astype(np.uint8))
    assert api.wc_get_status(h, True) == 0
    api.wc_table_destroy(h)


def test_sv_u32_2e20_load_0p8_full_oracle(env):
    wc, api, torch, to_device, to_numpy = env
    n = 1 << 20
    d = wc_inputs.sv_insert_retrieve_u32(0x57C00001, n, n, n)
    t = wc.SingleValueTable(4, 4, min_capacity=int(np.ceil(n / 0.8)), l2_persist=True)
    o = oracle.SingleValue(4, 4)
    assert t.insert(d["keys"], d["values"]) == o.insert(d["keys"], d["values"])
    for step in range(2):
        out, found, _ = t.retrieve(d["queries"])
        eo, ef, _ = o.retrieve(d["queries"])
        assert np.array_equal(found, ef) and np.array_equal(out, eo)
        drop = d["keys"][_sample(n, n // 2, 0x57C00001)]
        if step == 0:
            t.erase(drop)
            o.erase(drop)
            assert t.size() == o.size() == n - n // 2


def test_sv_u64_2e28_zipf(env):
    wc, api, torch, to_device, to_numpy = env
    dev = torch.device("cuda", 0)
    n = 1 << 28
    d = wc_inputs.sv_u64_zipf(0x57C00003, n, n)
    keys, vals, q = (to_device(d[k], 8, dev) for k in ("keys", "values", "queries"))
    h = api.wc_table_create(0, 8, 8, int(np.ceil(n / 0.9)), 0, 0, 0x5EEDC0DE, 0)
    api.wc_insert(h, keys, vals)
    del keys, vals
    assert api.wc_size(h) == n and api.wc_get_status(h, True) == 0
    out = torch.empty(n, dtype=torch.int64, device=dev)
    found = torch.empty(n, dtype=torch.uint8, device=dev)
    api.wc_retrieve(h, q, out, found)
    assert int(found.sum().item()) == n
    o = to_numpy(out, 8)
    assert np.array_equal(o, d["values"][d["q_src"]])
    idx = _sample(n, 1 << 15, 3)
    orc = oracle.SingleValue(8, 8)
    orc.insert(d["keys"][d["q_src"][idx]], d["values"][d["q_src"][idx]])
    eo, _, _ = orc.retrieve(d["queries"][idx])
    assert np.array_equal(o[idx], eo)
    api.wc_table_destroy(h)


def test_mv_2e28_zipf_over_2e24(env):
    wc, api, torch, to_device, to_numpy = env
    dev = torch.device("cuda", 0)
    uni, n, na = 1 << 24, 1 << 28, 1 << 22
    d = wc_inputs.mv_zipf_u64(0x57C00004, uni, n, na)
    h = api.wc_table_create(1, 8, 4, int(np.ceil(uni / 0.8)), 0, n + (n >> 3), 0x5EEDC0DE, 0)
    api.wc_insert(h, to_device(d["keys"], 8, dev), to_device(d["values"], 4, dev))
    assert api.wc_size(h) == n and api.wc_get_status(h, True) == 0
    counts = np.bincount(d["ranks"], minlength=uni)
    assert api.wc_num_keys(h) == int((counts > 0).sum())
    q = to_device(d["queries"], 8, dev)
    nq = q.numel()
    offs = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    total = api.wc_count_values(h, q, offs)
    assert total == n
    offs_h = to_numpy(offs, 8).astype(np.int64)
    src = d["q_src"]
    want = np.where(src >= 0, counts[np.maximum(src, 0)], 0)
    assert np.array_equal(np.diff(offs_h), want)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    api.wc_retrieve_multi(h, q, offs, out)
    vals = to_numpy(out, 4)
    # every insert index comes back exactly once, inside the segment of its own key
    assert np.array_equal(np.sort(vals), np.arange(n, dtype=np.uint32))
    seg = np.repeat(np.arange(nq, dtype=np.int64), np.diff(offs_h))
    assert np.array_equal(src[seg], d["ranks"][vals])
    # oracle on a sample of queries: the pairs of their keys only
    idx = _sample(nq, 4096, 4)
    sq = src[idx]
    order = np.argsort(d["ranks"], kind="stable")
    starts = np.concatenate([[0], np.cumsum(counts)])
    orc = oracle.MultiValue(8, 4)
    for u in sq[sq >= 0]:
        ii = order[starts[u]:starts[u + 1]]
        orc.insert(d["keys"][ii], d["values"][ii])
    eoffs, _ = orc.count_values(d["queries"][idx])
    ev, _ = orc.retrieve_multi(d["queries"][idx], eoffs)
    got = np.concatenate([vals[offs_h[i]:offs_h[i + 1]] for i in idx]) if idx.size else np.zeros(0, np.uint32)
    goffs = np.concatenate([[0], np.cumsum(np.diff(offs_h)[idx])])
    assert np.array_equal(goffs, eoffs.astype(np.int64))
    assert np.array_equal(oracle.sorted_segments(got, goffs), oracle.sorted_segments(ev, eoffs))
    api.wc_table_destroy(h)


@pytest.mark.parametrize("r", [1, 64])
def test_mv_oa_2e28_uniform_r(env, r):
    """Open-addressing multi-value table at the benchmark size (2^28 uint32 pairs, keys
    uniform over 1..n/r, load 0.8, default shapes with the region-split insert): exact
    per-query counts against the generator's histogram, every insert index returned
    once inside its own key's segment, and a sample of queries against the oracle."""
    wc, api, torch, to_device, to_numpy = env
    dev = torch.device("cuda", 0)
    n = 1 << 28
    d = wc_inputs.mv_uniform_r(0x57C00005 + r, n, r)
    keys = d["keys"].astype(np.uint32)
    h = api.wc_table_create(2, 4, 4, int(np.ceil(n / 0.8)), 0, 0, 0x5EEDC0DE, 0)
    api.wc_insert(h, to_device(keys, 4, dev), to_device(d["values"], 4, dev))
    assert api.wc_size(h) == n and api.wc_get_status(h, True) == 0
    counts = np.bincount(keys, minlength=n + 1)
    q = to_device(np.arange(1, n + 1, dtype=np.uint32), 4, dev)
    offs = torch.empty(n + 1, dtype=torch.int64, device=dev)
    assert api.wc_count_values(h, q, offs) == n
    offs_h = to_numpy(offs, 8).astype(np.int64)
    assert np.array_equal(np.diff(offs_h), counts[1:])
    out = torch.empty(n, dtype=torch.int32, device=dev)
    api.wc_retrieve_multi(h, q, offs, out)
    vals = to_numpy(out, 4)
    assert np.array_equal(np.sort(vals), np.arange(n, dtype=np.uint32))
    seg = np.repeat(np.arange(1, n + 1, dtype=np.uint32), counts[1:])
    assert np.array_equal(seg, keys[vals])
    del seg
    if r == 1:
        assert api.wc_num_keys(h) == int((counts > 0).sum())
    # oracle on a sample of queries: the pairs of their keys only
    qi = _sample(n, 4096, 6)
    qk = (qi + 1).astype(np.uint32)
    sel = np.isin(keys, qk)
    orc = oracle.MultiValue(4, 4)
    orc.insert(keys[sel], d["values"][sel])
    eoffs, _ = orc.count_values(qk)
    ev, _ = orc.retrieve_multi(qk, eoffs)
    got = np.concatenate([vals[offs_h[i]:offs_h[i + 1]] for i in qi])
    goffs = np.concatenate([[0], np.cumsum(np.diff(offs_h)[qi])])
    assert np.array_equal(goffs, eoffs.astype(np.int64))
    assert np.array_equal(oracle.sorted_segments(got, goffs), oracle.sorted_segments(ev, eoffs))
    api.wc_table_destroy(h)
