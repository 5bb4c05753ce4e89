"""Hash quality of tables built on the GPU, against the textbook closed forms for uniform
hashing (Knuth, TAOCP vol. 3, open addressing): a successful search probes about
(1/a) ln(1/(1-a)) slots and an unsuccessful one about 1/(1-a).  A walk visits whole
windows of W slots, so the mean windows per lookup, measured on the slot dump by the
oracle, must stay at or below those slot-level values at every load.  Also: the overflow
bits shorten the walks of absent keys and leave those of present keys alone."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import wc_inputs

pytestmark = pytest.mark.gpu
SEED = 0x9A1


@pytest.fixture(scope="module")
def wc():
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    return wc


def built(wc, kb, W, alpha, n, opt=0):
    keys = wc_inputs.distinct_u32(0x9A2, n) if kb == 4 else wc_inputs.distinct_u64(0x9A2, n)
    vals = (wc_inputs.uniform_u32(0x9A3, n) if kb == 4 else wc_inputs.uniform_u64(0x9A3, n)).astype(keys.dtype)
    t = wc.SingleValueTable(kb, kb, min_capacity=int(n / alpha), window_width=W, seed=SEED, options=opt)
    assert t.insert(keys, vals) == 0 and t.size() == n
    other = wc_inputs.distinct_u32(0x9A4, 100_000) if kb == 4 else wc_inputs.distinct_u64(0x9A4, 100_000)
    return t, other[~np.isin(other, keys)]


@pytest.mark.parametrize("kb,W", [(4, 8), (4, 4), (8, 4), (8, 2)])
@pytest.mark.parametrize("alpha", [0.5, 0.8, 0.9, 0.95])
def test_walks_within_uniform_hashing_bounds(wc, kb, W, alpha):
    t, absent = built(wc, kb, W, alpha, 400_000)
    info = t.info
    a = t.size() / info["capacity"]
    r = oracle.walk_stats(wc.api.wc_table_dump_slots(t.handle), info["windows"], info["window_width"],
                          info["slot_bytes"], SEED, absent, key_bytes=kb)
    assert r["hits"] == t.size() and r["misses"] == absent.size
    assert 1.0 <= r["hit"] <= (1 / a) * math.log(1 / (1 - a)), (r, a)
    assert 1.0 <= r["miss"] <= 1 / (1 - a), (r, a)


def test_overflow_bits_shorten_absent_walks(wc):
    """2^22 uint32 pairs at load 0.9, W = 8: present keys walk the same windows with or
    without the bits; absent keys walk less than 60 % as far with eight tagged bits."""
    n = 1 << 22
    plain, absent = built(wc, 4, 8, 0.9, n)
    tagged, _ = built(wc, 4, 8, 0.9, n, wc.WC_OPT_OVERFLOW_BITS)
    info = tagged.info
    bits = wc.api.wc_table_dump_overflow_bits(tagged.handle)
    r0 = oracle.walk_stats(wc.api.wc_table_dump_slots(plain.handle), info["windows"], 8, 8, SEED, absent)
    r1 = oracle.walk_stats(wc.api.wc_table_dump_slots(tagged.handle), info["windows"], 8, 8, SEED, absent, bits)
    assert abs(r0["hit"] - r1["hit"]) < 0.02, (r0, r1)
    assert r1["miss"] < 0.6 * r0["miss"], (r0, r1)
    assert 1.1 < r0["hit"] < 1.4 and r0["miss"] > 2.0, r0
