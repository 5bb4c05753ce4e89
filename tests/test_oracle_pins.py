"""Pins of the CPU oracle to things other than itself (no GPU needed).

* brute force: a list of (key, value) pairs searched by linear scan, written
  independently of the oracle, on tiny random operation sequences that mix insert,
  duplicate insert, erase, re-insert after erase and sentinel keys;
* invariants of the paper's definitions (every inserted key found, absent keys
  NOT_FOUND, size = distinct live keys, MV counts sum to the inserts, offsets are the
  exclusive prefix sum with offsets[n] = total);
* the paper's multi-value benchmark invariant (Sec. V-C): keys from 1..n/r queried over
  1..n return exactly n values;
* hand-derived worked examples under tests/golden/ (each line cites its section);
* the sharded multi-core form of the single-value oracle against the same brute force.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import wc_inputs
from tests.golden_fixtures import run_mv, run_sv

NF32 = 0xFFFFFFFF


class BruteSV:
    """Single-value semantics by linear scan over a list of pairs."""

    def __init__(self, kmax):
        self.pairs = []
        self.kmax = kmax

    def _find(self, k):
        for i, (kk, _) in enumerate(self.pairs):
            if kk == k:
                return i
        return -1

    def insert(self, ks, vs):
        f = 0
        for k, v in zip(ks, vs):
            if k == 0 or k == self.kmax:
                f |= 2
                continue
            i = self._find(k)
            if i < 0:
                self.pairs.append((k, v))
            else:
                self.pairs[i] = (k, v)
                f |= 1
        return f

    def erase(self, ks):
        f = 0
        for k in ks:
            if k == 0 or k == self.kmax:
                f |= 2
                continue
            i = self._find(k)
            if i >= 0:
                self.pairs.pop(i)
        return f

    def retrieve(self, ks, nf):
        out, found, f = [], [], 0
        for k in ks:
            if k == 0 or k == self.kmax:
                f |= 2
            i = -1 if (k == 0 or k == self.kmax) else self._find(k)
            out.append(self.pairs[i][1] if i >= 0 else nf)
            found.append(1 if i >= 0 else 0)
        return out, found, f


class BruteMV:
    def __init__(self, kmax):
        self.pairs = []
        self.kmax = kmax

    def insert(self, ks, vs):
        for k, v in zip(ks, vs):
            if k != 0 and k != self.kmax:
                self.pairs.append((k, v))

    def erase(self, ks):
        drop = {k for k in ks}
        self.pairs = [(k, v) for (k, v) in self.pairs if k not in drop]

    def values_of(self, k):
        return sorted(v for (kk, v) in self.pairs if kk == k)


@pytest.mark.parametrize("kb,vb", [(4, 4), (8, 8), (8, 4)])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sv_oracle_matches_brute_force(kb, vb, seed):
    kmax = (1 << (8 * kb)) - 1
    vmax = (1 << (8 * vb)) - 1
    kdt = np.uint32 if kb == 4 else np.uint64
    vdt = np.uint32 if vb == 4 else np.uint64
    rng = np.random.default_rng(seed)
    o = oracle.SingleValue(kb, vb)
    b = BruteSV(kmax)
    universe = np.array([0, kmax] + list(rng.integers(1, kmax, 40, dtype=np.uint64)), dtype=np.uint64)
    for step in range(60):
        op = rng.integers(0, 3)
        m = int(rng.integers(0, 12))
        ks = universe[rng.integers(0, universe.size, m)].astype(kdt)
        if op == 0:
            vs = rng.integers(0, vmax, m, dtype=np.uint64, endpoint=True).astype(vdt)
            # the oracle applies a batch in call order; so does the brute force
            assert o.insert(ks, vs) == b.insert([int(x) for x in ks], [int(x) for x in vs])
        elif op == 1:
            assert o.erase(ks) == b.erase([int(x) for x in ks])
        else:
            out, found, f = o.retrieve(ks)
            bo, bf, bfl = b.retrieve([int(x) for x in ks], vmax)
            assert [int(x) for x in out] == bo
            assert [int(x) for x in found] == bf
            assert f == bfl
        assert o.size() == len(b.pairs)


@pytest.mark.parametrize("kb,vb", [(4, 4), (8, 8)])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_sharded_sv_oracle_matches_brute_force(kb, vb, threads):
    """The sharded (multi-core) single-value oracle against the same linear-scan brute
    force, on batches that repeat keys inside one batch (so a shard's input order
    matters) and mix erase and sentinels."""
    kmax = (1 << (8 * kb)) - 1
    vmax = (1 << (8 * vb)) - 1
    kdt = np.uint32 if kb == 4 else np.uint64
    vdt = np.uint32 if vb == 4 else np.uint64
    rng = np.random.default_rng(100 + threads)
    o = oracle.ShardedSingleValue(kb, vb, threads=threads)
    b = BruteSV(kmax)
    universe = np.array([0, kmax] + list(rng.integers(1, kmax, 60, dtype=np.uint64)), dtype=np.uint64)
    for step in range(80):
        op = rng.integers(0, 3)
        m = int(rng.integers(0, 40))
        ks = universe[rng.integers(0, universe.size, m)].astype(kdt)
        if op == 0:
            vs = rng.integers(0, vmax, m, dtype=np.uint64, endpoint=True).astype(vdt)
            assert o.insert(ks, vs) == b.insert([int(x) for x in ks], [int(x) for x in vs])
        elif op == 1:
            assert o.erase(ks) == b.erase([int(x) for x in ks])
        else:
            out, found, f = o.retrieve(ks)
            bo, bf, bfl = b.retrieve([int(x) for x in ks], vmax)
            assert [int(x) for x in out] == bo
            assert [int(x) for x in found] == bf
            assert f == bfl
        assert o.size() == len(b.pairs)


@pytest.mark.parametrize("kb,vb", [(4, 4), (8, 4), (8, 8)])
@pytest.mark.parametrize("seed", [4, 5])
def test_mv_oracle_matches_brute_force(kb, vb, seed):
    kmax = (1 << (8 * kb)) - 1
    kdt = np.uint32 if kb == 4 else np.uint64
    vdt = np.uint32 if vb == 4 else np.uint64
    rng = np.random.default_rng(seed)
    o = oracle.MultiValue(kb, vb)
    b = BruteMV(kmax)
    universe = np.array([0, kmax] + list(rng.integers(1, 1000, 15)), dtype=np.uint64)
    for step in range(40):
        op = rng.integers(0, 3)
        m = int(rng.integers(0, 16))
        ks = universe[rng.integers(0, universe.size, m)].astype(kdt)
        if op == 0:
            vs = rng.integers(0, 50, m).astype(vdt)  # small range: equal values repeat
            o.insert(ks, vs)
            b.insert([int(x) for x in ks], [int(x) for x in vs])
        elif op == 1 and rng.random() < 0.3:
            o.erase(ks)
            b.erase([int(x) for x in ks])
        else:
            offs, _ = o.count_values(ks)
            out, _ = o.retrieve_multi(ks, offs)
            assert int(offs[0]) == 0
            for i, k in enumerate(ks):
                seg = sorted(int(x) for x in out[int(offs[i]):int(offs[i + 1])])
                want = [] if int(k) in (0, kmax) else b.values_of(int(k))
                assert seg == want
        assert o.size() == len(b.pairs)


def test_sv_invariants_random_batch():
    d = wc_inputs.sv_insert_retrieve_u32(11, 50_000, 20_000, 20_000)
    o = oracle.SingleValue(4, 4)
    assert o.insert(d["keys"], d["values"]) == 0
    assert o.size() == d["keys"].size
    out, found, _ = o.retrieve(d["queries"])
    pres = d["q_src"] >= 0
    assert found[pres].all() and not found[~pres].any()
    assert (out[pres] == d["values"][d["q_src"][pres]]).all()
    assert (out[~pres] == NF32).all()
    # erase half, the rest stays; size = distinct live keys
    o.erase(d["keys"][::2])
    assert o.size() == d["keys"].size - d["keys"][::2].size
    out, found, _ = o.retrieve(d["keys"])
    assert not found[::2].any() and found[1::2].all()
    assert (out[1::2] == d["values"][1::2]).all()


@pytest.mark.parametrize("r", [1, 2, 3, 8, 64])
def test_mv_paper_invariant_total_equals_n(r):
    """Sec. V-C: n keys drawn from 1..n/r, queried over 1..n -> exactly n values."""
    n = 4096
    d = wc_inputs.mv_uniform_r(100 + r, n, r)
    o = oracle.MultiValue(8, 4)
    o.insert(d["keys"], d["values"])
    offs, _ = o.count_values(d["queries"])
    assert int(offs[-1]) == n
    assert np.all(np.diff(offs.astype(np.int64)) >= 0)
    out, _ = o.retrieve_multi(d["queries"], offs)
    # every inserted value comes back exactly once (values are the insert indices)
    assert np.array_equal(np.sort(out), np.arange(n, dtype=np.uint32))
    # and each lands in its own key's segment
    seg_of = np.repeat(np.arange(n), np.diff(offs.astype(np.int64)))
    assert np.array_equal(d["queries"][seg_of], d["keys"][out])


def test_mv_counts_sum_to_inserts_zipf():
    d = wc_inputs.mv_zipf_u64(9, 1 << 12, 1 << 15, 1 << 10)
    o = oracle.MultiValue(8, 4)
    o.insert(d["keys"], d["values"])
    assert o.size() == d["keys"].size
    offs, _ = o.count_values(d["queries"])
    assert int(offs[-1]) == d["keys"].size  # the universe covers every inserted key
    assert o.num_keys() == np.unique(d["keys"]).size


def test_golden_sv_worked_example():
    assert run_sv("sv_ops.txt", lambda: oracle.SingleValue(4, 4)) >= 10


def test_golden_mv_worked_example():
    assert run_mv("mv_ops.txt", lambda: oracle.MultiValue(8, 4)) >= 8


def test_sentinels_are_rejected():
    o = oracle.SingleValue(8, 8)
    f = o.insert(np.array([0, 2 ** 64 - 1, 3], dtype=np.uint64), np.array([1, 2, 3], dtype=np.uint64))
    assert f == oracle.FLAG_INVALID_KEY and o.size() == 1


# ---- counting table and hash set (Sec. IV: CountingHashTable, HashSet) ----------------------

@pytest.mark.parametrize("kb", [4, 8])
def test_counting_oracle_against_brute_force(kb):
    """Counts equal np.unique's occurrence counts (unit weights), weighted sums wrap at the
    key width, erase removes keys; sentinels are skipped and flagged."""
    rng = np.random.default_rng(40 + kb)
    top = (1 << (8 * kb)) - 1
    universe = np.unique(rng.integers(1, min(top, 2 ** 62), 500, dtype=np.uint64))
    o = oracle.Counting(kb)
    ref = {}
    mask = (1 << (8 * kb)) - 1
    for step in range(6):
        ks = universe[rng.integers(0, universe.size, 3000)]
        if step % 2:
            ws = rng.integers(0, top, ks.size, dtype=np.uint64, endpoint=True)
            assert o.insert(ks, ws) == 0
            for k, w in zip(ks.tolist(), ws.tolist()):
                ref[k] = (ref.get(k, 0) + w) & mask
        else:
            assert o.insert(ks) == 0
            u, c = np.unique(ks, return_counts=True)
            for k, n in zip(u.tolist(), c.tolist()):
                ref[k] = (ref.get(k, 0) + n) & mask
        if step == 3:
            drop = universe[:50]
            o.erase(drop)
            for k in drop.tolist():
                ref.pop(k, None)
        out, found, _ = o.retrieve(universe)
        want = np.array([ref.get(k, mask) for k in universe.tolist()], dtype=np.uint64)
        np.testing.assert_array_equal(found, np.array([k in ref for k in universe.tolist()], np.uint8))
        np.testing.assert_array_equal(out.astype(np.uint64), want)
        assert o.size() == len(ref)
    assert o.insert(np.array([0, mask, 5], dtype=np.uint64)) == oracle.FLAG_INVALID_KEY


@pytest.mark.parametrize("kb", [4, 8])
def test_hash_set_oracle_against_python_set(kb):
    rng = np.random.default_rng(50 + kb)
    universe = np.unique(rng.integers(1, 2 ** 31, 800, dtype=np.uint64))
    o = oracle.HashSet(kb)
    ref = set()
    for step in range(5):
        ks = universe[rng.integers(0, universe.size, 400)]
        f = o.insert(ks)
        dup = any(k in ref for k in ks.tolist()) or len(set(ks.tolist())) < ks.size
        assert f == (oracle.FLAG_DUPLICATE_KEY if dup else 0)
        ref.update(ks.tolist())
        if step == 2:
            o.erase(universe[::3])
            ref.difference_update(universe[::3].tolist())
        found, _ = o.contains(universe)
        np.testing.assert_array_equal(found, np.array([k in ref for k in universe.tolist()], np.uint8))
        assert o.size() == len(ref)


def test_bloom_oracle_no_false_negatives_and_formula_rate():
    """The oracle's blocked Bloom filter: every inserted key is found, and the false
    positive rate on absent keys matches the Poisson-averaged blocked-filter formula."""
    import math
    n, blocks, k = 20_000, 20_000 * 10 // 256, 7
    o = oracle.BloomFilter(4, blocks, k, 123)
    rng = np.random.default_rng(9)
    keys = np.unique(rng.integers(1, 2 ** 31, n + 500, dtype=np.uint64))[:n].astype(np.uint32)
    o.insert(keys)
    found, _ = o.contains(keys)
    assert found.all()
    absent = (rng.integers(1, 2 ** 31, 200_000, dtype=np.uint64).astype(np.uint32) | np.uint32(1 << 31))
    fp = o.contains(absent)[0].mean()
    lam, p, total, x = 256.0 * n / (blocks * 256), None, 0.0, 0
    p = math.exp(-lam)
    while x < 200:
        total += p * (1 - (1 - 1 / 256) ** (k * x)) ** k
        x += 1
        p *= lam / x
    assert abs(fp - total) < 0.12 * total, (fp, total)
    # plain (unblocked) Bloom filters do better: the blocked layout costs a little FP rate
    assert total > (1 - math.exp(-k * n / (blocks * 256))) ** k


def test_bloom_oracle_is_empty_then_monotone():
    """Properties of any Bloom filter, independent of how bits are chosen: an empty filter
    reports no key; inserting more keys never turns a present answer into an absent one;
    a key's answer does not depend on the order of the inserts; with one bit per key and a
    filter of a single block, a key is present exactly when some inserted key has its bit."""
    rng = np.random.default_rng(21)
    probe = rng.integers(1, 2 ** 31, 50_000, dtype=np.uint64).astype(np.uint32)
    o = oracle.BloomFilter(4, 64, 5, 77)
    assert not o.contains(probe)[0].any()
    keys = rng.integers(1, 2 ** 31, 6_000, dtype=np.uint64).astype(np.uint32)
    prev = np.zeros(probe.size, dtype=np.uint8)
    for part in np.array_split(keys, 6):
        o.insert(part)
        cur = o.contains(probe)[0]
        assert (cur >= prev).all()
        prev = cur
    r = oracle.BloomFilter(4, 64, 5, 77)
    r.insert(keys[::-1])
    assert np.array_equal(r.contains(probe)[0], prev)
    # one block, one bit per key: 256 bits, so exactly the probes sharing a bit with an
    # inserted key are present -- and every probe that is an inserted key is present
    one = oracle.BloomFilter(4, 1, 1, 5)
    one.insert(keys[:40])
    got = one.contains(probe)[0]
    assert got.mean() < 1.0 and one.contains(keys[:40])[0].all()
    # the filter has 256 bits; 40 keys set at most 40 of them, so at most 40/256 of the
    # probes can be present (each probe maps to one bit; equality with the share of set bits)
    assert got.mean() <= 40 / 256 + 0.01


def _fmix64_py(x: int) -> int:
    m = (1 << 64) - 1
    x ^= x >> 33
    x = (x * 0xFF51AFD7ED558CCD) & m
    x ^= x >> 33
    x = (x * 0xC4CEB9FE1A85EC53) & m
    x ^= x >> 33
    return x


@pytest.mark.parametrize("kb,k", [(4, 1), (4, 7), (8, 8), (8, 9), (4, 16)])
def test_bloom_oracle_equals_the_documented_bit_rule(kb, k):
    """Exact pin of the oracle's Bloom filter: a Python restatement of the documented rule
    (block = hi32(h) * blocks >> 32 with h = fmix64(key ^ seed); bit i = byte i % 8 of
    g_{i/8+1}, g_1 = fmix64(h ^ 0x9e3779b97f4a7c15), g_{j+1} = fmix64(g_j)) on a filter small
    enough that most answers are false positives, so any change of the rule shows."""
    blocks, seed = 37, 0xB10C
    rng = np.random.default_rng(k * 10 + kb)
    top = 2 ** 31 if kb == 4 else 2 ** 62
    dt = np.uint32 if kb == 4 else np.uint64
    keys = rng.integers(1, top, 2000, dtype=np.uint64).astype(dt)
    queries = np.concatenate([rng.integers(1, top, 3000, dtype=np.uint64).astype(dt), keys[:200]])

    def bits_of(key):
        h = _fmix64_py(int(key) ^ seed)
        block = ((h >> 32) * blocks) >> 32
        g, pos = h ^ 0x9E3779B97F4A7C15, []
        for i in range(k):
            if i % 8 == 0:
                g = _fmix64_py(g)
            pos.append((g >> (8 * (i % 8))) & 255)
        return block, pos

    set_bits = set()
    for key in keys:
        b, pos = bits_of(key)
        set_bits.update((b, p) for p in pos)
    expect = np.array([all((b, p) in set_bits for p in pos) for b, pos in map(bits_of, queries)], np.uint8)
    o = oracle.BloomFilter(kb, blocks, k, seed)
    o.insert(keys)
    found, _ = o.contains(queries)
    np.testing.assert_array_equal(found, expect)
    assert expect[3000:].all() and 0 < expect[:3000].mean() < 1  # inserted keys found; both answers occur
