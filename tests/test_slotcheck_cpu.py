"""Pins of the slot-dump invariant checker (oracle.check_slots) on the CPU.

Valid dumps come from a brute-force insert written here with Python integers (walk the
key's windows, take the first empty slot of the first window that has one); mistakes are
then planted in those dumps -- an empty slot put back in front of a key, a key stored
twice, the wrong hash seed -- and each must be reported.  A tombstone in the same place
must not be (Sec. IV-B5: tombstones count as occupied for lookups)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

M64 = (1 << 64) - 1


def fmix64(k: int) -> int:
    k ^= k >> 33
    k = (k * 0xFF51AFD7ED558CCD) & M64
    k ^= k >> 33
    k = (k * 0xC4CEB9FE1A85EC53) & M64
    k ^= k >> 33
    return k


def tag(key: int, seed: int) -> int:
    """Overflow tag: the low three bits of the hash."""
    return fmix64((key ^ seed) & M64) & 7


def windows(key: int, seed: int, p: int):
    h = fmix64((key ^ seed) & M64)
    w = ((h >> 32) * p) >> 32
    step = 1 + (((h & 0xFFFFFFFF) * (p - 1)) >> 32)
    for _ in range(p):
        yield w
        w = (w + step) % p


class Table:
    """Brute-force table: keys per slot, 0 = empty, `tomb` = tombstone."""

    def __init__(self, p, W, slot_bytes, seed):
        self.p, self.W, self.sb, self.seed = p, W, slot_bytes, seed
        self.tomb = 0xFFFFFFFF if slot_bytes == 8 else M64
        self.keys = [0] * (p * W)
        self.where = {}
        self.ovf = np.zeros(p, dtype=np.uint8)  # eight overflow bits per window

    def insert(self, k):
        for j, w in enumerate(windows(k, self.seed, self.p)):
            for q in range(self.W):
                if self.keys[w * self.W + q] == 0:
                    self.keys[w * self.W + q] = k
                    self.where[k] = (w * self.W + q, j)
                    return True
            self.ovf[w] |= np.uint8(1 << tag(k, self.seed))  # walked past a window without an empty slot
        return False

    def dump(self) -> np.ndarray:
        if self.sb == 8:
            words = np.array(self.keys, dtype=np.uint64) | (np.uint64(7) << np.uint64(32))
            words[np.array(self.keys, dtype=np.uint64) == 0] = 0
            return words.view(np.uint8)
        out = np.zeros((len(self.keys), 2), dtype=np.uint64)
        out[:, 0] = np.array(self.keys, dtype=np.uint64)
        out[:, 1] = 99
        return out.view(np.uint8).reshape(-1)

    def check(self, seed=None, unique=True, bits=False):
        return oracle.check_slots(self.dump(), self.p, self.W, self.sb, self.seed if seed is None else seed, unique,
                                  self.ovf if bits else None)


def filled(slot_bytes, p=101, W=8, n=600, seed=0xC0FFEE):
    t = Table(p, W, slot_bytes, seed)
    rng = np.random.default_rng(slot_bytes * 1000 + W)
    top = 0xFFFFFFFE if slot_bytes == 8 else M64 - 1
    for k in rng.integers(1, top, n, dtype=np.uint64, endpoint=False):
        t.insert(int(k))
    return t


@pytest.mark.parametrize("sb", [8, 16])
def test_valid_dump_passes(sb):
    t = filled(sb)
    r = t.check()
    assert r == {"live": len(t.where), "dups": 0, "unreachable": 0}
    assert oracle.check_slots(np.zeros(101 * 8 * sb, np.uint8), 101, 8, sb, 1, True) == {
        "live": 0, "dups": 0, "unreachable": 0}


@pytest.mark.parametrize("sb", [8, 16])
def test_empty_slot_in_front_of_a_key_is_reported_but_a_tombstone_is_not(sb):
    t = filled(sb)
    # a key that sits in the second or a later window of its own sequence
    k, (slot, j) = next((k, v) for k, v in t.where.items() if v[1] >= 1)
    first = next(windows(k, t.seed, t.p))
    victim = first * t.W  # a slot of an earlier window of k's sequence (it was full)
    assert t.keys[victim] not in (0, t.tomb)
    t.keys[victim] = t.tomb
    r = t.check()
    assert r["unreachable"] == 0 and r["live"] == len(t.where) - 1
    t.keys[victim] = 0
    r = t.check()
    assert r["unreachable"] >= 1


@pytest.mark.parametrize("sb", [8, 16])
def test_duplicate_key_is_reported_only_when_keys_must_be_unique(sb):
    t = filled(sb, n=300)
    k = next(iter(t.where))
    for w in windows(k, t.seed, t.p):
        free = [w * t.W + q for q in range(t.W) if t.keys[w * t.W + q] == 0]
        if free:
            t.keys[free[-1]] = k
            break
    assert t.check() == {"live": len(t.where) + 1, "dups": 1, "unreachable": 0}
    assert t.check(unique=False)["dups"] == 0


def test_wrong_seed_breaks_reachability():
    t = filled(8, n=700)
    assert t.check()["unreachable"] == 0
    assert t.check(seed=t.seed + 1)["unreachable"] > 0


def test_geometry_is_validated():
    with pytest.raises(ValueError):
        oracle.check_slots(np.zeros(10, np.uint8), 11, 8, 8, 0, True)
    with pytest.raises(ValueError):
        oracle.check_slots(np.zeros(11 * 8 * 12, np.uint8), 11, 8, 12, 0, True)


def passed(t, k):
    """Windows key k's sequence passes before its own window."""
    slot, j = t.where[k]
    return [w for _, w in zip(range(j), windows(k, t.seed, t.p))]


@pytest.mark.parametrize("sb", [8, 16])
def test_overflow_bits(sb):
    """With overflow bits, a key is reachable only if every window its sequence passes
    before its own has the bit of the key's tag set; the brute-force insert sets exactly
    those bits.  Clearing one bit of a window makes unreachable exactly the keys of that
    tag that passed the window -- keys of the other seven tags are unaffected."""
    t = filled(sb, n=700)
    assert t.check(bits=True) == t.check() == {"live": len(t.where), "dups": 0, "unreachable": 0}
    k, (slot, j) = next((k, v) for k, v in t.where.items() if v[1] >= 1)
    first = next(windows(k, t.seed, t.p))
    g = tag(k, t.seed)
    for other in range(8):
        saved = t.ovf.copy()
        t.ovf[first] &= np.uint8(~(1 << other) & 0xFF)
        expect = sum(1 for q in t.where if tag(q, t.seed) == other and first in passed(t, q))
        assert expect >= (1 if other == g else 0)
        assert t.check()["unreachable"] == 0  # without the bits nothing changed
        assert t.check(bits=True)["unreachable"] == expect
        t.ovf = saved
    # as little-endian uint32 words (the library's dump format) the result is the same
    words = np.zeros((t.p + 3) // 4 * 4, np.uint8)
    words[:t.p] = t.ovf
    assert oracle.check_slots(t.dump(), t.p, t.W, t.sb, t.seed, True, words.view(np.uint32))["unreachable"] == 0
    assert oracle.check_slots(np.zeros(101 * 8 * sb, np.uint8), 101, 8, sb, 1, True, np.zeros(101, np.uint8))[
        "unreachable"] == 0
    # the bits are exactly those the stored keys' walks imply
    np.testing.assert_array_equal(oracle.overflow_bits_of(t.dump(), t.p, t.W, t.sb, t.seed), t.ovf)
    with pytest.raises(ValueError):  # too few bytes for the window count
        oracle.check_slots(t.dump(), t.p, t.W, t.sb, t.seed, True, np.zeros(25, np.uint32))


@pytest.mark.parametrize("sb", [8, 16])
def test_walk_stats_equal_brute_force(sb):
    """oracle.walk_stats: the mean windows of live keys equals the brute-force insert's own
    record (key stored in the j-th window of its walk: j + 1 windows), and the mean windows
    of absent keys equals a walk written here (to the first window with an empty slot, or
    with overflow bits to the first window that also has the key's tag bit clear)."""
    t = filled(sb, n=700)
    rng = np.random.default_rng(sb)
    top = 0xFFFFFFFE if sb == 8 else M64 - 1
    absent = [int(k) for k in rng.integers(1, top, 300, dtype=np.uint64) if int(k) not in t.where]
    dtype = np.uint32 if sb == 8 else np.uint64

    def miss_len(k, bits):
        g = tag(k, t.seed)
        for j, w in enumerate(windows(k, t.seed, t.p)):
            if 0 in t.keys[w * t.W:(w + 1) * t.W] or (bits and not (int(t.ovf[w]) >> g) & 1):
                return j + 1
        return None

    for bits in (False, True):
        r = oracle.walk_stats(t.dump(), t.p, t.W, t.sb, t.seed, np.array(absent, dtype=dtype),
                              t.ovf if bits else None)
        assert r["hits"] == len(t.where)
        assert r["hit"] == pytest.approx(np.mean([j + 1 for _, j in t.where.values()]), abs=1e-12)
        lens = [miss_len(k, bits) for k in absent]
        assert r["misses"] == len(absent)
        assert r["miss"] == pytest.approx(np.mean(lens), abs=1e-12)
    # at this load some walks are longer than one window, and the bits shorten misses
    assert oracle.walk_stats(t.dump(), t.p, t.W, t.sb, t.seed, np.array(absent, dtype=dtype))["miss"] > 1.0


def test_sequential_table_builder_equals_brute_force():
    """oracle.build_packed_table builds, key by key, the same slots and overflow bits as
    the brute-force insert written here in Python integers."""
    t = Table(101, 8, 8, 0xC0FFEE)
    rng = np.random.default_rng(5)
    keys = []
    for k in rng.integers(1, 0xFFFFFFFE, 760, dtype=np.uint64):
        if int(k) not in t.where and t.insert(int(k)):
            keys.append(int(k))
    dump, bits = oracle.build_packed_table(np.array(keys, dtype=np.uint32), np.full(len(keys), 7, np.uint32),
                                           101, 8, 0xC0FFEE)
    np.testing.assert_array_equal(dump, t.dump())
    np.testing.assert_array_equal(bits, t.ovf)


def test_walk_lengths_at_load_0p9():
    """Walk lengths of a table built key by key at load 0.9 (W = 8, 2^18 windows): present
    keys visit 1.22 windows; absent keys 2.87 without overflow bits, 2.07 with one bit per
    window (any key walked past) and 1.20 with eight bits selected by the key's tag."""
    import wc_inputs
    p, W = 262_139, 8  # prime
    n = int(0.9 * p * W)
    keys = wc_inputs.distinct_u32(0x51A, n + 200_000)
    absent, keys = keys[n:], keys[:n]
    dump, tags = oracle.build_packed_table(keys, None, p, W, 0x5EED)
    one_bit = np.where(tags != 0, 0xFF, 0).astype(np.uint8)
    plain = oracle.walk_stats(dump, p, W, 8, 0x5EED, absent)
    one = oracle.walk_stats(dump, p, W, 8, 0x5EED, absent, one_bit)
    tagged = oracle.walk_stats(dump, p, W, 8, 0x5EED, absent, tags)
    assert plain["hits"] == n and plain["misses"] == absent.size
    assert plain["hit"] == pytest.approx(1.22, abs=0.02)
    assert plain["miss"] == pytest.approx(2.87, abs=0.1)
    assert one["miss"] == pytest.approx(2.07, abs=0.1)
    assert tagged["miss"] == pytest.approx(1.20, abs=0.05)
    assert one["hit"] == tagged["hit"] == plain["hit"]
