"""CPU oracle of the bulk hash-table operations -- TEST INFRASTRUCTURE.

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may
import this package.  The GPU library never calls it and shares no code with it.

`oracle.cpp` implements the plain definitions over std::unordered_map (single-value,
Sec. IV-B3..IV-B5 of the paper) and std::unordered_multimap (multi-value, Sec. IV-B4);
this module compiles it with g++ and wraps it with ctypes over numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

FLAG_DUPLICATE_KEY = 1
FLAG_INVALID_KEY = 2

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (portable flags: x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        lib.oracle_create.restype = vp
        lib.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_destroy.argtypes = [vp]
        lib.oracle_insert.restype = u32
        lib.oracle_insert.argtypes = [vp, vp, vp, u64]
        lib.oracle_retrieve.restype = u32
        lib.oracle_retrieve.argtypes = [vp, vp, u64, vp, vp]
        lib.oracle_erase.restype = u32
        lib.oracle_erase.argtypes = [vp, vp, u64]
        lib.oracle_count_values.restype = u32
        lib.oracle_count_values.argtypes = [vp, vp, u64, vp]
        lib.oracle_retrieve_multi.restype = u32
        lib.oracle_retrieve_multi.argtypes = [vp, vp, u64, vp, vp]
        lib.oracle_size.restype = u64
        lib.oracle_size.argtypes = [vp]
        lib.oracle_num_keys.restype = u64
        lib.oracle_num_keys.argtypes = [vp]
        lib.oracle_reserve.argtypes = [vp, u64]
        lib.oracle_counts_create.restype = vp
        lib.oracle_counts_create.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.oracle_counts_destroy.argtypes = [vp]
        lib.oracle_counts_add.restype = u32
        lib.oracle_counts_add.argtypes = [vp, vp, vp, u64]
        lib.oracle_counts_get.restype = u32
        lib.oracle_counts_get.argtypes = [vp, vp, u64, vp, vp]
        lib.oracle_counts_erase.restype = u32
        lib.oracle_counts_erase.argtypes = [vp, vp, u64]
        lib.oracle_counts_size.restype = u64
        lib.oracle_counts_size.argtypes = [vp]
        lib.oracle_check_slots.restype = ctypes.c_int
        lib.oracle_check_slots.argtypes = [vp, u64, u32, u32, u32, u64, ctypes.c_int, vp, vp, vp, vp]
        lib.oracle_overflow_bits_of.restype = ctypes.c_int
        lib.oracle_walk_stats.restype = ctypes.c_int
        lib.oracle_build_packed_table.restype = ctypes.c_int64
        lib.oracle_build_packed_table.argtypes = [vp, vp, u64, u64, u32, u64, vp, vp]
        lib.oracle_walk_stats.argtypes = [vp, u64, u32, u32, u32, u64, vp, vp, u64, vp]
        lib.oracle_overflow_bits_of.argtypes = [vp, u64, u32, u32, u32, u64, vp]
        lib.oracle_sharded_create.restype = vp
        lib.oracle_sharded_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_sharded_destroy.argtypes = [vp]
        lib.oracle_sharded_insert.restype = u32
        lib.oracle_sharded_insert.argtypes = [vp, vp, vp, u64]
        lib.oracle_sharded_retrieve.restype = u32
        lib.oracle_sharded_retrieve.argtypes = [vp, vp, u64, vp, vp]
        lib.oracle_sharded_erase.restype = u32
        lib.oracle_sharded_erase.argtypes = [vp, vp, u64]
        lib.oracle_sharded_size.restype = u64
        lib.oracle_sharded_size.argtypes = [vp]
        lib.oracle_sharded_reserve.argtypes = [vp, u64]
        lib.oracle_bloom_create.restype = vp
        lib.oracle_bloom_create.argtypes = [ctypes.c_int, u64, ctypes.c_int, u64]
        lib.oracle_bloom_destroy.argtypes = [vp]
        lib.oracle_bloom_insert.restype = u32
        lib.oracle_bloom_insert.argtypes = [vp, vp, u64]
        lib.oracle_bloom_contains.restype = u32
        lib.oracle_bloom_contains.argtypes = [vp, vp, u64, vp]
        _lib = lib
    return _lib


def _dt(nbytes: int):
    return np.uint32 if nbytes == 4 else np.uint64


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Base:
    kind = -1

    def __init__(self, key_bytes: int = 4, value_bytes: int = 4):
        self._lib = _load()
        self.kb, self.vb = key_bytes, value_bytes
        self.kdt, self.vdt = _dt(key_bytes), _dt(value_bytes)
        self._h = self._lib.oracle_create(self.kind, key_bytes, value_bytes)
        if not self._h:
            raise ValueError("unsupported key/value widths")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _keys(self, keys):
        return np.ascontiguousarray(keys, dtype=self.kdt)

    def insert(self, keys, values) -> int:
        k = self._keys(keys)
        v = np.ascontiguousarray(values, dtype=self.vdt)
        assert k.size == v.size
        return int(self._lib.oracle_insert(self._h, _ptr(k), _ptr(v), k.size))

    def erase(self, keys) -> int:
        k = self._keys(keys)
        return int(self._lib.oracle_erase(self._h, _ptr(k), k.size))

    def size(self) -> int:
        return int(self._lib.oracle_size(self._h))

    def num_keys(self) -> int:
        return int(self._lib.oracle_num_keys(self._h))

    def reserve(self, n: int):
        self._lib.oracle_reserve(self._h, int(n))


class SingleValue(_Base):
    """std::unordered_map<K, V> with the single-value semantics of Sec. IV-B."""
    kind = 0

    def retrieve(self, keys):
        k = self._keys(keys)
        out = np.empty(k.size, dtype=self.vdt)
        found = np.empty(k.size, dtype=np.uint8)
        flags = int(self._lib.oracle_retrieve(self._h, _ptr(k), k.size, _ptr(out), _ptr(found)))
        return out, found, flags


class ShardedSingleValue:
    """The single-value definition on `threads` host cores: one plain std::unordered_map
    per shard, key k in shard std::hash(k) mod threads, each batch applied by one thread
    per shard walking it in input order.  Every result equals SingleValue's."""

    def __init__(self, key_bytes: int = 4, value_bytes: int = 4, threads: int | None = None):
        self._lib = _load()
        self.threads = int(threads or os.cpu_count() or 1)
        self.kdt, self.vdt = _dt(key_bytes), _dt(value_bytes)
        self._h = self._lib.oracle_sharded_create(key_bytes, value_bytes, self.threads)
        if not self._h:
            raise ValueError("unsupported key/value widths")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_sharded_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def insert(self, keys, values) -> int:
        k = np.ascontiguousarray(keys, dtype=self.kdt)
        v = np.ascontiguousarray(values, dtype=self.vdt)
        assert k.size == v.size
        return int(self._lib.oracle_sharded_insert(self._h, _ptr(k), _ptr(v), k.size))

    def retrieve(self, keys):
        k = np.ascontiguousarray(keys, dtype=self.kdt)
        out = np.empty(k.size, dtype=self.vdt)
        found = np.empty(k.size, dtype=np.uint8)
        flags = int(self._lib.oracle_sharded_retrieve(self._h, _ptr(k), k.size, _ptr(out), _ptr(found)))
        return out, found, flags

    def erase(self, keys) -> int:
        k = np.ascontiguousarray(keys, dtype=self.kdt)
        return int(self._lib.oracle_sharded_erase(self._h, _ptr(k), k.size))

    def size(self) -> int:
        return int(self._lib.oracle_sharded_size(self._h))

    def reserve(self, n: int):
        self._lib.oracle_sharded_reserve(self._h, int(n))


class MultiValue(_Base):
    """std::unordered_multimap<K, V> with the multi-value semantics of Sec. IV-B4."""
    kind = 1

    def count_values(self, keys):
        k = self._keys(keys)
        offs = np.empty(k.size + 1, dtype=np.uint64)
        flags = int(self._lib.oracle_count_values(self._h, _ptr(k), k.size, _ptr(offs)))
        return offs, flags

    def retrieve_multi(self, keys, offsets):
        k = self._keys(keys)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        assert offs.size == k.size + 1
        out = np.empty(int(offs[-1]), dtype=self.vdt)
        flags = int(self._lib.oracle_retrieve_multi(self._h, _ptr(k), k.size, _ptr(offs), _ptr(out)))
        return out, flags


class Counting:
    """Occurrence counts per key (Sec. IV, CountingHashTable): insert adds each key's
    weight (1 when no weights) to its count, modulo 2^(8 * key_bytes)."""

    is_set = False

    def __init__(self, key_bytes: int = 4):
        self._lib = _load()
        self.kb = key_bytes
        self.kdt = _dt(key_bytes)
        self._h = self._lib.oracle_counts_create(key_bytes, int(self.is_set))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_counts_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _keys(self, keys):
        return np.ascontiguousarray(np.asarray(keys).astype(self.kdt, copy=False))

    def insert(self, keys, weights=None) -> int:
        k = self._keys(keys)
        w = None if weights is None else np.ascontiguousarray(np.asarray(weights).astype(self.kdt, copy=False))
        return int(self._lib.oracle_counts_add(self._h, _ptr(k), None if w is None else _ptr(w), k.size))

    def retrieve(self, keys):
        k = self._keys(keys)
        out = np.empty(k.size, dtype=self.kdt)
        found = np.empty(k.size, dtype=np.uint8)
        f = self._lib.oracle_counts_get(self._h, _ptr(k), k.size, _ptr(out), _ptr(found))
        return out, found, int(f)

    def erase(self, keys) -> int:
        k = self._keys(keys)
        return int(self._lib.oracle_counts_erase(self._h, _ptr(k), k.size))

    def size(self) -> int:
        return int(self._lib.oracle_counts_size(self._h))


class HashSet(Counting):
    """A set of keys (Sec. IV, HashSet): insert raises DUPLICATE_KEY for a key already in
    the set; contains(keys) -> found mask."""

    is_set = True

    def contains(self, keys):
        k = self._keys(keys)
        found = np.empty(k.size, dtype=np.uint8)
        f = self._lib.oracle_counts_get(self._h, _ptr(k), k.size, None, _ptr(found))
        return found, int(f)


class BloomFilter:
    """Blocked Bloom filter by the library's documented definition (oracle.cpp): `blocks`
    blocks of 256 bits, k bits per key."""

    def __init__(self, key_bytes: int, blocks: int, k: int, seed: int):
        self._lib = _load()
        self.kdt = _dt(key_bytes)
        self._h = self._lib.oracle_bloom_create(key_bytes, blocks, k, seed & (2 ** 64 - 1))
        if not self._h:
            raise ValueError("bad Bloom filter parameters")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_bloom_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def insert(self, keys) -> int:
        k = np.ascontiguousarray(np.asarray(keys).astype(self.kdt, copy=False))
        return int(self._lib.oracle_bloom_insert(self._h, _ptr(k), k.size))

    def contains(self, keys):
        k = np.ascontiguousarray(np.asarray(keys).astype(self.kdt, copy=False))
        found = np.empty(k.size, dtype=np.uint8)
        f = self._lib.oracle_bloom_contains(self._h, _ptr(k), k.size, _ptr(found))
        return found, int(f)


def sorted_segments(values: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Sort every CSR segment in place-independent form (values compared as multisets)."""
    out = np.array(values, copy=True)
    offs = np.asarray(offsets, dtype=np.int64)
    n = offs.size - 1
    if n <= 0 or out.size == 0:
        return out
    seg = np.repeat(np.arange(n, dtype=np.int64), np.diff(offs))
    order = np.lexsort((out, seg))
    return out[order]


def check_slots(dump: np.ndarray, p: int, W: int, slot_bytes: int, seed: int, unique_keys: bool,
                overflow_bits: np.ndarray | None = None, key_bytes: int | None = None) -> dict:
    """Slot-dump invariant check of a table's slot array (host bytes, p * W slots):
    live slots, duplicate keys (when keys must be unique) and live keys that sit behind
    a window holding an empty slot on their own probing sequence -- or, when the table's
    overflow bits are given (one byte per window, as bytes or as the little-endian uint32
    words the library dumps), behind a window whose bit for the key's tag is clear (see
    oracle.cpp).  key_bytes defaults to 4 for 4- and 8-byte slots (packed 4+4-byte
    pairs) and 8 for 16-byte slots."""
    buf = np.ascontiguousarray(dump).view(np.uint8)
    if buf.size < p * W * slot_bytes:
        raise ValueError("dump holds %d bytes, need %d" % (buf.size, p * W * slot_bytes))
    out = np.zeros(3, dtype=np.uint64)
    ovf = None
    if overflow_bits is not None:
        ovf = np.ascontiguousarray(overflow_bits).view(np.uint8)
        if ovf.size < p:
            raise ValueError("overflow bits hold %d bytes, need %d" % (ovf.size, p))
    if key_bytes is None:
        key_bytes = 8 if slot_bytes == 16 else 4
    rc = _load().oracle_check_slots(_ptr(buf), p, W, slot_bytes, key_bytes, seed & (2 ** 64 - 1), int(unique_keys),
                                    None if ovf is None else _ptr(ovf),
                                    _ptr(out[0:]), ctypes.c_void_p(out.ctypes.data + 8),
                                    ctypes.c_void_p(out.ctypes.data + 16))
    if rc != 0:
        raise ValueError("bad table geometry")
    return {"live": int(out[0]), "dups": int(out[1]), "unreachable": int(out[2])}


def overflow_bits_of(dump: np.ndarray, p: int, W: int, slot_bytes: int, seed: int,
                     key_bytes: int | None = None) -> np.ndarray:
    """The overflow bits (one byte per window) that a table filled by inserts alone holds:
    for every live key, the bit of its tag in each window its sequence passes before the
    key's own window (see oracle.cpp)."""
    buf = np.ascontiguousarray(dump).view(np.uint8)
    if buf.size < p * W * slot_bytes:
        raise ValueError("dump holds %d bytes, need %d" % (buf.size, p * W * slot_bytes))
    if key_bytes is None:
        key_bytes = 8 if slot_bytes == 16 else 4
    out = np.zeros(p, dtype=np.uint8)
    if _load().oracle_overflow_bits_of(_ptr(buf), p, W, slot_bytes, key_bytes, seed & (2 ** 64 - 1), _ptr(out)) != 0:
        raise ValueError("bad table geometry")
    return out


def walk_stats(dump: np.ndarray, p: int, W: int, slot_bytes: int, seed: int, absent: np.ndarray | None = None,
               overflow_bits: np.ndarray | None = None, key_bytes: int | None = None) -> dict:
    """Mean windows a lookup visits on a slot dump: `hit` over the live keys (up to the
    window holding the key), `miss` over the `absent` keys (up to the first window with an
    empty slot, or with overflow bits given, also a window whose bit for the key's tag is
    clear); see oracle.cpp."""
    buf = np.ascontiguousarray(dump).view(np.uint8)
    if buf.size < p * W * slot_bytes:
        raise ValueError("dump holds %d bytes, need %d" % (buf.size, p * W * slot_bytes))
    if key_bytes is None:
        key_bytes = 8 if slot_bytes == 16 else 4
    ab = np.zeros(0, dtype=np.uint32 if key_bytes == 4 else np.uint64) if absent is None else \
        np.ascontiguousarray(absent, dtype=np.uint32 if key_bytes == 4 else np.uint64)
    ovf = None
    if overflow_bits is not None:
        ovf = np.ascontiguousarray(overflow_bits).view(np.uint8)
        if ovf.size < p:
            raise ValueError("overflow bits hold %d bytes, need %d" % (ovf.size, p))
    out = np.zeros(4, dtype=np.uint64)
    rc = _load().oracle_walk_stats(_ptr(buf), p, W, slot_bytes, key_bytes, seed & (2 ** 64 - 1),
                                   None if ovf is None else _ptr(ovf), _ptr(ab) if ab.size else None, ab.size,
                                   _ptr(out))
    if rc != 0:
        raise ValueError("bad table geometry")
    h, nh, m, nm = (int(x) for x in out)
    return {"hit": h / nh if nh else 0.0, "hits": nh, "miss": m / nm if nm else 0.0, "misses": nm}


def build_packed_table(keys: np.ndarray, values: np.ndarray | None, p: int, W: int, seed: int):
    """(slot dump as bytes, overflow bits as p bytes) of a packed 4+4-byte table built by
    inserting the distinct uint32 `keys` one at a time (see oracle.cpp)."""
    k = np.ascontiguousarray(keys, dtype=np.uint32)
    v = None if values is None else np.ascontiguousarray(values, dtype=np.uint32)
    slots = np.zeros(p * W, dtype=np.uint64)
    bits = np.zeros(p, dtype=np.uint8)
    failed = _load().oracle_build_packed_table(_ptr(k), None if v is None else _ptr(v), k.size, p, W,
                                               seed & (2 ** 64 - 1), _ptr(slots), _ptr(bits))
    if failed < 0:
        raise ValueError("bad table geometry")
    if failed:
        raise ValueError("%d keys found no slot" % failed)
    return slots.view(np.uint8), bits
