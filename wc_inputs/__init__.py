"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the bench.

This module holds random-number streams and workload recipes only.  It contains none of
the hash-table method's arithmetic (no table hashing, no probing), so the oracle and the
CUDA path can both consume its arrays without sharing any method code.

Published generators used (each restated here from its definition):

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
  OOPSLA 2014): state_i = seed + i * 0x9E3779B97F4A7C15, output = mix(state_i).  The mix
  is a bijection of 64-bit words, so the first 2^64 outputs of one stream are pairwise
  distinct -- this is how distinct uint64 keys are drawn without a sort.
* lowbias32 (C. Wellons, "hash-prospector", 2018): a bijective 32-bit mixer applied to a
  Weyl sequence (seed + i * odd) mod 2^32, which is likewise pairwise distinct for
  i < 2^32 -- distinct uint32 keys.
* Zipf(s) by inverse-transform sampling: an exact cumulative table over the head ranks
  with a guide table (Chen and Asau, 1974) and the integral approximation of the tail
  sum (Euler-Maclaurin midpoint rule) inverted in closed form.

Sentinels: key 0 is the empty marker and the all-ones key is the tombstone marker of
the tables (Sec. IV-B1 and IV-B5 of the paper), so every key generator drops them.
"""
from __future__ import annotations

import numpy as np

U64 = np.uint64
GOLDEN64 = U64(0x9E3779B97F4A7C15)
GOLDEN32 = np.uint32(0x9E3779B9)
EMPTY_KEY = 0
TOMBSTONE_KEY32 = 0xFFFFFFFF
TOMBSTONE_KEY64 = 0xFFFFFFFFFFFFFFFF

_CHUNK = 1 << 24  # elements per vector pass; bounds the temporaries

# Optional C fills of the same streams (_gen.c); numpy below is the definition they are
# tested against and the fallback when the helper is not built.
import ctypes as _ct
import os as _os
import subprocess as _sp

_HERE = _os.path.dirname(_os.path.abspath(__file__))
_GEN_SRC = _os.path.join(_HERE, "_gen.c")
_GEN_LIB = _os.path.join(_HERE, "libwcgen.so")
_gen = None


def build_helper() -> str:
    """Compile _gen.c into libwcgen.so next to it (portable flags)."""
    if not _os.path.exists(_GEN_LIB) or _os.path.getmtime(_GEN_LIB) < _os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + ".tmp%d" % _os.getpid()
        _sp.check_call(["gcc", "-O2", "-shared", "-fPIC", _GEN_SRC, "-o", tmp])
        _os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _helper():
    global _gen
    if _gen is None and _os.path.exists(_GEN_LIB):
        lib = _ct.CDLL(_GEN_LIB)
        u64, vp, u32 = _ct.c_uint64, _ct.c_void_p, _ct.c_uint32
        lib.wcgen_splitmix64.argtypes = [u64, u64, u64, vp]
        lib.wcgen_splitmix64_hi32.argtypes = [u64, u64, u64, vp]
        lib.wcgen_lowbias32_weyl.argtypes = [u32, u64, u64, vp]
        _gen = lib
    return _gen


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 stream with the given seed."""
    g = _helper()
    if g is not None and count > 4096:
        out = np.empty(count, dtype=np.uint64)
        g.wcgen_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, start, count, out.ctypes.data)
        return out
    return splitmix64_np(seed, start, count)


def splitmix64_np(seed: int, start: int, count: int) -> np.ndarray:
    """numpy definition of splitmix64 (the reference the C fill is checked against)."""
    out = np.empty(count, dtype=np.uint64)
    seed = U64(seed & 0xFFFFFFFFFFFFFFFF)
    c1 = U64(0xBF58476D1CE4E5B9)
    c2 = U64(0x94D049BB133111EB)
    with np.errstate(over="ignore"):
        for lo in range(0, count, _CHUNK):
            hi = min(count, lo + _CHUNK)
            z = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            z *= GOLDEN64
            z += seed
            z ^= z >> U64(30)
            z *= c1
            z ^= z >> U64(27)
            z *= c2
            z ^= z >> U64(31)
            out[lo:hi] = z
    return out


def lowbias32(x: np.ndarray) -> np.ndarray:
    """Wellons' lowbias32 mixer; a bijection on uint32 (xorshifts and odd multiplies)."""
    x = x.astype(np.uint32, copy=True)
    with np.errstate(over="ignore"):
        x ^= x >> np.uint32(16)
        x *= np.uint32(0x7FEB352D)
        x ^= x >> np.uint32(15)
        x *= np.uint32(0x846CA68B)
        x ^= x >> np.uint32(16)
    return x


def distinct_u32(seed: int, count: int) -> np.ndarray:
    """`count` pairwise-distinct uint32 keys, sentinels (0, 0xFFFFFFFF) excluded."""
    if count + 2 > (1 << 32):
        raise ValueError("at most 2^32 - 2 distinct uint32 keys exist")
    base = np.uint32((seed ^ (seed >> 32)) & 0xFFFFFFFF)
    g = _helper()
    if g is not None and count > 4096:
        out = np.empty(count + 2, dtype=np.uint32)
        g.wcgen_lowbias32_weyl(int(base), 0, count + 2, out.ctypes.data)
        keep = (out != 0) & (out != np.uint32(TOMBSTONE_KEY32))
        return out[keep][:count].copy()
    out = np.empty(count + 2, dtype=np.uint32)
    with np.errstate(over="ignore"):
        for lo in range(0, count + 2, _CHUNK):
            hi = min(count + 2, lo + _CHUNK)
            w = np.arange(lo, hi, dtype=np.uint64).astype(np.uint32)
            w *= GOLDEN32
            w += base
            out[lo:hi] = lowbias32(w)
    keep = (out != 0) & (out != np.uint32(TOMBSTONE_KEY32))
    return out[keep][:count].copy()


def distinct_u64(seed: int, count: int) -> np.ndarray:
    """`count` pairwise-distinct uint64 keys, sentinels (0, all ones) excluded."""
    out = splitmix64(seed, 0, count + 2)
    keep = (out != 0) & (out != U64(TOMBSTONE_KEY64))
    return out[keep][:count].copy()


def uniform_u32(seed: int, count: int) -> np.ndarray:
    """Uniform uint32 values (high halves of a SplitMix64 stream)."""
    g = _helper()
    if g is not None and count > 4096:
        out = np.empty(count, dtype=np.uint32)
        g.wcgen_splitmix64_hi32(seed & 0xFFFFFFFFFFFFFFFF, 0, count, out.ctypes.data)
        return out
    return (splitmix64(seed, 0, count) >> U64(32)).astype(np.uint32)


def uniform_u64(seed: int, count: int) -> np.ndarray:
    return splitmix64(seed, 0, count)


def uniform_unit(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, 0, count) >> U64(11)).astype(np.float64) * (2.0 ** -53)


def shuffle_index(seed: int, n: int) -> np.ndarray:
    """A seeded permutation of range(n), built as a bijection of the next power-of-two
    domain (rounds of odd multiply-add and xorshift modulo 2^b) with cycle walking back
    into [0, n).  Vectorised; used to put queries in random order."""
    if n <= 1:
        return np.zeros(n, dtype=np.int64)
    b = max(2, int(n - 1).bit_length())
    mask = U64((1 << b) - 1)
    params = splitmix64(seed, 0, 6)
    mults = [(int(params[i]) | 1) & ((1 << b) - 1) for i in range(3)]
    adds = [int(params[3 + i]) & ((1 << b) - 1) for i in range(3)]
    shift = U64(b // 2 + 1)

    def f(x: np.ndarray) -> np.ndarray:
        with np.errstate(over="ignore"):
            for r in range(3):
                x = (x * U64(mults[r]) + U64(adds[r])) & mask
                x ^= x >> shift
        return x

    out = f(np.arange(n, dtype=np.uint64))
    bad = np.nonzero(out >= U64(n))[0]
    while bad.size:
        out[bad] = f(out[bad])
        bad = bad[out[bad] >= U64(n)]
    return out.astype(np.int64)


class ZipfSampler:
    """Zipf(s) over ranks 1..N: P(r) proportional to r^-s, s > 1.

    Exact cumulative weights over the head ranks 1..R0 (R0 = min(N, 2^20)); the tail
    R0+1..N uses the midpoint integral of x^-s, inverted in closed form.  `sample`
    returns 0-based ranks (rank 1 -> 0)."""

    def __init__(self, n_ranks: int, s: float, head: int = 1 << 20, guide_bits: int = 22):
        if s <= 1.0:
            raise ValueError("s must exceed 1")
        self.N = int(n_ranks)
        self.s = float(s)
        self.R0 = min(self.N, head)
        r = np.arange(1, self.R0 + 1, dtype=np.float64)
        self.cum = np.cumsum(r ** -self.s)
        self.head_mass = float(self.cum[-1])
        if self.N > self.R0:
            a = (self.R0 + 0.5) ** (1.0 - self.s)
            b = (self.N + 0.5) ** (1.0 - self.s)
            self.tail_mass = (a - b) / (self.s - 1.0)
        else:
            self.tail_mass = 0.0
        self.total = self.head_mass + self.tail_mass
        m = 1 << guide_bits
        self.M = m
        edges = np.arange(m + 1, dtype=np.float64) * (self.head_mass / m)
        self.guide = np.searchsorted(self.cum, edges, side="right").astype(np.int64)

    def prob_rank1(self) -> float:
        return 1.0 / self.total

    def sample(self, seed: int, count: int) -> np.ndarray:
        out = np.empty(count, dtype=np.int64)
        for lo in range(0, count, _CHUNK):
            hi = min(count, lo + _CHUNK)
            u = (splitmix64(seed, lo, hi - lo) >> U64(11)).astype(np.float64) * (2.0 ** -53)
            out[lo:hi] = self._invert(u * self.total)
        return out

    def _invert(self, U: np.ndarray) -> np.ndarray:
        res = np.empty(U.size, dtype=np.int64)
        head = U < self.head_mass
        hu = U[head]
        b = np.minimum((hu * (self.M / self.head_mass)).astype(np.int64), self.M - 1)
        r = self.guide[b]
        r = np.minimum(r, self.R0 - 1)
        # r is a lower bound of the answer (first index with cum > U); walk forward.
        idx = np.nonzero(self.cum[r] <= hu)[0]
        while idx.size:
            r[idx] += 1
            np.minimum(r, self.R0 - 1, out=r)
            still = self.cum[r[idx]] <= hu[idx]
            still &= r[idx] < self.R0 - 1
            idx = idx[still]
        res[head] = r
        if self.tail_mass > 0.0:
            tail = ~head
            v = U[tail] - self.head_mass
            a = (self.R0 + 0.5) ** (1.0 - self.s)
            x = np.maximum(a - v * (self.s - 1.0), 1e-300) ** (1.0 / (1.0 - self.s))
            rt = np.floor(x - 0.5).astype(np.int64)  # 1-based rank
            res[tail] = np.clip(rt, self.R0 + 1, self.N) - 1
        return res


# ----------------------------------------------------------------------------------
# Workload recipes (shapes of the paper's experiments, Sec. V-A and V-C).
# ----------------------------------------------------------------------------------

def sv_insert_retrieve_u32(seed: int, n: int, n_present_q: int, n_absent_q: int):
    """Unique uint32 keys with uniform uint32 values, plus a shuffled query batch of
    `n_present_q` inserted keys and `n_absent_q` keys that were never inserted.

    Returns dict(keys, values, queries, q_src) where q_src[i] is the index into `keys`
    of query i, or -1 for an absent query."""
    allk = distinct_u32(seed, n + n_absent_q)
    keys = allk[:n]
    absent = allk[n:]
    values = uniform_u32(seed ^ 0x5A5A5A5A5A5A5A5A, n)
    if n_present_q > n:
        raise ValueError("more present queries than keys")
    src = np.concatenate([np.arange(n_present_q, dtype=np.int64),
                          -np.ones(n_absent_q, dtype=np.int64)])
    qk = np.concatenate([keys[:n_present_q], absent])
    perm = shuffle_index(seed ^ 0x0F0F0F0F0F0F0F0F, qk.size)
    return dict(keys=keys, values=values, queries=qk[perm], q_src=src[perm])


def sv_u64_zipf(seed: int, n: int, n_queries: int, s: float = 1.1):
    """Unique uint64 keys with uniform uint64 values; queries drawn Zipf(s) over the
    inserted keys (rank r maps to keys[r-1]; the key order is already random)."""
    keys = distinct_u64(seed, n)
    values = uniform_u64(seed ^ 0x5A5A5A5A5A5A5A5A, n)
    ranks = ZipfSampler(n, s).sample(seed ^ 0x3C3C3C3C3C3C3C3C, n_queries)
    return dict(keys=keys, values=values, queries=keys[ranks], q_src=ranks)


def mv_zipf_u64(seed: int, universe: int, n_inserts: int, n_absent: int, s: float = 1.1):
    """Multi-value workload: `n_inserts` pairs whose keys are drawn Zipf(s) over a
    universe of distinct uint64 keys, value = insert index (uint32); queries are the whole
    universe plus `n_absent` keys never inserted, shuffled."""
    allk = distinct_u64(seed, universe + n_absent)
    uni = allk[:universe]
    absent = allk[universe:]
    ranks = ZipfSampler(universe, s).sample(seed ^ 0x3C3C3C3C3C3C3C3C, n_inserts)
    keys = uni[ranks]
    values = np.arange(n_inserts, dtype=np.uint64).astype(np.uint32)
    qk = np.concatenate([uni, absent])
    src = np.concatenate([np.arange(universe, dtype=np.int64), -np.ones(n_absent, dtype=np.int64)])
    perm = shuffle_index(seed ^ 0x0F0F0F0F0F0F0F0F, qk.size)
    return dict(keys=keys, values=values, queries=qk[perm], ranks=ranks, q_src=src[perm])


def mv_uniform_r(seed: int, n: int, r: int):
    """The paper's multi-value benchmark shape (Sec. V-C): n keys drawn uniformly at
    random from 1..n/r (value = insert index), queries are all of 1..n, so exactly n
    values come back in total whatever the draw."""
    m = max(1, n // r)
    keys = (splitmix64(seed, 0, n) % U64(m)) + U64(1)
    values = np.arange(n, dtype=np.uint64).astype(np.uint32)
    queries = np.arange(1, n + 1, dtype=np.uint64)
    return dict(keys=keys, values=values, queries=queries)


def serving_trace(seed: int, n_tables: int = 64, log2_cap: tuple[float, float] = (16, 26),
                  n_requests: int = 256, log2_batch: tuple[float, float] = (np.log2(1000), 24),
                  mix: tuple[float, float, float] = (0.60, 0.35, 0.05), max_load: float = 0.9,
                  prefill: tuple[float, float] = (0.0, 0.6), scale_keys: float = 1.0):
    """The batched + served workload: tables with capacity 2^U(log2_cap), pre-filled to a
    load ~U(prefill); requests with batch size 2^U(log2_batch) (times `scale_keys`), op
    mix insert / retrieve / erase, inserts of fresh unique keys clamped to the room left
    below `max_load`, retrieves half present / half absent, erases of present keys.
    Arrival times are assigned by the caller (poisson_arrivals).

    Returns dict(caps, prefill_keys[t], prefill_vals[t], requests=[dict(op, table, keys,
    values)]) with ops 0 = insert, 1 = retrieve, 2 = erase."""
    u = uniform_unit(seed, 4 * n_tables + 8 * n_requests)
    caps = np.floor(2.0 ** (log2_cap[0] + (log2_cap[1] - log2_cap[0]) * u[:n_tables])).astype(np.int64)
    pre = prefill[0] + (prefill[1] - prefill[0]) * u[n_tables:2 * n_tables]
    universes, pf_keys, pf_vals, state, cursor, nlive = [], [], [], [], [], []
    for t in range(n_tables):
        m = int(caps[t])
        # keys [0, m) may be inserted; keys [m, 2m) never are (the absent queries)
        uk = distinct_u32(seed * 1000003 + t, 2 * m)
        universes.append(uk)
        k = int(pre[t] * m)
        pf_keys.append(uk[:k].copy())
        pf_vals.append(uniform_u32(seed * 7 + t, k))
        st = np.zeros(m, dtype=np.int8)  # 0 never inserted, 1 live, 2 erased
        st[:k] = 1
        state.append(st)
        cursor.append(k)
        nlive.append(k)
    reqs = []
    base = 2 * n_tables
    for i in range(n_requests):
        t = int(u[base + 8 * i] * n_tables) % n_tables
        r = u[base + 8 * i + 1]
        op = 0 if r < mix[0] else (1 if r < mix[0] + mix[1] else 2)
        nb = max(1, int(2.0 ** (log2_batch[0] + (log2_batch[1] - log2_batch[0]) * u[base + 8 * i + 2]) * scale_keys))
        m = int(caps[t])
        uk = universes[t]
        rs = seed * 31 + i
        if op == 0:
            room = min(int(max_load * m) - nlive[t], m - cursor[t])
            if room > 0:
                nb = min(nb, room)
                idx = np.arange(cursor[t], cursor[t] + nb)
                cursor[t] += nb
                state[t][idx] = 1
                nlive[t] += nb
                reqs.append(dict(op=0, table=t, keys=uk[idx], values=uniform_u32(rs, nb)))
                continue
            op = 1  # table full: serve a retrieve instead
        if op == 2 and nlive[t] > 0:
            # a window of insertion positions from a random start; its live keys go
            off = int(splitmix64(rs, 0, 1)[0] % np.uint64(cursor[t]))
            cand = np.arange(off, min(cursor[t], off + 2 * nb))
            gone = cand[state[t][cand] == 1][:nb]
            if gone.size:
                state[t][gone] = 2
                nlive[t] -= gone.size
                reqs.append(dict(op=2, table=t, keys=uk[gone]))
                continue
            op = 1
        # retrieve: each query independently present or absent with probability 1/2;
        # present keys are a window of insertion positions from a random start (the
        # universe is in random order, so this is a random subset) -- erased ones among
        # them are absent queries too; absent keys come from the never-inserted half
        coin = uniform_unit(rs, nb) < 0.5
        r2 = splitmix64(rs + 1, 0, 2)
        cur = max(cursor[t], 1)
        ip = (int(r2[0] % np.uint64(cur)) + np.arange(nb, dtype=np.int64)) % cur
        ia = m + (int(r2[1] % np.uint64(m)) + np.arange(nb, dtype=np.int64)) % m
        use_p = coin & (state[t][ip] == 1) if cursor[t] else np.zeros(nb, dtype=bool)
        q = np.where(use_p, uk[ip], uk[ia])
        reqs.append(dict(op=1, table=t, keys=q))
    return dict(caps=caps, prefill_keys=pf_keys, prefill_vals=pf_vals, requests=reqs)


def poisson_arrivals(seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (ns) of a Poisson process: exponential gaps by inverse transform."""
    u = uniform_unit(seed, n)
    gaps = -np.log1p(-u) / rate_per_s
    return (np.cumsum(gaps) * 1e9).astype(np.uint64)
