// Open-addressing multi-value table (the paper's MultiValueHashTable, Sec. IV and
// Sec. V-C): every (key, value) pair occupies its own slot of the same slot layouts as
// the single-value table, along the key's probing sequence.
//
//   insert         claims an empty-or-tombstoned slot of the first window of the sequence
//                  that has one, with one CAS of the packed pair (Sec. IV-B2 steps 1-7,
//                  without the duplicate check: the same key may occur many times);
//   count_values   walks the sequence up to the first window holding an empty slot and
//                  counts the matches of each window with a group vote (the parallel
//                  match counting of Sec. V-C), then an exclusive scan gives the offsets;
//   retrieve_multi walks the same windows and writes each match to its query's segment
//                  (lanes of a group write their matches at consecutive positions);
//   erase          tombstones every copy of the key.
// Every window before a copy's window was full when the copy was claimed, and slots never
// go back to empty except by a clear, so every copy sits at or before the first window of
// its sequence holding an empty slot: the walks see every copy.
#pragma once

#include "wc_device.cuh"
#include "wc_internal.h"
#include "wc_sv_kernels.cuh"

namespace wc {

// Sum of a value over the G lanes of my group (every lane of the warp calls).
template <int G>
__device__ __forceinline__ uint32_t group_sum(uint32_t x) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Exclusive prefix of a value over the lanes of my group, in lane order.
template <int G>
__device__ __forceinline__ uint32_t group_exclusive(uint32_t x, int r) {
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (r >= o) inc += y;
  }
  return inc - x;
}

// Position of the (n+1)-th set bit of m (n < popc(m)).
__device__ __forceinline__ int nth_set(uint32_t m, uint32_t n) {
  for (uint32_t i = 0; i < n; ++i) m &= m - 1;
  return __ffs(m) - 1;
}

// Inputs per chunk of the strided walks (two input prefetches of a warp).
constexpr uint32_t kWalkChunk = 128;

// ---- insert: append the pair -----------------------------------------------------------
// counter == nullptr: each warp takes its static range; else warps pull `chunk` inputs at a
// time in order (a batch split by table region is then inserted region by region).
//
// The walks below scan whole windows and stop after the first window holding an empty
// slot, so a pair may take ANY free slot of the first window of its sequence that has one
// (not only the lowest): every window before it is then full, which is all the walks need.
// Each pair picks among the window's free slots by a hash of its input position, so the
// copies of a hot key, which all probe the same windows, claim different slots at once
// instead of all racing for the lowest one.
template <class L, int G, int S>
__global__ void __launch_bounds__(256) k_oa_insert(TableDesc t, const typename L::Key* __restrict__ keys,
                                                   const typename L::Val* __restrict__ vals, uint64_t n,
                                                   uint64_t per_warp, unsigned long long* counter, uint32_t chunk) {
  using Slot = typename L::Slot;
  using Key = typename L::Key;
  using Val = typename L::Val;
  RangeSrc src(n, per_warp, counter, chunk);
  if (counter == nullptr && src.next >= src.end) return;
  const SvLane<L, G, S> ln;
  constexpr int W = G * S;
  Slot* slots = static_cast<Slot*>(t.slots);
  bool act = false;
  Key k = 0;
  Val v = 0;
  uint32_t w = 0, step = 0, j = 0, flags = 0, salt = 0;
  long long added = 0;
  Feed<Key> fk;
  Feed<Val> fv;
  while (true) {
    const bool more = src.ensure();
    if (more && src.fresh) {
      fk.load(keys, src.next, src.end);
      fv.load(vals, src.next, src.end);
      src.fresh = false;
    }
    uint64_t np = 0;
    const bool got = more && take_next(!act, ln.r, ln.gbase, src.next, src.end, np);
    const Key kin = fk.get(np, got);
    const Val vin = fv.get(np, got);
    if (more) {
      fk.advance(src.next);
      fv.advance(src.next);
    }
    if (got) {
      k = kin;
      if (is_sentinel(k)) {
        flags |= kFlagInvalid;
      } else {
        v = vin;
        act = true;
        j = 0;
        salt = static_cast<uint32_t>(np) * 0x9E3779B1u;
        probe_init(static_cast<uint64_t>(k), t.seed, t.p, w, step);
      }
    }
    if (__ballot_sync(kFull, act) == 0) {
      if (!more) break;
      continue;
    }
    Slot s[S];
    uint32_t mm = 0, me = 0, mt = 0;
    const uint64_t lane_slot = static_cast<uint64_t>(w) * W + ln.r * S;
    if (act) {
      load_slots<L, S>(slots + lane_slot, s);
      classify<L, S>(s, k, mm, me, mt);
    }
    const uint32_t fr = me | mt;
    const uint32_t bc = group_vote<G>(fr != 0, ln.gbase);
    // lane of the group that claims (group-uniform), then the slot inside that lane
    const int cl = bc ? nth_set(bc, (salt >> 16) % __popc(bc)) : 0;
    bool ok = false;
    if (act && bc && ln.r == cl) {
      const int sub = nth_set(fr, (salt >> 8) % __popc(fr));
      ok = L::cas(slots + lane_slot + sub, pick<L, S>(s, sub), L::make(k, v));
    }
    if constexpr (G > 1) ok = __shfl_sync(kFull, ok, ln.gbase + cl);
    if (act) {
      if (ok) {
        if (ln.r == 0) ++added;
        act = false;
      } else if (!bc) {
        if (++j >= t.p) {
          flags |= kFlagProbeLimit;
          act = false;
        } else {
          w = probe_next(w, step, t.p);
        }
      } else {
        salt = salt * 0x2C9277B5u + 0xAC564B05u;  // lost the slot: read the window again, pick anew
      }
    }
  }
  flush_flags(t.status, flags);
  flush_delta(t.size, added);
}

// ---- count_values / retrieve_multi: walk to the first window with an empty slot -------
// kWrite = false: offs[pos] = number of copies of keys[pos].
// kWrite = true: the copies go to out[offs[pos] ..) (at most offs[pos+1] - offs[pos]);
// a walk ends early once its segment is full.
template <class L, int G, int S, bool kWrite>
__global__ void __launch_bounds__(256) k_oa_walk(TableDesc t, const typename L::Key* __restrict__ keys, uint64_t n,
                                                 uint64_t* __restrict__ offs,
                                                 typename L::Val* __restrict__ out) {
  using Slot = typename L::Slot;
  using Key = typename L::Key;
  RangeSrc src(StridedChunks{}, n, kWalkChunk);
  if (src.next >= src.end) return;
  const SvLane<L, G, S> ln;
  constexpr int W = G * S;
  const Slot* slots = static_cast<const Slot*>(t.slots);
  bool act = false;
  uint64_t pos = 0, base = 0, cap = 0, cnt = 0;
  Key k = 0;
  uint32_t w = 0, step = 0, j = 0, flags = 0;
  Feed<Key> fk;
  while (true) {
    const bool more = src.ensure();
    if (more && src.fresh) {
      fk.load(keys, src.next, src.end);
      src.fresh = false;
    }
    uint64_t np = 0;
    const bool got = more && take_next(!act, ln.r, ln.gbase, src.next, src.end, np);
    const Key kin = fk.get(np, got);
    if (more) fk.advance(src.next);
    if (got) {
      pos = np;
      k = kin;
      cnt = 0;
      if (kWrite) {
        base = offs[pos];
        cap = offs[pos + 1] - base;
      }
      if (is_sentinel(k)) {
        flags |= kFlagInvalid;
        if (!kWrite && ln.r == 0) offs[pos] = 0;
      } else if (!kWrite || cap != 0) {  // a query counted 0 has nothing to copy
        act = true;
        j = 0;
        probe_init(static_cast<uint64_t>(k), t.seed, t.p, w, step);
      }
    }
    if (__ballot_sync(kFull, act) == 0) {
      if (!more) break;
      continue;
    }
    Slot s[S];
    uint32_t mm = 0, me = 0, mt = 0;
    if (act) {
      load_slots<L, S>(slots + static_cast<uint64_t>(w) * W + ln.r * S, s);
      classify<L, S>(s, k, mm, me, mt);
    }
    const uint32_t mine = __popc(mm);
    const uint32_t here = group_sum<G>(mine);
    const uint32_t before = kWrite ? group_exclusive<G>(mine, ln.r) : 0u;  // every lane shuffles
    const uint32_t be = group_vote<G>(me != 0, ln.gbase);
    if (kWrite && act && mine) {
      uint64_t o = cnt + before;
#pragma unroll
      for (int i = 0; i < S; ++i)
        if ((mm >> i) & 1u) {
          if (o < cap) out[base + o] = L::val(s[i]);
          ++o;
        }
    }
    if (act) {
      cnt += here;
      if (be || (kWrite && cnt >= cap) || ++j >= t.p) {
        if (!kWrite && ln.r == 0) offs[pos] = cnt;
        act = false;
      } else {
        w = probe_next(w, step, t.p);
      }
    }
  }
  flush_flags(t.status, flags);
}

// ---- erase: every copy of the key becomes a tombstone -----------------------------------
template <class L, int G, int S>
__global__ void __launch_bounds__(256) k_oa_erase(TableDesc t, const typename L::Key* __restrict__ keys, uint64_t n) {
  using Slot = typename L::Slot;
  using Key = typename L::Key;
  RangeSrc src(StridedChunks{}, n, kWalkChunk);
  if (src.next >= src.end) return;
  const SvLane<L, G, S> ln;
  constexpr int W = G * S;
  Slot* slots = static_cast<Slot*>(t.slots);
  bool act = false;
  Key k = 0;
  uint32_t w = 0, step = 0, j = 0, flags = 0;
  long long removed = 0;
  Feed<Key> fk;
  while (true) {
    const bool more = src.ensure();
    if (more && src.fresh) {
      fk.load(keys, src.next, src.end);
      src.fresh = false;
    }
    uint64_t np = 0;
    const bool got = more && take_next(!act, ln.r, ln.gbase, src.next, src.end, np);
    const Key kin = fk.get(np, got);
    if (more) fk.advance(src.next);
    if (got) {
      k = kin;
      if (is_sentinel(k)) {
        flags |= kFlagInvalid;
      } else {
        act = true;
        j = 0;
        probe_init(static_cast<uint64_t>(k), t.seed, t.p, w, step);
      }
    }
    if (__ballot_sync(kFull, act) == 0) {
      if (!more) break;
      continue;
    }
    Slot s[S];
    uint32_t mm = 0, me = 0, mt = 0;
    const uint64_t lane_slot = static_cast<uint64_t>(w) * W + ln.r * S;
    if (act) {
      load_slots<L, S>(slots + lane_slot, s);
      classify<L, S>(s, k, mm, me, mt);
#pragma unroll
      for (int i = 0; i < S; ++i)
        if ((mm >> i) & 1u) removed += L::cas(slots + lane_slot + i, s[i], L::tomb()) ? 1 : 0;
    }
    const uint32_t be = group_vote<G>(me != 0, ln.gbase);
    if (act) {
      if (be || ++j >= t.p) act = false;
      else w = probe_next(w, step, t.p);
    }
  }
  flush_flags(t.status, flags);
  flush_delta(t.size, -removed);
}

// ---- num_keys: distinct live keys --------------------------------------------------------
// One thread per slot: a live slot counts when it holds the first copy of its key along the
// key's probing sequence (window order, then slot order inside the window).  The slot
// itself lies on that sequence, so the walk ends at it at the latest.
template <class L>
__global__ void __launch_bounds__(256) k_oa_num_keys(TableDesc t, uint64_t capacity) {
  using Slot = typename L::Slot;
  using Key = typename L::Key;
  const Slot* slots = static_cast<const Slot*>(t.slots);
  unsigned long long mine = 0;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < capacity;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    Slot s[1];
    load_slots<L, 1>(slots + i, s);
    const Key k = L::key(s[0]);
    if (is_sentinel(k)) continue;
    uint32_t w = 0, step = 0;
    probe_init(static_cast<uint64_t>(k), t.seed, t.p, w, step);
    uint64_t first = i;
    for (uint32_t j = 0; j < t.p; ++j) {
      bool hit = false;
      for (uint32_t q = 0; q < t.W; ++q) {
        const uint64_t at = static_cast<uint64_t>(w) * t.W + q;
        if (at == i) {
          hit = true;
          break;
        }
        Slot o[1];
        load_slots<L, 1>(slots + at, o);
        if (L::key(o[0]) == k) {
          first = at;
          hit = true;
          break;
        }
      }
      if (hit) break;
      w = probe_next(w, step, t.p);
    }
    mine += first == i ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(kFull, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(t.nkeys, mine);
}

}  // namespace wc
