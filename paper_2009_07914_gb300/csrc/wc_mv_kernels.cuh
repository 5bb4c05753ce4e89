// Multi-value kernels (Sec. IV-B4 and IV-C).
//
// Storage: each distinct key is stored ONCE in a key store of 16-byte slots
// {uint64 key, uint64 handle} (the single-value table of list handles of Sec. IV-C);
// its values live in a value pool.  A bulk insert appends, for every key of the batch,
// one bucket of exactly that batch's count of the key -- the bucket list with growth
// lambda = 1 and s0 = count (Sec. V-C's "optimal growth strategy") -- linked to the key's
// earlier buckets by a header that holds the previous handle (the back reference of
// Sec. IV-C).  Handle bits: [0, 28) total values of the key, bit 28 "has an earlier
// bucket", [29, 64) pool offset of the newest bucket (in value elements).
//
// Bulk insert = three passes over the batch (plus a clear of the per-slot counters):
//   1. count: aggregate the batch tile by tile in shared memory (a hot key costs one
//      global probe and one atomic per tile instead of one per occurrence), insert each
//      distinct key into the key store, add its tile count to pending[slot], and record
//      per tile the distinct keys' slots and counts and per element its key's list
//      position and its rank among the tile's copies of the key (TileRecord);
//   2. allocate: one pass over the key store reserves every key's bucket from the pool
//      (block-aggregated bump allocation) and rewrites its handle;
//   3. place: from the record, reserve each tile's run inside each key's bucket with one
//      atomic on pending[slot] and write every value at run start + rank (no key is
//      hashed or looked up again).
// Within a bucket the order of values is unspecified (the paper's multi-value semantics
// do not order values).
#pragma once

#include "wc_device.cuh"
#include "wc_internal.h"
#include "wc_partition.cuh"
#include "wc_sv_kernels.cuh"

namespace wc {

using KsL = LayoutP64;
using KsSlot = LayoutP64::Slot;

constexpr uint64_t kCountBits = 28;
constexpr uint64_t kMaxCount = (1ull << kCountBits) - 1;
constexpr uint32_t kPoison = 0x80000000u;  // pending[] mark of a bucket that was not allocated

__device__ __forceinline__ uint64_t h_count(uint64_t h) { return h & kMaxCount; }
__device__ __forceinline__ bool h_prev(uint64_t h) { return (h >> kCountBits) & 1ull; }
__device__ __forceinline__ uint64_t h_offset(uint64_t h) { return h >> (kCountBits + 1); }
__device__ __forceinline__ uint64_t h_make(uint64_t off, uint64_t cnt, bool prev) {
  return (off << (kCountBits + 1)) | (static_cast<uint64_t>(prev) << kCountBits) | cnt;
}

// Header elements in front of a non-first bucket (one uint64 previous handle).
template <int VB>
struct Hdr {
  static constexpr uint64_t kElems = 8 / VB;
};

template <int VB>
struct PoolT;
template <>
struct PoolT<4> {
  using T = uint32_t;
};
template <>
struct PoolT<8> {
  using T = unsigned long long;
};

// ---- bucket growth strategy (Sec. IV-C) ----------------------------------------------------
// With a growth strategy a key's buckets have fixed sizes s_0, s_1, ... (its bucket i holds
// its values S_{i-1} .. S_i - 1, S_i = s_0 + ... + s_i); an insert call first fills the
// key's last bucket, then allocates the buckets it still needs in one contiguous chunk.
// Every bucket but the first leads with a header holding the handle of the previous
// bucket {its start, S_{i-1}, i - 1 > 0}, the same back references as the exact layout,
// so the count and retrieve kernels read both layouts alike.

// Values in buckets 0..i (0 for i < 0).
__device__ __forceinline__ uint64_t g_cum_size(const PoolDesc& pd, int64_t i) {
  if (i < 0) return 0;
  if (pd.growth == kGrowConst) return static_cast<uint64_t>(i + 1) * pd.s0;
  return __ldg(pd.cum_size + i);
}

// Pool elements of buckets 0..i (0 for i < 0).
__device__ __forceinline__ uint64_t g_cum_foot(const PoolDesc& pd, int64_t i) {
  if (i < 0) return 0;
  if (pd.growth == kGrowConst) return pd.foot0 + static_cast<uint64_t>(i) * pd.foot;
  return __ldg(pd.cum_foot + i);
}

// Bucket holding the key's value number v (0-based, insertion order).
__device__ __forceinline__ int64_t g_bucket_of(const PoolDesc& pd, uint64_t v) {
  if (pd.growth == kGrowConst) return static_cast<int64_t>(v / pd.s0);
  uint32_t lo = 0, hi = pd.nbuckets - 1;  // first i with S_i > v (S_{last} >= 2^28 > v)
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(pd.cum_size + mid) > v) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Pool index of value number v of a key whose handle after this call's allocation is H
// and whose count before the call was c0 (v >= c0: a value of this call).
template <int VB>
__device__ __forceinline__ uint64_t g_value_index(const PoolDesc& pd, uint64_t H, uint64_t c0, uint64_t v) {
  using V = typename PoolT<VB>::T;
  const uint64_t c1 = h_count(H), o1 = h_offset(H);
  const int64_t b1 = g_bucket_of(pd, c1 - 1), i = g_bucket_of(pd, v);
  uint64_t start;
  if (i == b1) {
    start = o1;
  } else if (g_cum_size(pd, i - 1) >= c0) {  // allocated by this call: in the chunk ending with b1
    start = o1 - (g_cum_foot(pd, b1 - 1) - g_cum_foot(pd, i - 1));
  } else {  // the key's earlier last bucket: bucket i + 1 (first of the chunk) links to it
    const uint64_t next = o1 - (g_cum_foot(pd, b1 - 1) - g_cum_foot(pd, i));
    start = h_offset(*reinterpret_cast<const unsigned long long*>(static_cast<const V*>(pd.pool) + next));
  }
  return start + (i > 0 ? Hdr<VB>::kElems : 0) + (v - g_cum_size(pd, i - 1));
}

// ---- key store probes by one thread (W slots per window) ------------------------------

// Find the key; returns its slot index and handle, or -1 if absent (Sec. IV-B4 early
// exit at the first window holding an empty slot).
template <int W>
__device__ int64_t ks_find(const TableDesc& t, uint64_t k, uint64_t& handle) {
  const KsSlot* slots = static_cast<const KsSlot*>(t.slots);
  uint32_t w, step;
  probe_init(k, t.seed, t.p, w, step);
  for (uint32_t j = 0; j < t.p; ++j) {
    KsSlot s[W];
    const uint64_t base = static_cast<uint64_t>(w) * W;
    load_slots<KsL, W>(slots + base, s);
    uint32_t mm, me, mt;
    classify<KsL, W>(s, k, mm, me, mt);
    if (mm) {
      handle = pick<KsL, W>(s, __ffs(mm) - 1).v;
      return static_cast<int64_t>(base + __ffs(mm) - 1);
    }
    if (me) return -1;
    w = probe_next(w, step, t.p);
  }
  return -1;
}

// ---- passes 1 and 3: tile aggregation in shared memory ----------------------------------

// A block of kThreads threads aggregates tiles of kThreads * kAggPerThread batch elements
// in a shared table of twice as many slots (load <= 1/2).  Smaller blocks hold smaller
// tables, so more of them fit on an SM and more tiles' probe phases overlap.
constexpr int kAggPerThread = 4;
template <int kThreads>
struct Agg {
  static constexpr int kTile = kThreads * kAggPerThread;  // batch elements per tile
  static constexpr int kSlots = 2 * kTile;
  // the tile's hash table (keys, counts, list, key-store slots, list positions), then the
  // next tile's input keys (key_bytes each), copied in while the current tile is processed
  static constexpr size_t table_bytes() {
    return kSlots * (sizeof(unsigned long long) + sizeof(uint32_t) + sizeof(unsigned short)) +
           kTile * (sizeof(uint32_t) + sizeof(unsigned short));
  }
  static constexpr size_t smem_bytes(size_t key_bytes) { return table_bytes() + kTile * key_bytes; }
};

// What the counting pass leaves for the placing pass (k_mv_place), per tile of the batch:
// the tile's distinct keys as (key-store slot, count) at list[tile * kTile ..] (slot all
// ones: the key could not be stored), their number at len[tile], and for every element
// elem[e] = (position of its key in the list) << 16 | (its rank among the tile's elements
// of that key), or all ones for a sentinel key.
struct TileRecord {
  uint2* list;
  uint32_t* elem;
  uint32_t* len;
};

template <int kSlots>
__device__ __forceinline__ int smem_find_or_insert(unsigned long long* s_key, unsigned long long key) {
  volatile unsigned long long* vk = s_key;
  uint32_t h = static_cast<uint32_t>(fmix64(key) >> 40) & (kSlots - 1);
  while (true) {  // at most kSlots / 2 distinct keys in a table of kSlots slots
    const unsigned long long cur = vk[h];
    if (cur == key) return static_cast<int>(h);
    if (cur == 0ull) {
      const unsigned long long prev = atomicCAS(s_key + h, 0ull, key);
      if (prev == 0ull || prev == key) return static_cast<int>(h);
    }
    h = (h + 1) & (kSlots - 1);
  }
}

// Exclusive block scan of one uint32 per thread; total gets the sum.
template <int kThreads>
__device__ __forceinline__ uint32_t block_exclusive_u32(uint32_t x, uint32_t& total, uint32_t* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
  total = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) {
    if (w < warp) before += s_w[w];
    total += s_w[w];
  }
  __syncthreads();
  return before + inc - x;
}

// The global phase of one tile: every distinct key of the tile (s_list[0..len)) is found
// in or inserted into the key store with one lane per key.
// The loop is warp-uniform: each trip loads one window for every lane holding a key,
// so a warp's window loads are in flight together, and a lane that finishes takes the
// next key of the list.  pending[slot] += the key's tile count, and s_ks[i] = slot for
// the key at list position i (it stays all ones for a key the key store could not take).
template <int W>
__device__ __forceinline__ void ks_global_phase(const TableDesc& t, const PoolDesc& pd,
                                                unsigned long long* s_key, uint32_t* s_cnt,
                                                uint32_t* s_ks,
                                                const unsigned short* s_list,
                                                uint32_t len, uint32_t* s_next, uint32_t& flags,
                                                long long& created) {
  KsSlot* slots = static_cast<KsSlot*>(t.slots);
  const int lane = threadIdx.x & 31;
  bool act = false, more = true;
  uint32_t e = 0, w = 0, step = 0, j = 0, li = 0;
  unsigned long long k = 0;
  bool have_t = false;
  uint64_t t_slot = 0;
  KsSlot t_word{};
  while (true) {
    const uint32_t idle = __ballot_sync(kFull, !act);
    if (idle && more) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(s_next, static_cast<uint32_t>(__popc(idle)));
      base = __shfl_sync(kFull, base, 0);
      const uint32_t mine = base + __popc(idle & ((1u << lane) - 1u));
      if (!act && mine < len) {
        li = mine;
        e = s_list[mine];
        k = s_key[e];
        act = true;
        j = 0;
        have_t = false;
        probe_init(k, t.seed, t.p, w, step);
      }
      more = base + __popc(idle) < len;
    }
    if (__ballot_sync(kFull, act) == 0) {
      if (!more) break;
      continue;
    }
    if (act) {
      KsSlot sl[W];
      const uint64_t b = static_cast<uint64_t>(w) * W;
      load_slots<KsL, W>(slots + b, sl);
      uint32_t mm, me, mt;
      classify<KsL, W>(sl, k, mm, me, mt);
      int64_t slot = -1;
      if (mm) {
        slot = static_cast<int64_t>(b + __ffs(mm) - 1);
      } else {
        const bool last = j + 1 >= t.p;
        if (me || last) {
          if (have_t) {
            if (KsL::cas(slots + t_slot, t_word, KsL::make(k, 0))) {
              slot = static_cast<int64_t>(t_slot);
              ++created;
            } else {
              have_t = false;  // the tombstone was taken: probe again from the start
              j = 0;
              probe_init(k, t.seed, t.p, w, step);
            }
          } else if (me | mt) {
            const int sub = __ffs(me | mt) - 1;
            if (KsL::cas(slots + b + sub, pick<KsL, W>(sl, sub), KsL::make(k, 0))) {
              slot = static_cast<int64_t>(b + sub);
              ++created;
            }
            // else: the slot was taken; read the window again
          } else {
            flags |= kFlagProbeLimit;
            act = false;
          }
        } else {
          if (mt && !have_t) {
            have_t = true;
            t_slot = b + __ffs(mt) - 1;
            t_word = pick<KsL, W>(sl, __ffs(mt) - 1);
          }
          ++j;
          w = probe_next(w, step, t.p);
        }
      }
      if (slot >= 0) {
        atomicAdd(pd.pending + slot, s_cnt[e]);
        s_ks[li] = static_cast<uint32_t>(slot);
        act = false;
      }
    }
  }
}

template <class KIn, int W, int kAggThreads>
// tile_counter != nullptr: blocks take tiles in increasing order from it (the batch is
// sorted by key-store region, so the active tiles touch one region of the key store and
// one range of the value pool at a time); otherwise tiles are strided over the grid.
__global__ void __launch_bounds__(kAggThreads, W <= 4 ? 1280 / kAggThreads : 1) k_mv_aggregate(TableDesc t, PoolDesc pd, const KIn* __restrict__ keys,
                                                              uint64_t n, unsigned long long* tile_counter,
                                                              TileRecord rec) {
  constexpr int kAggTile = Agg<kAggThreads>::kTile;
  constexpr int kAggSlots = Agg<kAggThreads>::kSlots;
  extern __shared__ unsigned long long agg_smem[];  // Agg<kAggThreads>::smem_bytes(sizeof(KIn)) bytes
  unsigned long long* s_key = agg_smem;
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(agg_smem + kAggSlots);
  uint32_t* s_ks = s_cnt + kAggSlots;  // key-store slot of every list entry (kAggTile)
  unsigned short* s_pos = reinterpret_cast<unsigned short*>(s_ks + kAggTile);  // list position of every table entry
  unsigned short* s_list = s_pos + kAggSlots;  // the tile's distinct keys (table entries), kAggTile
  KIn* s_in = reinterpret_cast<KIn*>(reinterpret_cast<char*>(agg_smem) + Agg<kAggThreads>::table_bytes());
  __shared__ uint32_t s_wsum[kAggThreads / 32];
  __shared__ uint32_t s_len, s_next;
  const int lane = threadIdx.x & 31;
  const uint64_t ntiles = (n + kAggTile - 1) / kAggTile;
  uint32_t flags = 0;
  long long created = 0;
  __shared__ unsigned long long s_tile, s_ntile;
  // the keys of tile `tl` go to s_in asynchronously (cp.async) while the block works on
  // the tile before it, so a tile starts without a wait on HBM
  auto prefetch = [&](uint64_t tl) {
    const uint64_t b = tl * kAggTile;
    const uint32_t cnt = static_cast<uint32_t>(n - b < kAggTile ? n - b : kAggTile);
    for (uint32_t i = threadIdx.x; i < cnt; i += kAggThreads) cp_async_elem(s_in + i, keys + b + i);
  };
  uint64_t tile = blockIdx.x;
  if (tile_counter != nullptr) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1ull);
    __syncthreads();
    tile = s_tile;
  }
  if (tile < ntiles) prefetch(tile);
  while (tile < ntiles) {
    // the next tile: taken now, so that its keys can be copied in during this one
    uint64_t next = tile + gridDim.x;
    if (tile_counter != nullptr) {
      if (threadIdx.x == 0) s_ntile = atomicAdd(tile_counter, 1ull);
    }
    for (int e = threadIdx.x; e < kAggSlots; e += kAggThreads) {
      s_key[e] = 0ull;
      s_cnt[e] = 0u;
      if (e < kAggTile) s_ks[e] = ~0u;
    }
    cp_async_wait_all();
    __syncthreads();
    if (tile_counter != nullptr) next = s_ntile;
    KIn kin_t[kAggPerThread];
#pragma unroll
    for (int k = 0; k < kAggPerThread; ++k) {
      const uint64_t e = tile * kAggTile + static_cast<uint64_t>(k) * kAggThreads + threadIdx.x;
      kin_t[k] = e < n ? s_in[k * kAggThreads + threadIdx.x] : KIn(0);
    }
    __syncthreads();  // s_in is free again
    if (next < ntiles) prefetch(next);
    int my_slot[kAggPerThread];
    uint32_t my_rank[kAggPerThread];
#pragma unroll
    for (int k = 0; k < kAggPerThread; ++k) {
      const uint64_t e = tile * kAggTile + static_cast<uint64_t>(k) * kAggThreads + threadIdx.x;
      unsigned long long key = 0ull;
      bool valid = false;
      if (e < n) {
        const KIn kin = kin_t[k];
        valid = !is_sentinel(kin);
        if (valid) key = static_cast<unsigned long long>(kin);
        else flags |= kFlagInvalid;
      }
      // equal keys of the warp are counted by their lowest lane
      const uint32_t peers = __match_any_sync(kFull, key);
      const int leader = __ffs(peers) - 1;
      int slot = -1;
      uint32_t base = 0;
      if (valid && lane == leader) {
        slot = smem_find_or_insert<kAggSlots>(s_key, key);
        base = atomicAdd(s_cnt + slot, static_cast<uint32_t>(__popc(peers)));
      }
      slot = __shfl_sync(kFull, slot, leader);
      base = __shfl_sync(kFull, base, leader);
      my_slot[k] = valid ? slot : -1;
      my_rank[k] = base + __popc(peers & ((1u << lane) - 1u));
    }
    __syncthreads();
    // compact the tile's distinct keys into a list, then probe them warp-uniformly; a
    // thread takes every kAggThreads-th table entry, so a warp reads consecutive entries
    // (the list order is of no consequence)
    {
      constexpr int kPer = kAggSlots / kAggThreads;
      uint32_t c = 0;
      bool used[kPer];
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        used[i] = s_key[i * kAggThreads + threadIdx.x] != 0ull;
        c += used[i];
      }
      uint32_t total = 0;
      uint32_t pos = block_exclusive_u32<kAggThreads>(c, total, s_wsum);
#pragma unroll
      for (int i = 0; i < kPer; ++i)
        if (used[i]) {
          const int e = i * kAggThreads + threadIdx.x;
          s_pos[e] = static_cast<unsigned short>(pos);
          s_list[pos++] = static_cast<unsigned short>(e);
        }
      if (threadIdx.x == 0) {
        s_len = total;
        s_next = 0;
      }
      __syncthreads();
    }
    {
      // the record of this tile for the placing pass: element words now (the list
      // positions are known), the (slot, count) list after the key-store phase
#pragma unroll
      for (int k = 0; k < kAggPerThread; ++k) {
        const uint64_t e = tile * kAggTile + static_cast<uint64_t>(k) * kAggThreads + threadIdx.x;
        if (e < n)
          rec.elem[e] = my_slot[k] < 0 ? ~0u : (static_cast<uint32_t>(s_pos[my_slot[k]]) << 16) | my_rank[k];
      }
    }
    ks_global_phase<W>(t, pd, s_key, s_cnt, s_ks, s_list, s_len, &s_next, flags, created);
    {
      __syncthreads();
      const uint32_t len = s_len;
      for (uint32_t i = threadIdx.x; i < len; i += kAggThreads) {
        rec.list[tile * kAggTile + i] = make_uint2(s_ks[i], s_cnt[s_list[i]]);
      }
      if (threadIdx.x == 0) rec.len[tile] = len;
    }
    __syncthreads();
    tile = next;
  }
  cp_async_wait_all();
  flush_flags(t.status, flags);
  flush_delta(t.nkeys, created);
}

// ---- pass 3: placing the values ------------------------------------------------------------
// With the counting pass's record of every tile (TileRecord), no key is looked up again:
// per tile, each distinct key reserves its run in its bucket with one atomic on the
// pending counter that pass 2 reset (Sec. IV-C's per-key cursor), and every element writes
// its value at run start + its rank.  Tiles are taken in increasing order from
// tile_counter when given (a region-split batch: the pool is written range by range),
// else strided over the grid.  Element words and values are loaded at the start of a tile,
// so their loads overlap the reservations.
template <int VB, int kThreads>
__global__ void __launch_bounds__(kThreads) k_mv_place(TableDesc t, PoolDesc pd, TileRecord rec,
                                                       const void* __restrict__ vals, uint64_t n,
                                                       unsigned long long* tile_counter) {
  using V = typename PoolT<VB>::T;
  constexpr int kTile = Agg<kThreads>::kTile;
  constexpr int kPer = kTile / kThreads;  // list entries and elements per thread
  __shared__ unsigned long long s_b[kTile];  // run start of each distinct key (all ones: none)
  __shared__ unsigned long long s_h[kTile];  // growth strategy: the key's handle
  __shared__ uint32_t s_c[kTile];            // growth strategy: the key's count before the call
  __shared__ unsigned long long s_tile, s_ntile;
  const KsSlot* slots = static_cast<const KsSlot*>(t.slots);
  V* pool = static_cast<V*>(pd.pool);
  const V* vin = static_cast<const V*>(vals);
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  uint64_t tile = blockIdx.x;
  if (tile_counter != nullptr) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1ull);
    __syncthreads();
    tile = s_tile;
  }
  while (tile < ntiles) {
    uint32_t ew[kPer];
    V v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint64_t e = tile * kTile + static_cast<uint64_t>(k) * kThreads + threadIdx.x;
      ew[k] = e < n ? rec.elem[e] : ~0u;
      v[k] = e < n ? vin[e] : V(0);
    }
    const uint32_t len = rec.len[tile];
    uint2 r[kPer];
    uint32_t old[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = static_cast<uint32_t>(k) * kThreads + threadIdx.x;
      r[k] = i < len ? rec.list[tile * kTile + i] : make_uint2(~0u, 0u);
    }
    // the reservations and the handle loads of all the thread's keys go out together
    uint64_t handle[kPer];
    uint32_t c0[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const bool ok = r[k].x != ~0u;
      old[k] = ok ? atomicAdd(pd.pending + r[k].x, r[k].y) : kPoison;
      handle[k] = ok ? slots[r[k].x].v : 0ull;
      c0[k] = ok && pd.growth != kGrowExact ? pd.base[r[k].x] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = static_cast<uint32_t>(k) * kThreads + threadIdx.x;
      if (i >= len) continue;
      if (old[k] & kPoison) {  // no stored key, or no bucket was allocated for it
        s_b[i] = ~0ull;
        continue;
      }
      if (pd.growth == kGrowExact) {
        s_b[i] = h_offset(handle[k]) + (h_prev(handle[k]) ? Hdr<VB>::kElems : 0) + old[k];
      } else {
        // growth: `old` is the value number of the run's first value; the handle and the
        // key's count before the call give each value's place
        s_b[i] = old[k];
        s_h[i] = handle[k];
        s_c[i] = c0[k];
      }
    }
    if (tile_counter != nullptr && threadIdx.x == 0) s_ntile = atomicAdd(tile_counter, 1ull);
    __syncthreads();
    const uint64_t next = tile_counter != nullptr ? s_ntile : tile + gridDim.x;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (ew[k] == ~0u) continue;
      const uint32_t i = ew[k] >> 16, rank = ew[k] & 0xffffu;
      const unsigned long long b = s_b[i];
      if (b == ~0ull) continue;
      if (pd.growth == kGrowExact)
        pool[b + rank] = v[k];
      else
        pool[g_value_index<VB>(pd, s_h[i], s_c[i], b + rank)] = v[k];
    }
    __syncthreads();
    tile = next;
  }
}

// ---- pass 2: bucket allocation ----------------------------------------------------------

constexpr int kAllocThreads = 256;
constexpr int kAllocItems = 8;

// Exclusive block scan of one uint64 per thread; returns this thread's prefix and the
// block total through `total`.
template <int kThreads>
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t x, uint64_t& total, uint64_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    constexpr int nw = kThreads / 32;
    uint64_t v = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += y;
    }
    if (lane < nw) s_warp[lane] = v;  // inclusive warp totals
  }
  __syncthreads();
  total = s_warp[kThreads / 32 - 1];
  const uint64_t before = warp > 0 ? s_warp[warp - 1] : 0;
  __syncthreads();
  return before + inc - x;
}

template <int VB>
__global__ void __launch_bounds__(kAllocThreads) k_mv_alloc(TableDesc t, PoolDesc pd, uint64_t capacity) {
  using V = typename PoolT<VB>::T;
  __shared__ uint64_t s_warp[kAllocThreads / 32];
  __shared__ unsigned long long s_block_base;
  __shared__ int s_ok;
  KsSlot* slots = static_cast<KsSlot*>(t.slots);
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * (kAllocThreads * kAllocItems);
  uint32_t c[kAllocItems];
  uint64_t h[kAllocItems];
  uint64_t need[kAllocItems];
  uint64_t mine = 0;
  uint32_t flags = 0;
#pragma unroll
  for (int k = 0; k < kAllocItems; ++k) {
    const uint64_t s = base + static_cast<uint64_t>(k) * kAllocThreads + threadIdx.x;
    c[k] = s < capacity ? pd.pending[s] : 0u;
    h[k] = 0;
    need[k] = 0;
    if (c[k]) {
      h[k] = slots[s].v;
      const uint64_t old = h_count(h[k]);
      if ((c[k] & kPoison) || old + c[k] > kMaxCount) {
        flags |= kFlagCountOverflow;
        pd.pending[s] = kPoison;
        c[k] = 0;
      } else {
        const uint64_t hdr = old ? Hdr<VB>::kElems : 0;
        need[k] = c[k] + hdr;
        if (VB == 4) need[k] = (need[k] + 1) & ~1ull;  // keep bucket starts 8-byte aligned
      }
    }
    mine += need[k];
  }
  uint64_t total = 0;
  const uint64_t pre = block_exclusive_scan<kAllocThreads>(mine, total, s_warp);
  if (threadIdx.x == 0) {
    const unsigned long long b = total ? atomicAdd(pd.cursor, static_cast<unsigned long long>(total)) : 0ull;
    s_block_base = b;
    s_ok = b + total <= pd.capacity;
  }
  __syncthreads();
  long long added = 0;
  uint64_t off = s_block_base + pre;
#pragma unroll
  for (int k = 0; k < kAllocItems; ++k) {
    if (need[k] == 0) continue;
    const uint64_t s = base + static_cast<uint64_t>(k) * kAllocThreads + threadIdx.x;
    if (!s_ok) {
      flags |= kFlagPoolExhausted;
      pd.pending[s] = kPoison;
      continue;
    }
    const uint64_t old = h_count(h[k]);
    if (old) *reinterpret_cast<unsigned long long*>(static_cast<V*>(pd.pool) + off) = h[k];
    slots[s].v = h_make(off, old + c[k], old != 0);
    pd.pending[s] = 0u;  // becomes the bucket's fill cursor for pass 3
    added += c[k];
    off += need[k];
  }
  flush_flags(t.status, flags);
  flush_delta(t.size, added);
}

// Pass 2 with a growth strategy: a key with c new values and c0 old ones needs its
// buckets first..b1 (first = the bucket after its last one, b1 = the bucket of value
// c0 + c - 1); they are allocated as one chunk, their headers written, the handle pointed
// at bucket b1.  pending[s] and base[s] become c0: pass 3 counts value numbers from there.
template <int VB>
__global__ void __launch_bounds__(kAllocThreads) k_mv_alloc_growth(TableDesc t, PoolDesc pd, uint64_t capacity) {
  using V = typename PoolT<VB>::T;
  __shared__ uint64_t s_warp[kAllocThreads / 32];
  __shared__ unsigned long long s_block_base;
  __shared__ int s_ok;
  KsSlot* slots = static_cast<KsSlot*>(t.slots);
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * (kAllocThreads * kAllocItems);
  uint32_t c[kAllocItems];
  uint64_t h[kAllocItems];
  uint64_t need[kAllocItems];
  uint64_t mine = 0;
  uint32_t flags = 0;
#pragma unroll
  for (int k = 0; k < kAllocItems; ++k) {
    const uint64_t s = base + static_cast<uint64_t>(k) * kAllocThreads + threadIdx.x;
    c[k] = s < capacity ? pd.pending[s] : 0u;
    h[k] = 0;
    need[k] = 0;
    if (c[k]) {
      h[k] = slots[s].v;
      const uint64_t old = h_count(h[k]);
      if ((c[k] & kPoison) || old + c[k] > kMaxCount) {
        flags |= kFlagCountOverflow;
        pd.pending[s] = kPoison;
        c[k] = 0;
      } else {
        const int64_t first = old ? g_bucket_of(pd, old - 1) + 1 : 0;
        const int64_t b1 = g_bucket_of(pd, old + c[k] - 1);
        need[k] = first <= b1 ? g_cum_foot(pd, b1) - g_cum_foot(pd, first - 1) : 0;
      }
    }
    mine += need[k];
  }
  uint64_t total = 0;
  const uint64_t pre = block_exclusive_scan<kAllocThreads>(mine, total, s_warp);
  if (threadIdx.x == 0) {
    const unsigned long long b = total ? atomicAdd(pd.cursor, static_cast<unsigned long long>(total)) : 0ull;
    s_block_base = b;
    s_ok = b + total <= pd.capacity;
  }
  __syncthreads();
  long long added = 0;
  uint64_t off = s_block_base + pre;
  V* pool = static_cast<V*>(pd.pool);
#pragma unroll
  for (int k = 0; k < kAllocItems; ++k) {
    if (c[k] == 0) continue;
    const uint64_t s = base + static_cast<uint64_t>(k) * kAllocThreads + threadIdx.x;
    if (need[k] != 0 && !s_ok) {
      flags |= kFlagPoolExhausted;
      pd.pending[s] = kPoison;
      continue;
    }
    const uint64_t old = h_count(h[k]);
    const int64_t first = old ? g_bucket_of(pd, old - 1) + 1 : 0;
    const int64_t b1 = g_bucket_of(pd, old + c[k] - 1);
    uint64_t tail = h_offset(h[k]);  // start of the key's last bucket so far
    for (int64_t i = first; i <= b1; ++i) {
      const uint64_t start = off + (g_cum_foot(pd, i - 1) - g_cum_foot(pd, first - 1));
      if (i > 0)
        *reinterpret_cast<unsigned long long*>(pool + start) = h_make(tail, g_cum_size(pd, i - 1), i - 1 > 0);
      tail = start;
    }
    slots[s].v = h_make(tail, old + c[k], b1 > 0);
    pd.pending[s] = static_cast<uint32_t>(old);  // value number of the call's first value
    pd.base[s] = static_cast<uint32_t>(old);
    added += c[k];
    off += need[k];
  }
  flush_flags(t.status, flags);
  flush_delta(t.size, added);
}

// ---- count_values: per-query count (the retrieve engine over the key store) ------------

struct EmitCount {
  uint64_t* __restrict__ offs;
  __device__ void operator()(uint64_t pos, bool hit, const KsSlot& s, uint64_t) const {
    offs[pos] = hit ? h_count(s.v) : 0;
  }
};

template <class KIn, int G, int S>
__global__ void __launch_bounds__(256) k_mv_count(TableDesc t, const KIn* __restrict__ keys, uint64_t n,
                                                  uint64_t per_warp, uint64_t* __restrict__ offs) {
  RangeSrc src(n, per_warp, nullptr, 0);
  if (src.next >= src.end) return;
  uint32_t flags = 0;
  EmitCount emit{offs};
  sv_retrieve_range<KsL, G, S, EmitCount, KIn>(t, keys, src, emit, flags);
  flush_flags(t.status, flags);
}

// ---- erase: tombstone the key-store entry, drop every value of the key ------------------

struct OnEraseMV {
  long long pairs = 0;
  __device__ void operator()(const KsSlot& s) { pairs += static_cast<long long>(h_count(s.v)); }
};

template <class KIn, int G, int S>
__global__ void __launch_bounds__(256) k_mv_erase(TableDesc t, const KIn* __restrict__ keys, uint64_t n,
                                                  uint64_t per_warp) {
  RangeSrc src(n, per_warp, nullptr, 0);
  if (src.next >= src.end) return;
  uint32_t flags = 0;
  long long removed = 0;
  OnEraseMV oe;
  sv_erase_range<KsL, G, S, OnEraseMV, KIn>(t, keys, src, flags, removed, oe);
  flush_flags(t.status, flags);
  flush_delta(t.nkeys, -removed);
  flush_delta(t.size, -oe.pairs);
}

// ---- retrieve_multi: load-balanced CSR gather ---------------------------------------------
//
// The work is the merge of the n row ends (offsets[1..n]) with the `total` output
// positions (merge-path decomposition, Merrill and Garland, SC'16): chunk c covers merge
// items [c * L, (c + 1) * L), i.e. a fixed share of rows plus values whatever the skew,
// so one key with 30 M values is spread over thousands of blocks.  A chunk probes the
// key store for each of its rows with a non-zero count (one probe per row, Sec. IV-B4),
// then copies its value range with consecutive threads on consecutive output positions
// (coalesced reads inside a bucket, coalesced writes; the cooperative bucket read of
// Sec. IV-C).

constexpr int kRmThreads = 256;
constexpr int kRmItems = 2048;

// Rows whose end marker lies before merge position d: the first i in [0, n] with
// offs[i + 1] + i >= d (offs[n + 1] taken as infinite).  One warp, 32 probes per step.
__device__ __forceinline__ uint64_t merge_search(const uint64_t* __restrict__ offs, uint64_t n, uint64_t total,
                                                 uint64_t d) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = d > total ? d - total : 0;
  uint64_t hi = d < n ? d : n;
  while (lo < hi) {
    const uint64_t span = hi - lo;
    const uint64_t step = (span + 31) / 32;
    const uint64_t x = lo + static_cast<uint64_t>(lane) * step;
    const bool valid = x < hi;
    const bool ge = valid && (offs[x + 1] + x >= d);
    const uint32_t b = __ballot_sync(kFull, ge);
    if (b) {
      const int k = __ffs(b) - 1;
      const uint64_t nhi = lo + static_cast<uint64_t>(k) * step;
      lo = k == 0 ? lo : lo + static_cast<uint64_t>(k - 1) * step + 1;
      hi = nhi;
    } else {
      const uint64_t last = (hi - 1 - lo) / step;  // last lane that tested a valid point
      lo = lo + last * step + 1;
    }
  }
  return lo;
}

// Pool index of value q (0-based) of a key whose newest bucket handle is h; buckets are
// read newest first.  The walk is bounded by the key's value count.
template <int VB>
__device__ __forceinline__ uint64_t value_index(const PoolDesc& pd, uint64_t h, uint64_t q) {
  using V = typename PoolT<VB>::T;
  const V* pool = static_cast<const V*>(pd.pool);
  for (uint64_t guard = 0; h_prev(h) && guard <= kMaxCount; ++guard) {
    const uint64_t prev = *reinterpret_cast<const unsigned long long*>(pool + h_offset(h));
    const uint64_t here = h_count(h) - h_count(prev);
    if (q < here) return h_offset(h) + Hdr<VB>::kElems + q;
    q -= here;
    h = prev;
  }
  return h_offset(h) + q;
}

// kGrowth: the table uses a bucket growth strategy (rows are copied by walking their
// bucket lists); otherwise every value is found from its row's handle.
template <class KIn, int VB, int W, bool kGrowth>
__global__ void __launch_bounds__(kRmThreads) k_mv_retrieve_multi(TableDesc t, PoolDesc pd, const KIn* __restrict__ keys,
                                                                  uint64_t n, const uint64_t* __restrict__ offs,
                                                                  void* __restrict__ out) {
  using V = typename PoolT<VB>::T;
  __shared__ uint64_t s_off[kRmItems + 2];
  __shared__ uint64_t s_h[kRmItems + 1];
  __shared__ uint64_t s_bounds[2];
  const uint64_t total = offs[n];
  const uint64_t items = n + total;
  const uint64_t nchunks = (items + kRmItems - 1) / kRmItems;
  const int warp = threadIdx.x >> 5;
  const V* pool = static_cast<const V*>(pd.pool);
  V* o = static_cast<V*>(out);
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint64_t d0 = c * kRmItems;
    const uint64_t d1 = d0 + kRmItems < items ? d0 + kRmItems : items;
    if (warp < 2) {
      const uint64_t i = merge_search(offs, n, total, warp == 0 ? d0 : d1);
      if ((threadIdx.x & 31) == 0) s_bounds[warp] = i;
    }
    __syncthreads();
    const uint64_t i0 = s_bounds[0], i1 = s_bounds[1];
    const uint64_t j0 = d0 - i0, j1 = d1 - i1;
    const uint64_t rlast = i1 < n ? i1 : n - 1;
    const int R = i0 < n ? static_cast<int>(rlast - i0 + 1) : 0;
    for (int r = threadIdx.x; r <= R; r += kRmThreads) s_off[r] = offs[i0 + r];
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += kRmThreads) {
      uint64_t h = 0;
      if (s_off[r + 1] > s_off[r]) {
        const KIn kin = keys[i0 + r];
        uint64_t hh = 0;
        if (!is_sentinel(kin) && ks_find<W>(t, static_cast<uint64_t>(kin), hh) >= 0) h = hh;
      }
      s_h[r] = h;
    }
    __syncthreads();
    if constexpr (kGrowth) {
      // growth layouts: a key may have many buckets, so each row's part of the chunk is
      // copied by one thread walking the row's buckets newest first, once
      for (int r = threadIdx.x; r < R; r += kRmThreads) {
        const uint64_t qa = (j0 > s_off[r] ? j0 : s_off[r]) - s_off[r];
        const uint64_t qb = (j1 < s_off[r + 1] ? j1 : s_off[r + 1]) - s_off[r];
        uint64_t h = s_h[r];
        if (qa >= qb || qb > h_count(h)) continue;  // nothing here, or the count changed
        uint64_t acc = 0;  // rank (newest first) of the current bucket's first value
        for (uint64_t guard = 0; guard <= kMaxCount && acc < qb; ++guard) {
          const bool prev = h_prev(h);
          const uint64_t below = prev ? h_count(*reinterpret_cast<const unsigned long long*>(pool + h_offset(h))) : 0;
          const uint64_t here = h_count(h) - below;
          const uint64_t vstart = h_offset(h) + (prev ? Hdr<VB>::kElems : 0);
          const uint64_t lo = qa > acc ? qa : acc, hi = qb < acc + here ? qb : acc + here;
          for (uint64_t q = lo; q < hi; ++q) o[s_off[r] + q] = pool[vstart + (q - acc)];
          acc += here;
          if (!prev) break;
          h = *reinterpret_cast<const unsigned long long*>(pool + h_offset(h));
        }
      }
      __syncthreads();
      continue;
    } else {
    for (uint64_t j = j0 + threadIdx.x; j < j1; j += kRmThreads) {
      int lo = 0, hi = R - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= j) lo = mid;
        else hi = mid - 1;
      }
      const uint64_t q = j - s_off[lo];
      const uint64_t h = s_h[lo];
      // a key whose count changed since count_values keeps its slot in the output
      if (q < h_count(h)) o[j] = pool[value_index<VB>(pd, h, q)];
    }
    }
    __syncthreads();
  }
}

}  // namespace wc
