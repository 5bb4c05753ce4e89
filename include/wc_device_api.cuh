/*
 * wc_device_api.cuh -- device-side API: per-element operations on a single-value table from
 * inside user kernels, and the higher-order bulk calls for_each / for_all (Sec. IV-A:
 * the device-sided interface that fused pipelines call, Sec. IV-B4: for_each(keys,
 * callback) and for_all(callback) with a device callback).  Header-only CUDA C++;
 * include it from .cu files compiled for sm_103a (with --extended-lambda for device
 * lambdas).  It holds the probing sequence the library's own kernels use, so a key
 * inserted here is found by wc_retrieve and the other way round.
 *
 * A table is reached through a wc_device_view (wc.h: wc_table_device_view), a plain
 * struct of device pointers and geometry, passed to kernels by value.  Rules as for the
 * bulk calls: operations of one kind may run concurrently (from any number of threads and
 * kernels); an insert or erase must not overlap a retrieve on the same table (Sec. IV-D).
 *
 * Bucket multi-value tables with a growth strategy take per-element appends (append
 * below; Sec. IV-C), which the bulk count / retrieve calls see; hash sets take set_insert /
 * set_contains / set_erase and counting tables count_add / count_get (Sec. IV's HashSet
 * and CountingHashTable), on the slots the bulk calls use.
 *
 * Per-element operations are executed by the calling thread alone: it walks the key's
 * probing sequence window by window (W slots each) -- the paper's cooperative group of
 * one thread.  Status conditions (DUPLICATE_KEY, INVALID_KEY, PROBE_LIMIT) are returned
 * and also OR-ed into the table's status word; the pair count is updated with one atomic
 * per converged group of threads.  insert_group / retrieve_group spread one element over
 * a tile of G threads (one window load per tile).  A kernel of many inserts or appends
 * should use insert_uncounted / append_uncounted and add its counts once per thread
 * (add_size, add_counts): the table's pair and key counters are single words, and one
 * atomic on them per element (or per warp) bounds such a kernel.
 */
#ifndef WC_DEVICE_API_CUH_
#define WC_DEVICE_API_CUH_

#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
#include <cooperative_groups/scan.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "wc.h"

namespace wc_dev {

// ---- probing sequence (Sec. IV-B2): outer double hashing over p windows ----------------

// MurmurHash3's 64-bit finalizer "fmix64" (A. Appleby, public domain): an invertible
// avalanche mix.  h1 and h2 of the outer double hashing are its two 32-bit halves.
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// First window w_0 = floor(h1 * p / 2^32) and step = 1 + floor(h2 * (p - 1) / 2^32) of a
// key's sequence w_j = (w_0 + j * step) mod p; requires p >= 2.
__device__ __forceinline__ void probe_init(uint64_t key, uint64_t seed, uint32_t p, uint32_t& w, uint32_t& step) {
  const uint64_t h = fmix64(key ^ seed);
  w = __umulhi(static_cast<uint32_t>(h >> 32), p);
  step = 1u + __umulhi(static_cast<uint32_t>(h), p - 1u);
}

// The same, plus the key's overflow tag (WC_OPT_OVERFLOW_BITS): the low three bits of the
// hash.  w_0 comes from the high half and the step from the top bits of the low half, so
// the tag is close to independent of both.
__device__ __forceinline__ void probe_init(uint64_t key, uint64_t seed, uint32_t p, uint32_t& w, uint32_t& step,
                                           uint32_t& tag) {
  const uint64_t h = fmix64(key ^ seed);
  w = __umulhi(static_cast<uint32_t>(h >> 32), p);
  step = 1u + __umulhi(static_cast<uint32_t>(h), p - 1u);
  tag = static_cast<uint32_t>(h) & 7u;
}

// Overflow bits (WC_OPT_OVERFLOW_BITS): eight per window, byte w of the array (four windows
// per 32-bit word, little-endian) for window w.  An insert of a key with tag g that walks
// past window w sets bit g of byte w; a lookup of such a key may stop at a window without
// the key, without an empty slot and with bit g clear.  Position of that bit in its word:
__device__ __forceinline__ uint32_t overflow_shift(uint32_t w, uint32_t tag) { return ((w & 3u) << 3) | tag; }

// (w + step) mod p for w, step < p < 2^32 (the u32 sum may wrap).
__device__ __forceinline__ uint32_t probe_next(uint32_t w, uint32_t step, uint32_t p) {
  uint32_t x = w + step;
  if (x < w || x >= p) x -= p;
  return x;
}

// ---- slot words of the two single-value layouts (wc.h: wc_table_config) ---------------
// 4+4-byte pairs: one 64-bit word, key in the low half.  8+8-byte pairs: 16 bytes, key
// first.  Key 0 = empty, all ones = tombstone.
template <class K>
struct Slots;

template <>
struct Slots<uint32_t> {
  using V = uint32_t;
  struct Word {
    unsigned long long w;
  };
  static __device__ __forceinline__ Word load(const void* slots, uint64_t i) {
    return Word{__ldcg(static_cast<const unsigned long long*>(slots) + i)};
  }
  static __device__ __forceinline__ uint32_t key(const Word& s) { return static_cast<uint32_t>(s.w); }
  static __device__ __forceinline__ uint32_t val(const Word& s) { return static_cast<uint32_t>(s.w >> 32); }
  static __device__ __forceinline__ bool cas(void* slots, uint64_t i, const Word& old, uint32_t k, uint32_t v) {
    const unsigned long long nw = (static_cast<unsigned long long>(v) << 32) | k;
    return atomicCAS(static_cast<unsigned long long*>(slots) + i, old.w, nw) == old.w;
  }
  static __device__ __forceinline__ bool cas_tomb(void* slots, uint64_t i, const Word& old) {
    return atomicCAS(static_cast<unsigned long long*>(slots) + i, old.w, 0xffffffffull) == old.w;
  }
  static __device__ __forceinline__ void set_val(void* slots, uint64_t i, uint32_t v) {
    atomicExch(reinterpret_cast<unsigned int*>(static_cast<unsigned long long*>(slots) + i) + 1, v);
  }
  static __device__ __forceinline__ void add_val(void* slots, uint64_t i, uint32_t v) {
    atomicAdd(reinterpret_cast<unsigned int*>(static_cast<unsigned long long*>(slots) + i) + 1, v);
  }
};

template <>
struct Slots<unsigned long long> {
  using V = unsigned long long;
  struct Word {
    unsigned long long k, v;
  };
  static __device__ __forceinline__ Word load(const void* slots, uint64_t i) {
    const ulonglong2 x = __ldcg(static_cast<const ulonglong2*>(slots) + i);
    return Word{x.x, x.y};
  }
  static __device__ __forceinline__ unsigned long long key(const Word& s) { return s.k; }
  static __device__ __forceinline__ unsigned long long val(const Word& s) { return s.v; }
  // one 128-bit CAS of the whole pair (sm_90 and later)
  static __device__ __forceinline__ bool cas128(void* slots, uint64_t i, const Word& old, unsigned long long k,
                                                unsigned long long v) {
    void* p = static_cast<char*>(slots) + i * 16;
    unsigned long long ok, ov;
    asm volatile(
        "{\n\t.reg .b128 d, c, s;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 s, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], c, s;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(ok), "=l"(ov)
        : "l"(old.k), "l"(old.v), "l"(k), "l"(v), "l"(p)
        : "memory");
    return ok == old.k && ov == old.v;
  }
  static __device__ __forceinline__ bool cas(void* slots, uint64_t i, const Word& old, unsigned long long k,
                                             unsigned long long v) {
    return cas128(slots, i, old, k, v);
  }
  static __device__ __forceinline__ bool cas_tomb(void* slots, uint64_t i, const Word& old) {
    return cas128(slots, i, old, ~0ull, 0ull);
  }
  static __device__ __forceinline__ void set_val(void* slots, uint64_t i, unsigned long long v) {
    atomicExch(reinterpret_cast<unsigned long long*>(static_cast<char*>(slots) + i * 16) + 1, v);
  }
  static __device__ __forceinline__ void add_val(void* slots, uint64_t i, unsigned long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(static_cast<char*>(slots) + i * 16) + 1, v);
  }
};

template <class K>
__device__ __forceinline__ bool is_sentinel(K k) {
  return k == K(0) || k == K(~K(0));
}

// Pair-count update aggregated over the threads that arrive together.
__device__ __forceinline__ void add_size(const wc_device_view& t, long long d) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  const long long sum = cg::reduce(g, d, cg::plus<long long>());
  if (g.thread_rank() == 0 && sum != 0) atomicAdd(t.size, static_cast<unsigned long long>(sum));
}

__device__ __forceinline__ void raise(const wc_device_view& t, uint32_t f) {
  if (f) atomicOr(t.status, f);
}

// ---- per-element operations (single-value tables) ---------------------------------------

// The W slots of window w, loaded with 32-byte vector loads issued together (a window
// holds a multiple of four 64-bit words for every supported width; windows are aligned).
template <class K, int W>
struct Window {
  using S = Slots<K>;
  static constexpr int kWords = W * static_cast<int>(sizeof(K) == 4 ? 1 : 2);
  unsigned long long u[kWords];
  __device__ __forceinline__ void load(const void* slots, uint32_t w) {
    const unsigned long long* p = static_cast<const unsigned long long*>(slots) + static_cast<uint64_t>(w) * kWords;
#pragma unroll
    for (int i = 0; i < kWords; i += 4)
      asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
                   : "=l"(u[i]), "=l"(u[i + 1]), "=l"(u[i + 2]), "=l"(u[i + 3])
                   : "l"(p + i));
  }
  __device__ __forceinline__ typename S::Word slot(int q) const {
    if constexpr (sizeof(K) == 4) {
      return typename S::Word{u[q]};
    } else {
      return typename S::Word{u[2 * q], u[2 * q + 1]};
    }
  }
};

__device__ __forceinline__ bool overflow_clear(const wc_device_view& t, uint32_t w, uint32_t tag) {
  return t.overflow_bits != nullptr && !((__ldcg(t.overflow_bits + (w >> 2)) >> overflow_shift(w, tag)) & 1u);
}

// kAdd: a counting table -- a stored key gets the value added to its count (no warning),
// an absent one is stored with the value as its count.  kSize = false: a new key leaves
// the table's size to the caller (see insert_uncounted).
template <class K, int W, bool kAdd = false, bool kSize = true>
__device__ uint32_t insert_w(const wc_device_view& t, K key, typename Slots<K>::V value) {
  using S = Slots<K>;
  using Word = typename S::Word;
  uint32_t w0, step, tag;
  probe_init(static_cast<uint64_t>(key), t.seed, t.windows, w0, step, tag);
  uint32_t w = w0, j = 0;
  bool have_t = false;  // first tombstone of the walk, claimed if the key turns out absent
  uint64_t t_slot = 0;
  Word t_word{};
  // Every failed CAS means another insert consumed a free slot, so the retries end.
  while (j < t.windows) {
    Window<K, W> win;
    win.load(t.slots, w);
    const uint64_t base = static_cast<uint64_t>(w) * W;
    bool empty = false;
    int free_q = -1;  // first empty or tombstoned slot of the window
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const K k = S::key(win.slot(q));
      if (k == key) {
        if constexpr (kAdd) {
          S::add_val(t.slots, base + q, value);
          return 0;
        } else {
          S::set_val(t.slots, base + q, value);
          raise(t, WC_FLAG_DUPLICATE_KEY);
          return WC_FLAG_DUPLICATE_KEY;
        }
      }
      const bool is_empty = k == K(0);
      empty |= is_empty;
      if ((is_empty || k == K(~K(0))) && free_q < 0) free_q = q;
    }
    if (empty || j + 1 == t.windows) {  // the key is absent: claim the earliest candidate
      if (have_t) {
        if (S::cas(t.slots, t_slot, t_word, key, value)) break;
        have_t = false;  // the tombstone was taken: walk again from the start
        w = w0;
        j = 0;
        continue;
      }
      if (free_q < 0) {  // last window and nothing free anywhere
        raise(t, WC_FLAG_PROBE_LIMIT);
        return WC_FLAG_PROBE_LIMIT;
      }
      Word fw = win.slot(0);
#pragma unroll
      for (int q = 1; q < W; ++q)
        if (q == free_q) fw = win.slot(q);
      if (S::cas(t.slots, base + free_q, fw, key, value)) break;
      continue;  // lost the slot: read the window again
    }
    if (free_q >= 0 && !have_t) {  // a full window: its free slots are tombstones
      have_t = true;
      t_slot = base + free_q;
      t_word = win.slot(0);
#pragma unroll
      for (int q = 1; q < W; ++q)
        if (q == free_q) t_word = win.slot(q);
    }
    if (t.overflow_bits) atomicOr(t.overflow_bits + (w >> 2), 1u << overflow_shift(w, tag));
    w = probe_next(w, step, t.windows);
    ++j;
  }
  if constexpr (kSize) add_size(t, 1);
  return 0;
}

template <class K, int W>
__device__ bool retrieve_w(const wc_device_view& t, K key, typename Slots<K>::V& value) {
  using S = Slots<K>;
  uint32_t w, step, tag;
  probe_init(static_cast<uint64_t>(key), t.seed, t.windows, w, step, tag);
  for (uint32_t j = 0; j < t.windows; ++j) {
    Window<K, W> win;
    win.load(t.slots, w);
    bool empty = false, hit = false;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const typename S::Word s = win.slot(q);
      if (S::key(s) == key) {
        value = S::val(s);
        hit = true;
      }
      empty |= S::key(s) == K(0);
    }
    if (hit) return true;
    if (empty || overflow_clear(t, w, tag)) return false;
    w = probe_next(w, step, t.windows);
  }
  return false;
}

template <class K, int W>
__device__ bool erase_w(const wc_device_view& t, K key) {
  using S = Slots<K>;
  uint32_t w, step, tag;
  probe_init(static_cast<uint64_t>(key), t.seed, t.windows, w, step, tag);
  for (uint32_t j = 0; j < t.windows; ++j) {
    Window<K, W> win;
    win.load(t.slots, w);
    const uint64_t base = static_cast<uint64_t>(w) * W;
    bool empty = false;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const typename S::Word s = win.slot(q);
      if (S::key(s) == key) {
        // only an erase of the same key can change this slot now: one CAS decides
        const bool ok = S::cas_tomb(t.slots, base + q, s);
        if (ok) add_size(t, -1);
        return ok;
      }
      empty |= S::key(s) == K(0);
    }
    if (empty || overflow_clear(t, w, tag)) return false;
    w = probe_next(w, step, t.windows);
  }
  return false;
}

// ---- group-cooperative operations (Sec. IV-B2: a cooperative group probes each window) --
//
// The G threads of a tile (cooperative_groups::thread_block_tile<G>) serve ONE key together,
// every thread of the tile passing the same key (and value): thread r reads slots
// [r * W/G, (r + 1) * W/G) of each window, votes run over the tile, and one thread claims.
// This is the paper's device-side interface (a group per operation); with G > 1 a window
// is read by G threads with one load request, and the walk's control is shared.

// The S consecutive slot words of one thread (S words of 8 bytes for 4+4-byte pairs, of 16
// for 8+8), loaded with one vector load of up to 32 bytes per instruction.
template <class K, int S>
struct LaneSlots {
  using Sl = Slots<K>;
  static constexpr int kWords = S * static_cast<int>(sizeof(K) == 4 ? 1 : 2);
  unsigned long long u[kWords];
  __device__ __forceinline__ void load(const void* slots, uint64_t first) {
    const unsigned long long* p = static_cast<const unsigned long long*>(slots) + first * (sizeof(K) == 4 ? 1 : 2);
    if constexpr (kWords == 1) {
      asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(u[0]) : "l"(p));
    } else if constexpr (kWords == 2) {
      asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(u[0]), "=l"(u[1]) : "l"(p));
    } else {
#pragma unroll
      for (int i = 0; i < kWords; i += 4)
        asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
                     : "=l"(u[i]), "=l"(u[i + 1]), "=l"(u[i + 2]), "=l"(u[i + 3])
                     : "l"(p + i));
    }
  }
  __device__ __forceinline__ typename Sl::Word slot(int q) const {
    if constexpr (sizeof(K) == 4) {
      return typename Sl::Word{u[q]};
    } else {
      return typename Sl::Word{u[2 * q], u[2 * q + 1]};
    }
  }
};

template <class K, int W, int G>
__device__ bool retrieve_group(const cooperative_groups::thread_block_tile<G>& g, const wc_device_view& t, K key,
                               typename Slots<K>::V& value) {
  using Sl = Slots<K>;
  constexpr int S = W / G;
  static_assert(S >= 1 && W % G == 0, "a window is split evenly over the tile");
  const int r = static_cast<int>(g.thread_rank());
  uint32_t w, step, tag;
  probe_init(static_cast<uint64_t>(key), t.seed, t.windows, w, step, tag);
  for (uint32_t j = 0; j < t.windows; ++j) {
    LaneSlots<K, S> ls;
    ls.load(t.slots, static_cast<uint64_t>(w) * W + r * S);
    int hit_q = -1;
    bool empty = false;
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const K k = Sl::key(ls.slot(q));
      if (k == key && hit_q < 0) hit_q = q;
      empty |= k == K(0);
    }
    const unsigned hm = g.ballot(hit_q >= 0);
    if (hm) {
      typename Sl::V v = 0;
#pragma unroll
      for (int q = 0; q < S; ++q)
        if (q == hit_q) v = Sl::val(ls.slot(q));
      value = g.shfl(v, __ffs(hm) - 1);
      return true;
    }
    if (g.any(empty) || overflow_clear(t, w, tag)) return false;
    w = probe_next(w, step, t.windows);
  }
  return false;
}

template <class K, int W, int G, bool kSize = true>
__device__ uint32_t insert_group(const cooperative_groups::thread_block_tile<G>& g, const wc_device_view& t, K key,
                                 typename Slots<K>::V value) {
  using Sl = Slots<K>;
  using Word = typename Sl::Word;
  constexpr int S = W / G;
  static_assert(S >= 1 && W % G == 0, "a window is split evenly over the tile");
  const int r = static_cast<int>(g.thread_rank());
  uint32_t w0, step, tag;
  probe_init(static_cast<uint64_t>(key), t.seed, t.windows, w0, step, tag);
  uint32_t w = w0, j = 0;
  bool have_t = false;  // first tombstone of the walk (the same on every thread of the tile)
  uint64_t t_slot = 0;
  Word t_word{};
  while (j < t.windows) {
    LaneSlots<K, S> ls;
    const uint64_t mine = static_cast<uint64_t>(w) * W + r * S;
    ls.load(t.slots, mine);
    int match_q = -1, free_q = -1;
    bool empty = false;
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const K k = Sl::key(ls.slot(q));
      if (k == key && match_q < 0) match_q = q;
      const bool is_empty = k == K(0);
      empty |= is_empty;
      if ((is_empty || k == K(~K(0))) && free_q < 0) free_q = q;
    }
    Word fw = ls.slot(0);
#pragma unroll
    for (int q = 1; q < S; ++q)
      if (q == free_q) fw = ls.slot(q);
    const unsigned mm = g.ballot(match_q >= 0);
    if (mm) {  // the key is present: its value is replaced (Sec. IV-B3)
      if (r == __ffs(mm) - 1) Sl::set_val(t.slots, mine + match_q, value);
      if (r == 0) raise(t, WC_FLAG_DUPLICATE_KEY);
      return WC_FLAG_DUPLICATE_KEY;
    }
    const unsigned fm = g.ballot(free_q >= 0);
    if (g.any(empty) || j + 1 == t.windows) {  // absent: claim the earliest candidate
      bool ok = false;
      if (have_t) {
        if (r == 0) ok = Sl::cas(t.slots, t_slot, t_word, key, value);
        if (g.shfl(ok, 0)) break;
        have_t = false;  // the tombstone was taken: walk again from the start
        w = w0;
        j = 0;
        continue;
      }
      if (!fm) {
        if (r == 0) raise(t, WC_FLAG_PROBE_LIMIT);
        return WC_FLAG_PROBE_LIMIT;
      }
      const int src = __ffs(fm) - 1;
      if (r == src) ok = Sl::cas(t.slots, mine + free_q, fw, key, value);
      if (g.shfl(ok, src)) break;
      continue;  // lost the slot: read the window again
    }
    if (fm && !have_t) {  // a full window: its free slots are tombstones
      const int src = __ffs(fm) - 1;
      have_t = true;
      t_slot = g.shfl(mine + static_cast<uint64_t>(free_q < 0 ? 0 : free_q), src);
      if constexpr (sizeof(K) == 4) {
        t_word = Word{g.shfl(fw.w, src)};
      } else {
        t_word = Word{g.shfl(fw.k, src), g.shfl(fw.v, src)};
      }
    }
    if (t.overflow_bits && r == 0) atomicOr(t.overflow_bits + (w >> 2), 1u << overflow_shift(w, tag));
    w = probe_next(w, step, t.windows);
    ++j;
  }
  if constexpr (kSize) {
    if (r == 0) add_size(t, 1);
  }
  return 0;
}

// insert_w / retrieve_w / erase_w take the table's window width W as a template argument
// (it must equal view.window_width): a kernel that knows W keeps one window in registers
// instead of the widest one.  insert / retrieve / erase below pick W at run time.

// Window widths a table of key type K can have (wc.h: window_width).
#define WC_DEV_DISPATCH(K, CALL)                                          \
  if constexpr (sizeof(K) == 4) {                                         \
    switch (t.window_width) {                                             \
      case 4: return CALL(4);                                             \
      case 8: return CALL(8);                                             \
      case 16: return CALL(16);                                           \
      default: return CALL(32);                                           \
    }                                                                     \
  } else {                                                                \
    switch (t.window_width) {                                             \
      case 2: return CALL(2);                                             \
      case 4: return CALL(4);                                             \
      case 8: return CALL(8);                                             \
      default: return CALL(16);                                           \
    }                                                                     \
  }

// Insert (Sec. IV-B2 steps 1-7, IV-B3): walk to the first window holding an empty slot or
// the key; a present key gets its value replaced (WC_FLAG_DUPLICATE_KEY), else the
// earliest free or tombstoned slot of the walk is claimed with one CAS.  Returns the
// WC_FLAG_* bits of this insert (0 = stored as a new key).
template <class K>
__device__ uint32_t insert(const wc_device_view& t, K key, typename Slots<K>::V value) {
  if (is_sentinel(key)) {
    raise(t, WC_FLAG_INVALID_KEY);
    return WC_FLAG_INVALID_KEY;
  }
#define WC_DEV_CALL(Wv) insert_w<K, Wv>(t, key, value)
  WC_DEV_DISPATCH(K, WC_DEV_CALL)
#undef WC_DEV_CALL
}

// insert, except that a new key does not update the table's size: it returns 0 for a new
// key, and the caller adds the number of them with add_size(view, n) -- once per thread or
// warp instead of once per element, which keeps a kernel that inserts many keys off the
// one size counter.  The size is right once every such count has been added.
template <class K>
__device__ uint32_t insert_uncounted(const wc_device_view& t, K key, typename Slots<K>::V value) {
  if (is_sentinel(key)) {
    raise(t, WC_FLAG_INVALID_KEY);
    return WC_FLAG_INVALID_KEY;
  }
#define WC_DEV_CALL(Wv) insert_w<K, Wv, false, false>(t, key, value)
  WC_DEV_DISPATCH(K, WC_DEV_CALL)
#undef WC_DEV_CALL
}

// Retrieve (Sec. IV-B4): the key's value, or false when absent (the walk stops at a window
// holding an empty slot -- or, with overflow bits, a window whose bit for the key's tag is
// clear).
template <class K>
__device__ bool retrieve(const wc_device_view& t, K key, typename Slots<K>::V& value) {
  if (is_sentinel(key)) return false;
#define WC_DEV_CALL(Wv) retrieve_w<K, Wv>(t, key, value)
  WC_DEV_DISPATCH(K, WC_DEV_CALL)
#undef WC_DEV_CALL
}

// Erase (Sec. IV-B5): the key's slot becomes a tombstone; false when the key is absent.
template <class K>
__device__ bool erase(const wc_device_view& t, K key) {
  if (is_sentinel(key)) return false;
#define WC_DEV_CALL(Wv) erase_w<K, Wv>(t, key)
  WC_DEV_DISPATCH(K, WC_DEV_CALL)
#undef WC_DEV_CALL
}

// Counting tables (Sec. IV, CountingHashTable; wc_table_device_view of a WC_COUNTING
// table): count_add adds `weight` to the key's count, storing the key with that count when
// absent (counts wrap at the key width); count_get reads it (false when absent).  Returns
// 0, or WC_FLAG_INVALID_KEY / WC_FLAG_PROBE_LIMIT.
template <class K>
__device__ uint32_t count_add(const wc_device_view& t, K key, typename Slots<K>::V weight) {
  if (is_sentinel(key)) {
    raise(t, WC_FLAG_INVALID_KEY);
    return WC_FLAG_INVALID_KEY;
  }
#define WC_DEV_CALL(Wv) insert_w<K, Wv, true>(t, key, weight)
  WC_DEV_DISPATCH(K, WC_DEV_CALL)
#undef WC_DEV_CALL
}

template <class K>
__device__ bool count_get(const wc_device_view& t, K key, typename Slots<K>::V& count) {
  return retrieve<K>(t, key, count);
}

#undef WC_DEV_DISPATCH

// ---- hash sets (Sec. IV, HashSet): key-only slots ----------------------------------------

// The W keys of window w (4- or 8-byte slots), loaded with 32-byte vector loads issued
// together (a set's window holds a multiple of 32 bytes; windows are aligned).
template <class K, int W>
struct KeyWindow {
  static constexpr int kWords = W * static_cast<int>(sizeof(K)) / 8;
  static_assert(kWords % 4 == 0, "windows of whole 32-byte sectors");
  unsigned long long u[kWords];
  __device__ __forceinline__ void load(const void* slots, uint32_t w) {
    const unsigned long long* p = static_cast<const unsigned long long*>(slots) + static_cast<uint64_t>(w) * kWords;
#pragma unroll
    for (int i = 0; i < kWords; i += 4)
      asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
                   : "=l"(u[i]), "=l"(u[i + 1]), "=l"(u[i + 2]), "=l"(u[i + 3])
                   : "l"(p + i));
  }
  __device__ __forceinline__ K key(int q) const {
    if constexpr (sizeof(K) == 4) {
      return static_cast<uint32_t>(u[q >> 1] >> (32 * (q & 1)));
    } else {
      return u[q];
    }
  }
};

// Key-only CAS (a 4- or 8-byte slot).
template <class K>
__device__ __forceinline__ bool key_cas(void* slots, uint64_t i, K old, K key) {
  if constexpr (sizeof(K) == 4) {
    return atomicCAS(static_cast<unsigned int*>(slots) + i, old, key) == old;
  } else {
    return atomicCAS(static_cast<unsigned long long*>(slots) + i, old, key) == old;
  }
}

template <class K, int W>
__device__ uint32_t set_insert_w(const wc_device_view& t, K key) {
  uint32_t w0, step, tag;
  probe_init(static_cast<uint64_t>(key), t.seed, t.windows, w0, step, tag);
  uint32_t w = w0, j = 0;
  bool have_t = false;  // first tombstone of the walk, claimed if the key turns out absent
  uint64_t t_slot = 0;
  while (j < t.windows) {
    KeyWindow<K, W> win;
    win.load(t.slots, w);
    const uint64_t base = static_cast<uint64_t>(w) * W;
    bool empty = false;
    int free_q = -1;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const K k = win.key(q);
      if (k == key) {
        raise(t, WC_FLAG_DUPLICATE_KEY);
        return WC_FLAG_DUPLICATE_KEY;
      }
      const bool is_empty = k == K(0);
      empty |= is_empty;
      if ((is_empty || k == K(~K(0))) && free_q < 0) free_q = q;
    }
    if (empty || j + 1 == t.windows) {  // absent: claim the earliest candidate
      if (have_t) {
        if (key_cas<K>(t.slots, t_slot, K(~K(0)), key)) break;
        have_t = false;  // the tombstone was taken: walk again from the start
        w = w0;
        j = 0;
        continue;
      }
      if (free_q < 0) {
        raise(t, WC_FLAG_PROBE_LIMIT);
        return WC_FLAG_PROBE_LIMIT;
      }
      K fk = win.key(0);
#pragma unroll
      for (int q = 1; q < W; ++q)
        if (q == free_q) fk = win.key(q);
      if (key_cas<K>(t.slots, base + free_q, fk, key)) break;
      continue;  // lost the slot: read the window again
    }
    if (free_q >= 0 && !have_t) {  // a full window: its free slots are tombstones
      have_t = true;
      t_slot = base + free_q;
    }
    if (t.overflow_bits) atomicOr(t.overflow_bits + (w >> 2), 1u << overflow_shift(w, tag));
    w = probe_next(w, step, t.windows);
    ++j;
  }
  add_size(t, 1);
  return 0;
}

template <class K, int W>
__device__ bool set_find_w(const wc_device_view& t, K key, bool erase) {
  uint32_t w, step, tag;
  probe_init(static_cast<uint64_t>(key), t.seed, t.windows, w, step, tag);
  for (uint32_t j = 0; j < t.windows; ++j) {
    KeyWindow<K, W> win;
    win.load(t.slots, w);
    bool empty = false;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const K k = win.key(q);
      if (k == key) {
        if (!erase) return true;
        // only an erase of the same key can change this slot now: one CAS decides
        const bool ok = key_cas<K>(t.slots, static_cast<uint64_t>(w) * W + q, key, K(~K(0)));
        if (ok) add_size(t, -1);
        return ok;
      }
      empty |= k == K(0);
    }
    if (empty || overflow_clear(t, w, tag)) return false;
    w = probe_next(w, step, t.windows);
  }
  return false;
}

#define WC_SET_DISPATCH(K, CALL)                                          \
  if constexpr (sizeof(K) == 4) {                                         \
    switch (t.window_width) {                                             \
      case 8: return CALL(8);                                             \
      case 16: return CALL(16);                                           \
      default: return CALL(32);                                           \
    }                                                                     \
  } else {                                                                \
    switch (t.window_width) {                                             \
      case 4: return CALL(4);                                             \
      case 8: return CALL(8);                                             \
      case 16: return CALL(16);                                           \
      default: return CALL(32);                                           \
    }                                                                     \
  }

// Set insert (wc_table_device_view of a WC_HASH_SET table): stores an absent key in the
// earliest free or tombstoned slot of its walk; a stored key raises WC_FLAG_DUPLICATE_KEY and
// changes nothing.  Returns the WC_FLAG_* bits (0 = stored).
template <class K>
__device__ uint32_t set_insert(const wc_device_view& t, K key) {
  if (is_sentinel(key)) {
    raise(t, WC_FLAG_INVALID_KEY);
    return WC_FLAG_INVALID_KEY;
  }
#define WC_DEV_CALL(Wv) set_insert_w<K, Wv>(t, key)
  WC_SET_DISPATCH(K, WC_DEV_CALL)
#undef WC_DEV_CALL
}

// Set membership (the lookup's stop rules of Sec. IV-B4).
template <class K>
__device__ bool set_contains(const wc_device_view& t, K key) {
  if (is_sentinel(key)) return false;
#define WC_DEV_CALL(Wv) set_find_w<K, Wv>(t, key, false)
  WC_SET_DISPATCH(K, WC_DEV_CALL)
#undef WC_DEV_CALL
}

// Set erase (Sec. IV-B5): the key's slot becomes a tombstone; false when absent.
template <class K>
__device__ bool set_erase(const wc_device_view& t, K key) {
  if (is_sentinel(key)) return false;
#define WC_DEV_CALL(Wv) set_find_w<K, Wv>(t, key, true)
  WC_SET_DISPATCH(K, WC_DEV_CALL)
#undef WC_DEV_CALL
}

#undef WC_SET_DISPATCH

// ---- per-element appends to a bucket multi-value table (Sec. IV-C) ----------------------
//
// A bucket multi-value table keeps each key once, in a key store of 16-byte slots
// {uint64 key, uint64 list handle}, and the key's values in buckets of a value pool.  With
// a growth strategy the key's buckets have the sizes s_0, s_i = ceil(lambda * s_(i-1)),
// fixed when the table is created, and every bucket after the first starts with an 8-byte
// header holding the handle of the bucket before it (the back reference the bulk count and
// retrieve kernels follow).  The handle packs: bits [0, 28) the key's values, bit 28 "the
// newest bucket has a predecessor", bits [29, 63) the pool offset of the newest bucket, and
// bit 63 "blocked": a thread is making the key's next bucket (zero whenever no append runs,
// so the bulk calls read the same handles).
//
// An append takes the next value number of its key with one CAS on the handle while the
// newest bucket has room.  The value that finds it full (or the key without a bucket) CASes
// the handle to blocked, takes the next bucket of the growth sequence from the pool,
// writes the back reference and its value, and publishes the new handle with a release
// store.  Appends that find the handle blocked back off exponentially; a wait is bounded
// by view.wait_ns (%globaltimer), after which the append gives up with
// WC_FLAG_QUEUE_TIMEOUT.  Appends may run concurrently with each other from any threads
// and kernels; like every insert they must not overlap a lookup of the table (Sec. IV-D).

namespace bl {

constexpr uint64_t kCountBits = 28;
constexpr uint64_t kMaxCount = (1ull << kCountBits) - 1;
constexpr uint64_t kBlocked = 1ull << 63;

__device__ __forceinline__ uint64_t count(uint64_t h) { return h & kMaxCount; }
__device__ __forceinline__ uint64_t offset(uint64_t h) { return (h & ~kBlocked) >> (kCountBits + 1); }
__device__ __forceinline__ uint64_t make(uint64_t off, uint64_t cnt, bool prev) {
  return (off << (kCountBits + 1)) | (static_cast<uint64_t>(prev) << kCountBits) | cnt;
}

// Values held by buckets 0..i, and their pool elements (headers and padding included).
__device__ __forceinline__ uint64_t cum_size(const wc_device_view& t, int64_t i) {
  if (i < 0) return 0;
  return t.growth == 1 ? static_cast<uint64_t>(i + 1) * t.bucket_size : t.bucket_cum_size[i];
}
__device__ __forceinline__ uint64_t cum_foot(const wc_device_view& t, int64_t i) {
  if (i < 0) return 0;
  return t.growth == 1 ? t.bucket_foot0 + static_cast<uint64_t>(i) * t.bucket_foot : t.bucket_cum_foot[i];
}
// The bucket holding value number v.
__device__ __forceinline__ int64_t bucket_of(const wc_device_view& t, uint64_t v) {
  if (t.growth == 1) return static_cast<int64_t>(v / t.bucket_size);
  uint32_t lo = 0, hi = t.bucket_count - 1;  // first i with cum_size(i) > v
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (t.bucket_cum_size[mid] > v) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t x;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(x));
  return x;
}

__device__ __forceinline__ uint64_t load_relaxed(const unsigned long long* p) {
  uint64_t x;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(x) : "l"(p) : "memory");
  return x;
}

__device__ __forceinline__ void store_release(unsigned long long* p, uint64_t x) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(x) : "memory");
}

// `n` elements of the pool cursor for every converged thread at once: one atomic per
// coalesced group (the threads that reach the allocation together), each thread's share by
// an exclusive scan -- hot appends would otherwise serialise on the one cursor.
__device__ __forceinline__ uint64_t pool_alloc(const wc_device_view& t, uint64_t n) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  const unsigned long long before = cg::exclusive_scan(g, static_cast<unsigned long long>(n));
  unsigned long long base = 0;
  if (g.thread_rank() == g.size() - 1) base = atomicAdd(t.pool_cursor, before + n);
  base = g.shfl(base, g.size() - 1);
  return base + before;
}

// Distinct-key count update aggregated over the converged threads.
__device__ __forceinline__ void add_keys(const wc_device_view& t, unsigned long long d) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  const unsigned long long sum = cg::reduce(g, d, cg::plus<unsigned long long>());
  if (g.thread_rank() == 0 && sum != 0) atomicAdd(t.num_keys, sum);
}

// The key's slot in the key store (windows of W 16-byte slots, the probing sequence of
// the bulk calls), inserted with handle 0 (no bucket) when absent: the earliest empty or
// tombstoned slot of the walk, claimed with one 128-bit CAS.  -1 with the flag set when
// the key store is full.
// new_keys != nullptr: a key it stores is counted there instead of in the table.
template <int W>
__device__ int64_t key_slot(const wc_device_view& t, unsigned long long key, uint32_t& flags,
                            unsigned long long* new_keys = nullptr) {
  using S = Slots<unsigned long long>;
  using Word = typename S::Word;
  uint32_t w0, step;
  probe_init(key, t.seed, t.windows, w0, step);
  uint32_t w = w0, j = 0;
  bool have_t = false;
  uint64_t t_slot = 0;
  Word t_word{};
  while (j < t.windows) {
    Window<unsigned long long, W> win;
    win.load(t.slots, w);
    const uint64_t base = static_cast<uint64_t>(w) * W;
    bool empty = false;
    int free_q = -1;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const unsigned long long k = S::key(win.slot(q));
      if (k == key) return static_cast<int64_t>(base + q);
      const bool is_empty = k == 0ull;
      empty |= is_empty;
      if ((is_empty || k == ~0ull) && free_q < 0) free_q = q;
    }
    if (empty || j + 1 == t.windows) {
      if (have_t) {
        if (S::cas(t.slots, t_slot, t_word, key, 0ull)) {
          if (new_keys) ++*new_keys;
          else add_keys(t, 1ull);
          return static_cast<int64_t>(t_slot);
        }
        have_t = false;  // the tombstone was taken: walk again from the start
        w = w0;
        j = 0;
        continue;
      }
      if (free_q < 0) {
        flags |= WC_FLAG_PROBE_LIMIT;
        return -1;
      }
      Word fw = win.slot(0);
#pragma unroll
      for (int q = 1; q < W; ++q)
        if (q == free_q) fw = win.slot(q);
      if (S::cas(t.slots, base + free_q, fw, key, 0ull)) {
        if (new_keys) ++*new_keys;
        else add_keys(t, 1ull);
        return static_cast<int64_t>(base + free_q);
      }
      continue;  // the slot was taken (maybe by this key): read the window again
    }
    if (free_q >= 0 && !have_t) {
      have_t = true;
      t_slot = base + free_q;
      t_word = win.slot(0);
#pragma unroll
      for (int q = 1; q < W; ++q)
        if (q == free_q) t_word = win.slot(q);
    }
    w = probe_next(w, step, t.windows);
    ++j;
  }
  flags |= WC_FLAG_PROBE_LIMIT;
  return -1;
}

template <class V>
__device__ __forceinline__ void put(const wc_device_view& t, uint64_t index, V value) {
  static_cast<V*>(t.pool)[index] = value;
}

// Append value number c (the caller holds it) at its place in the key's bucket b whose
// pool start is `start`.
template <class V>
__device__ __forceinline__ void put_value(const wc_device_view& t, uint64_t start, int64_t b, uint64_t c, V value) {
  constexpr uint64_t hdr = 8 / sizeof(V);  // header elements of a non-first bucket
  put<V>(t, start + (b > 0 ? hdr : 0) + (c - cum_size(t, b - 1)), value);
}

// Counts of appends that leave the table's counters to their caller (append_uncounted).
struct Counts {
  unsigned long long values = 0, keys = 0;
};

// counts != nullptr: the appended value and a new key are counted there, not in the table.
template <int W, class V>
__device__ uint32_t append_w(const wc_device_view& t, unsigned long long key, V value, Counts* counts = nullptr) {
  uint32_t flags = 0;
  const int64_t slot = key_slot<W>(t, key, flags, counts ? &counts->keys : nullptr);
  if (slot < 0) {
    atomicOr(t.status, flags);
    return flags;
  }
  unsigned long long* handle = reinterpret_cast<unsigned long long*>(static_cast<char*>(t.slots) + slot * 16 + 8);
  const uint64_t limit = t.wait_ns ? t.wait_ns : 1000000000ull;
  uint64_t t0 = 0;
  uint32_t pause = 32;
  for (uint32_t it = 0;; ++it) {
    const uint64_t h = load_relaxed(handle);
    const uint64_t c = count(h);
    const bool blocked = (h & kBlocked) != 0;
    if (!blocked && c >= kMaxCount) {
      flags |= WC_FLAG_COUNT_OVERFLOW;
      break;
    }
    const int64_t newest = c == 0 ? -1 : bucket_of(t, c - 1);
    if (!blocked && newest >= 0 && c < cum_size(t, newest)) {
      // room in the newest bucket: take value number c
      if (atomicCAS(handle, h, h + 1) == h) {
        put_value<V>(t, offset(h), newest, c, value);
        if (counts) ++counts->values;
        else add_size(t, 1);
        return 0;
      }
    } else if (!blocked) {
      // the newest bucket is full (or there is none): make bucket newest + 1
      if (atomicCAS(handle, h, h | kBlocked) == h) {
        const int64_t b = newest + 1;
        const uint64_t foot = cum_foot(t, b) - cum_foot(t, b - 1);
        const uint64_t off = pool_alloc(t, foot);
        if (off + foot > t.pool_capacity) {
          store_release(handle, h);  // unblock, unchanged
          flags |= WC_FLAG_POOL_EXHAUSTED;
          break;
        }
        if (b > 0) {
          // back reference: the handle of the bucket before, as the bulk layout has it
          *reinterpret_cast<unsigned long long*>(static_cast<char*>(t.pool) + off * sizeof(V)) = h;
        }
        put_value<V>(t, off, b, c, value);
        store_release(handle, make(off, c + 1, b > 0));
        if (counts) ++counts->values;
        else add_size(t, 1);
        return 0;
      }
    } else {
      // another thread is making the next bucket: back off, at most `limit` in all
      if (t0 == 0) {
        t0 = now_ns();
      } else if (now_ns() - t0 > limit) {
        flags |= WC_FLAG_QUEUE_TIMEOUT;
        break;
      }
      __nanosleep(pause);
      pause = pause < 4096 ? pause * 2 : pause;
    }
    // a lost CAS means another append went ahead; the same time bound covers the retries
    if ((it & 63) == 63) {
      if (t0 == 0) t0 = now_ns();
      else if (now_ns() - t0 > limit) {
        flags |= WC_FLAG_QUEUE_TIMEOUT;
        break;
      }
    }
  }
  atomicOr(t.status, flags);
  return flags;
}

}  // namespace bl

// Append (key, value) to a bucket multi-value table with a growth strategy (wc_device_view
// from wc_table_device_view): K is the table's key type (uint32_t or unsigned long long),
// V its value type.  Returns 0, or the WC_FLAG_* bits of a failed append (INVALID_KEY,
// PROBE_LIMIT, POOL_EXHAUSTED, COUNT_OVERFLOW, QUEUE_TIMEOUT), also OR-ed into the table's
// status word.  The bulk count_values / retrieve_multi calls see the appended values.
template <class K, class V>
__device__ uint32_t append(const wc_device_view& t, K key, V value) {
  if (is_sentinel(key)) {
    atomicOr(t.status, static_cast<uint32_t>(WC_FLAG_INVALID_KEY));
    return WC_FLAG_INVALID_KEY;
  }
  const unsigned long long k = static_cast<unsigned long long>(key);  // keys are stored as 8 bytes
  switch (t.window_width) {
    case 2: return bl::append_w<2, V>(t, k, value);
    case 4: return bl::append_w<4, V>(t, k, value);
    default: return bl::append_w<8, V>(t, k, value);
  }
}

// append, except that the table's pair and key counters are left to the caller: the value
// and a new key are counted in c, and add_counts(view, c) adds them -- once per thread
// instead of once per element, which keeps a kernel of many appends off the two counters.
template <class K, class V>
__device__ uint32_t append_uncounted(const wc_device_view& t, K key, V value, bl::Counts& c) {
  if (is_sentinel(key)) {
    atomicOr(t.status, static_cast<uint32_t>(WC_FLAG_INVALID_KEY));
    return WC_FLAG_INVALID_KEY;
  }
  const unsigned long long k = static_cast<unsigned long long>(key);
  switch (t.window_width) {
    case 2: return bl::append_w<2, V>(t, k, value, &c);
    case 4: return bl::append_w<4, V>(t, k, value, &c);
    default: return bl::append_w<8, V>(t, k, value, &c);
  }
}

__device__ __forceinline__ void add_counts(const wc_device_view& t, const bl::Counts& c) {
  add_size(t, static_cast<long long>(c.values));
  bl::add_keys(t, c.keys);
}

// ---- higher-order bulk calls ----------------------------------------------------------

template <class K, class F>
__global__ void for_each_kernel(wc_device_view t, const K* __restrict__ keys, uint64_t n, F f) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    typename Slots<K>::V v;
    if (retrieve<K>(t, keys[i], v)) f(keys[i], v, i);
  }
}

template <class K, class F>
__global__ void for_all_kernel(wc_device_view t, F f) {
  using S = Slots<K>;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < t.capacity; i += stride) {
    const typename S::Word s = S::load(t.slots, i);
    if (!is_sentinel(S::key(s))) f(S::key(s), S::val(s), i);
  }
}

// for_each(keys, callback): callback(key, value, i) for every keys[i] found, on `stream`
// (asynchronous).  K = uint32_t for 4+4-byte tables, unsigned long long for 8+8.
template <class K, class F>
cudaError_t for_each(const wc_device_view& t, const K* d_keys, uint64_t n, F f, cudaStream_t stream = 0) {
  if (n == 0) return cudaSuccess;
  if (t.key_bytes != static_cast<int32_t>(sizeof(K))) return cudaErrorInvalidValue;
  const uint64_t blocks = (n + 255) / 256;
  for_each_kernel<K, F><<<static_cast<unsigned>(blocks < 65536 ? blocks : 65536), 256, 0, stream>>>(t, d_keys, n, f);
  return cudaGetLastError();
}

// for_all(callback): callback(key, value, slot) for every stored pair (asynchronous).
template <class K, class F>
cudaError_t for_all(const wc_device_view& t, F f, cudaStream_t stream = 0) {
  if (t.key_bytes != static_cast<int32_t>(sizeof(K))) return cudaErrorInvalidValue;
  const uint64_t blocks = (t.capacity + 255) / 256;
  for_all_kernel<K, F><<<static_cast<unsigned>(blocks < 65536 ? blocks : 65536), 256, 0, stream>>>(t, f);
  return cudaGetLastError();
}

}  // namespace wc_dev

#endif /* WC_DEVICE_API_CUH_ */
