// Single-value bulk kernels: insert, retrieve, erase (Sec. IV-B2 .. IV-B5).
//
// One group of G lanes serves one key at a time (the cooperative group of Sec. IV-B2).
// Every warp runs a warp-uniform loop; one trip probes ONE window for every group of
// the warp that holds a key, so all of the warp's window loads are in flight together.
// A group that finishes a key takes the next input position of its warp's range in the
// same trip (take_next), which keeps every lane busy until the range is exhausted
// instead of idling behind the warp's longest probe sequence.
//
// Insert claims the earliest candidate slot of the key's probing sequence (steps 1-7 of
// Sec. IV-B2).  A tombstone is a candidate (Sec. IV-B5), but probing continues past it
// to the first window holding an empty slot or the key itself, so a key erased and
// inserted again can never be stored twice; with no tombstones in the table this is
// exactly the paper's insertion.  Retrieval stops at the key or at the first window
// that holds an empty slot (valid because a slot never returns to empty except by a
// clear, Sec. IV-B4) -- or, in tables with overflow bits, at a window without an empty
// slot whose bit for the key's tag is clear (no key of that tag walked past it).
#pragma once

#include <type_traits>

#include "wc_device.cuh"
#include "wc_internal.h"

namespace wc {

template <class L, int G, int S>
struct SvLane {
  static constexpr int W = G * S;
  int lane, r, gbase;
  __device__ SvLane() {
    lane = threadIdx.x & 31;
    r = lane & (G - 1);
    gbase = lane - r;
  }
};

// Masks of one lane's S slots: bit i set if slot i holds the key / is empty / is a
// tombstone.
template <class L, int S>
__device__ __forceinline__ void classify(const typename L::Slot (&s)[S], typename L::Key k, uint32_t& mm,
                                         uint32_t& me, uint32_t& mt) {
  mm = me = mt = 0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const typename L::Key kk = L::key(s[i]);
    mm |= static_cast<uint32_t>(kk == k) << i;
    me |= static_cast<uint32_t>(kk == L::kEmpty) << i;
    mt |= static_cast<uint32_t>(kk == L::kTomb) << i;
  }
}

// Steps of a window walk (a window of H steps of SW slots): offset of step h in the
// window, whether h is its last step, whether steps follow.  With H == 1 they are the
// constants 0 / true / false, so a whole-window walk carries no step bookkeeping.
template <int H>
struct Steps {
  static __device__ __forceinline__ uint32_t offset(uint32_t h, int SW) {
    if constexpr (H == 1) {
      return 0;
    } else {
      return h * static_cast<uint32_t>(SW);
    }
  }
  static __device__ __forceinline__ bool last(uint32_t h) {
    if constexpr (H == 1) {
      return true;
    } else {
      return h + 1 == static_cast<uint32_t>(H);
    }
  }
  static __device__ __forceinline__ bool more(uint32_t h) {
    if constexpr (H == 1) {
      return false;
    } else {
      return h + 1 < static_cast<uint32_t>(H);
    }
  }
};

template <class K>
__device__ __forceinline__ bool is_sentinel(K k) {
  return k == K(0) || k == K(~K(0));
}

// Range of input positions of this warp: [begin, end).
__device__ __forceinline__ void warp_range(uint64_t n, uint64_t per_warp, uint64_t& begin, uint64_t& end) {
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  begin = warp * per_warp;
  end = begin + per_warp < n ? begin + per_warp : n;
}

// Where a warp's input positions come from.  With counter == nullptr the warp owns the
// static range [next, end).  Otherwise warps pull `chunk` positions at a time from a
// global counter, so the whole grid sweeps the input front to back -- a batch sorted by
// table region is then probed region by region, with the active regions held in L2.
struct StridedChunks {};

struct RangeSrc {
  uint64_t next, end, n;
  unsigned long long* counter;
  uint32_t chunk;
  bool done;
  bool fresh;  // [next, end) is a new range whose inputs have not been prefetched yet
  uint64_t base = 0, stride = 0;  // strided mode: current chunk start, chunks of all warps
  __device__ RangeSrc(uint64_t n_, uint64_t per_warp, unsigned long long* counter_, uint32_t chunk_)
      : n(n_), counter(counter_), chunk(chunk_), done(false), fresh(true) {
    if (counter == nullptr) {
      warp_range(n, per_warp, next, end);
    } else {
      next = end = 0;
    }
  }
  // A fixed range [begin, end) (one tile of the batched executor).
  __device__ RangeSrc(uint64_t begin, uint64_t end_)
      : next(begin), end(end_), n(end_), counter(nullptr), chunk(0), done(false), fresh(true) {}
  // Warp w takes chunks w, w + warps, w + 2 * warps, ... of `chunk_` positions: spreads
  // inputs whose cost depends on their position (a sorted query range whose first part
  // holds every present key) over all warps without a shared counter.
  __device__ RangeSrc(StridedChunks, uint64_t n_, uint32_t chunk_)
      : n(n_), counter(nullptr), chunk(chunk_), done(false), fresh(true) {
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    stride = (static_cast<uint64_t>(gridDim.x) * blockDim.x >> 5) * chunk;
    base = warp * chunk;
    next = base < n ? base : n;
    end = base + chunk < n ? base + chunk : n;
  }
  // Warp-uniform: true while positions are left in [next, end) or can be pulled.
  __device__ __forceinline__ bool ensure() {
    if (next < end) return true;
    if (stride != 0) {
      base += stride;
      if (base >= n) return false;
      next = base;
      end = base + chunk < n ? base + chunk : n;
      fresh = true;
      return true;
    }
    if (counter == nullptr || done) return false;
    unsigned long long c = 0;
    if ((threadIdx.x & 31) == 0) c = atomicAdd(counter, static_cast<unsigned long long>(chunk));
    c = __shfl_sync(kFull, c, 0);
    if (c >= n) {
      done = true;
      return false;
    }
    next = c;
    end = c + chunk < n ? c + chunk : n;
    fresh = true;
    return true;
  }
};

// The warp's next 64 input elements, prefetched into registers with coalesced loads
// (lane l holds elements base + l and base + 32 + l).  Groups receive their key by
// shuffle, so the input load is off the per-key critical path; the second half is
// reloaded while the first is being consumed.
template <class T>
struct Feed {
  T b0, b1;
  uint64_t base, lim;
  const T* __restrict__ src;
  __device__ __forceinline__ void load(const T* p, uint64_t start, uint64_t end) {
    const uint64_t lane = threadIdx.x & 31;
    src = p;
    base = start;
    lim = end;
    b0 = start + lane < end ? ldg_stream(p + start + lane) : T(0);
    b1 = start + 32 + lane < end ? ldg_stream(p + start + 32 + lane) : T(0);
  }
  // Element at `pos` (valid lanes); every lane must call.
  __device__ __forceinline__ T get(uint64_t pos, bool valid) const {
    const uint32_t o = valid ? static_cast<uint32_t>(pos - base) : 0u;
    const T x0 = __shfl_sync(kFull, b0, o & 31);
    const T x1 = __shfl_sync(kFull, b1, o & 31);
    return o < 32 ? x0 : x1;
  }
  // After positions up to `next` were handed out (warp-uniform).
  __device__ __forceinline__ void advance(uint64_t next) {
    if (next - base >= 32) {
      const uint64_t lane = threadIdx.x & 31;
      b0 = b1;
      base += 32;
      b1 = base + 32 + lane < lim ? ldg_stream(src + base + 32 + lane) : T(0);
    }
  }
};

// Feed that also groups equal keys inside each 32-element block of the warp's input (the
// warp-level aggregation of duplicate queries, __match_any_sync): next to its element,
// lane l keeps the mask of the block's lanes holding the same key if l is the lowest of
// them (the leader), 0 if a lower lane holds it (a follower), and 1 << l for a sentinel
// (never grouped).  Only leaders probe; a leader writes the result of every follower.
template <class T>
struct DedupFeed : Feed<T> {
  uint32_t m0, m1;
  static __device__ __forceinline__ uint32_t group(T x) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t peers = __match_any_sync(kFull, x);
    if (x == T(0) || x == T(~T(0))) return 1u << lane;
    return static_cast<uint32_t>(__ffs(peers) - 1) == lane ? peers : 0u;
  }
  __device__ __forceinline__ void load(const T* p, uint64_t start, uint64_t end) {
    Feed<T>::load(p, start, end);
    m0 = group(this->b0);
    m1 = group(this->b1);
  }
  // Group mask of the element at `pos` (valid lanes); every lane must call.
  __device__ __forceinline__ uint32_t mask(uint64_t pos, bool valid) const {
    const uint32_t o = valid ? static_cast<uint32_t>(pos - this->base) : 0u;
    const uint32_t x0 = __shfl_sync(kFull, m0, o & 31);
    const uint32_t x1 = __shfl_sync(kFull, m1, o & 31);
    return o < 32 ? x0 : x1;
  }
  __device__ __forceinline__ void advance(uint64_t next) {
    if (next - this->base >= 32) {
      Feed<T>::advance(next);
      m0 = m1;
      m1 = group(this->b1);
    }
  }
};

// ---------------------------------------------------------------------------------------
// retrieve: out[i] = value of keys[i] or NOT_FOUND; found[i] = 1/0 (Sec. IV-B4).
// Emit is called by one lane per finished query: emit(pos, hit, slot, index) -- index is
// the matching slot's position in the table (struct-of-arrays layouts read the value
// there; 0 for other layouts).  kDedup: equal queries of a 32-element block are probed
// once, the result emitted for each of their positions (skewed query streams).
template <class L, int G, int S, class Emit, class KIn = typename L::Key, bool kDedup = false, int H = 1>
__device__ __forceinline__ void sv_retrieve_range(const TableDesc& t, const KIn* __restrict__ keys, RangeSrc& src,
                                                  Emit& emit, uint32_t& flags) {
  using Slot = typename L::Slot;
  using Key = typename L::Key;
  const SvLane<L, G, S> ln;
  constexpr int SW = G * S;  // slots of one step; a window is walked in H steps
  constexpr int W = SW * H;
  const Slot* slots = static_cast<const Slot*>(t.slots);
  bool act = false;
  uint64_t pos = 0;
  Key k = 0;
  uint32_t w = 0, step = 0, j = 0, tag = 0, h = 0;
  uint32_t fm = 0;  // kDedup: group mask of the query being probed
  std::conditional_t<kDedup, DedupFeed<KIn>, Feed<KIn>> fk;
  while (true) {
    const bool more = src.ensure();
    if (more && src.fresh) {
      fk.load(keys, src.next, src.end);
      src.fresh = false;
    }
    uint64_t np = 0;
    const bool got = more && take_next(!act, ln.r, ln.gbase, src.next, src.end, np);
    const KIn kin = fk.get(np, got);
    if constexpr (kDedup) {
      const uint32_t m = fk.mask(np, got);  // a shuffle: every lane calls
      if (got) fm = m;
    }
    if (more) fk.advance(src.next);
    if (got) {
      pos = np;
      k = static_cast<Key>(kin);
      if (is_sentinel(kin)) {
        flags |= kFlagInvalid;
        if (ln.r == 0) emit(pos, false, Slot{}, 0ull);
      } else if (!kDedup || fm != 0) {  // a follower is answered by its leader
        act = true;
        j = 0;
        h = 0;
        probe_init(static_cast<uint64_t>(k), t.seed, t.p, w, step, tag);
      }
    }
    if (__ballot_sync(kFull, act) == 0) {
      if (!more) break;
      continue;
    }
    Slot s[S];
    uint32_t mm = 0, me = 0, mt = 0;
    if (act) {
      load_slots<L, S>(slots + static_cast<uint64_t>(w) * W + Steps<H>::offset(h, SW) + ln.r * S, s);
      classify<L, S>(s, k, mm, me, mt);
    }
    const uint32_t bm = group_vote<G>(mm != 0, ln.gbase);
    const uint32_t be = group_vote<G>(me != 0, ln.gbase);
    // The overflow bit only matters for a window without the key and without an empty
    // slot, so its word is read only then.  Reading it in the same trip as the window
    // (to save the dependent round trip) measured slower: the lookup is bound by the L2's
    // request rate, and every trip would then make two requests.
    uint32_t fw = 0xffffffffu;
    if (t.ovf != nullptr && act && !bm && !be && Steps<H>::last(h)) fw = ovf_word(t.ovf, w);
    Slot hit = pick<L, S>(s, mm ? __ffs(mm) - 1 : 0);
    if constexpr (G > 1) hit = L::shfl(hit, ln.gbase + (bm ? __ffs(bm) - 1 : 0));
    uint64_t hidx = 0;
    if constexpr (L::kSoA) {
      hidx = static_cast<uint64_t>(w) * W + Steps<H>::offset(h, SW) + ln.r * S + (mm ? __ffs(mm) - 1 : 0);
      if constexpr (G > 1) hidx = __shfl_sync(kFull, hidx, ln.gbase + (bm ? __ffs(bm) - 1 : 0));
    }
    if constexpr (kDedup) {
      if (act) {
        // an empty slot ends the walk wherever it is; the rest of a window follows its
        // first part; a whole window without either ends it through its overflow bit
        const bool next_part = !bm && !be && Steps<H>::more(h);
        const bool done = !next_part && (bm || be || !ovf_bit(fw, w, tag) || ++j >= t.p);
        if (done && ln.r == 0) {
          emit(pos, bm != 0, hit, hidx);
          const uint64_t first = pos - static_cast<uint64_t>(__ffs(fm) - 1);  // the leader is the lowest lane
          for (uint32_t f = fm & (fm - 1); f != 0; f &= f - 1) emit(first + (__ffs(f) - 1), bm != 0, hit, hidx);
        }
        if (done) {
          act = false;
        } else if (next_part) {
          ++h;
        } else {
          h = 0;
          w = probe_next(w, step, t.p);
        }
      }
    } else if (act) {
      if (bm) {
        if (ln.r == 0) emit(pos, true, hit, hidx);
        act = false;
      } else if (!be && Steps<H>::more(h)) {
        ++h;  // the rest of this window
      } else if (be || !ovf_bit(fw, w, tag) || ++j >= t.p) {
        if (ln.r == 0) emit(pos, false, hit, hidx);
        act = false;
      } else {
        h = 0;
        w = probe_next(w, step, t.p);
      }
    }
  }
}

// The same lookup with K keys per group in flight: every trip, each group loads the
// windows of up to K keys at once (all of a warp's loads are issued before any is used), so
// a warp keeps K times as many random window reads in flight.  A lookup is bound by how
// many reads are in flight against the memory latency, not by the instructions of a trip.
// Each of a group's K keys is an independent probe with the retrieve's own stop rules.
template <class L, int G, int S, int K, class Emit, class KIn = typename L::Key, int H = 1>
__device__ __forceinline__ void sv_retrieve_range_k(const TableDesc& t, const KIn* __restrict__ keys, RangeSrc& src,
                                                    Emit& emit, uint32_t& flags) {
  using Slot = typename L::Slot;
  using Key = typename L::Key;
  const SvLane<L, G, S> ln;
  constexpr int SW = G * S;  // slots of one step; a window is walked in H steps
  constexpr int W = SW * H;
  const Slot* slots = static_cast<const Slot*>(t.slots);
  bool act[K];
  uint64_t pos[K];
  Key k[K];
  uint32_t w[K], step[K], j[K], tag[K], h[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    act[q] = false;
    pos[q] = 0;
    k[q] = 0;
    w[q] = step[q] = j[q] = tag[q] = h[q] = 0;
  }
  Feed<KIn> fk;
  while (true) {
    const bool more = src.ensure();
    if (more && src.fresh) {
      fk.load(keys, src.next, src.end);
      src.fresh = false;
    }
    bool any = false;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      uint64_t np = 0;
      const bool got = more && take_next(!act[q], ln.r, ln.gbase, src.next, src.end, np);
      const KIn kin = fk.get(np, got);
      if (more) fk.advance(src.next);
      if (got) {
        pos[q] = np;
        k[q] = static_cast<Key>(kin);
        if (is_sentinel(kin)) {
          flags |= kFlagInvalid;
          if (ln.r == 0) emit(pos[q], false, Slot{}, 0ull);
        } else {
          act[q] = true;
          j[q] = 0;
          h[q] = 0;
          probe_init(static_cast<uint64_t>(k[q]), t.seed, t.p, w[q], step[q], tag[q]);
        }
      }
      any |= act[q];
    }
    if (__ballot_sync(kFull, any) == 0) {
      if (!more) break;
      continue;
    }
    Slot s[K][S];
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (act[q]) load_slots<L, S>(slots + static_cast<uint64_t>(w[q]) * W + Steps<H>::offset(h[q], SW) + ln.r * S, s[q]);
#pragma unroll
    for (int q = 0; q < K; ++q) {
      uint32_t mm = 0, me = 0, mt = 0;
      if (act[q]) classify<L, S>(s[q], k[q], mm, me, mt);
      const uint32_t bm = group_vote<G>(mm != 0, ln.gbase);
      const uint32_t be = group_vote<G>(me != 0, ln.gbase);
      uint32_t fw = 0xffffffffu;
      if (t.ovf != nullptr && act[q] && !bm && !be && Steps<H>::last(h[q])) fw = ovf_word(t.ovf, w[q]);
      Slot hit = pick<L, S>(s[q], mm ? __ffs(mm) - 1 : 0);
      if constexpr (G > 1) hit = L::shfl(hit, ln.gbase + (bm ? __ffs(bm) - 1 : 0));
      uint64_t hidx = 0;
      if constexpr (L::kSoA) {
        hidx = static_cast<uint64_t>(w[q]) * W + Steps<H>::offset(h[q], SW) + ln.r * S + (mm ? __ffs(mm) - 1 : 0);
        if constexpr (G > 1) hidx = __shfl_sync(kFull, hidx, ln.gbase + (bm ? __ffs(bm) - 1 : 0));
      }
      if (act[q]) {
        if (bm) {
          if (ln.r == 0) emit(pos[q], true, hit, hidx);
          act[q] = false;
        } else if (!be && Steps<H>::more(h[q])) {
          ++h[q];  // the rest of this window
        } else if (be || !ovf_bit(fw, w[q], tag[q]) || ++j[q] >= t.p) {
          if (ln.r == 0) emit(pos[q], false, hit, hidx);
          act[q] = false;
        } else {
          h[q] = 0;
          w[q] = probe_next(w[q], step[q], t.p);
        }
      }
    }
  }
}

template <class L>
struct EmitValue {
  typename L::Val* __restrict__ out;
  uint8_t* __restrict__ found;
  const void* vals;  // struct-of-arrays value array (else unused)
  __device__ void operator()(uint64_t pos, bool hit, const typename L::Slot& s, uint64_t idx) const {
    if (out) out[pos] = hit ? slot_value<L>(s, vals, idx) : L::kNotFound;  // no output: membership only
    if (found) found[pos] = hit ? 1 : 0;
  }
};

// Packed 8-byte slots with at most 32 bytes of the window per lane fit six 256-thread
// blocks per SM (40 registers) without spilling; more warps in flight hide more of the
// random-read latency.  Wider per-lane loads keep the compiler's choice.
template <class L, int S>
constexpr int retrieve_min_blocks() {
  return (L::kWords == 1 && sizeof(typename L::Key) == 4 && S <= 4) ? 6 : 1;
}

template <class L, int G, int S, int H = 1>
__global__ void __launch_bounds__(256, retrieve_min_blocks<L, S>()) k_sv_retrieve(TableDesc t, const typename L::Key* __restrict__ keys, uint64_t n,
                                                     uint64_t per_warp, typename L::Val* __restrict__ out,
                                                     uint8_t* __restrict__ found) {
  RangeSrc src(n, per_warp, nullptr, 0);
  if (src.next >= src.end) return;
  uint32_t flags = 0;
  EmitValue<L> emit{out, found, t.vals};
  sv_retrieve_range<L, G, S, EmitValue<L>, typename L::Key, false, H>(t, keys, src, emit, flags);
  flush_flags(t.status, flags);
}

// The same with two keys per group in flight (launch keys_in_flight = 2).
template <class L, int G, int S, int H = 1>
__global__ void __launch_bounds__(256) k_sv_retrieve2(TableDesc t, const typename L::Key* __restrict__ keys, uint64_t n,
                                                      uint64_t per_warp, typename L::Val* __restrict__ out,
                                                      uint8_t* __restrict__ found) {
  RangeSrc src(n, per_warp, nullptr, 0);
  if (src.next >= src.end) return;
  uint32_t flags = 0;
  EmitValue<L> emit{out, found, t.vals};
  sv_retrieve_range_k<L, G, S, 2, EmitValue<L>, typename L::Key, H>(t, keys, src, emit, flags);
  flush_flags(t.status, flags);
}

// The same with equal queries of each 32-element block probed once (WC_SCHEME_DEDUP).
template <class L, int G, int S, int H = 1>
__global__ void __launch_bounds__(256) k_sv_retrieve_dedup(TableDesc t, const typename L::Key* __restrict__ keys,
                                                           uint64_t n, uint64_t per_warp,
                                                           typename L::Val* __restrict__ out,
                                                           uint8_t* __restrict__ found) {
  RangeSrc src(n, per_warp, nullptr, 0);
  if (src.next >= src.end) return;
  uint32_t flags = 0;
  EmitValue<L> emit{out, found, t.vals};
  sv_retrieve_range<L, G, S, EmitValue<L>, typename L::Key, true, H>(t, keys, src, emit, flags);
  flush_flags(t.status, flags);
}

// Retrieve over a batch split by table region (the blocked scheme): warps pull chunks in
// order, so the probes sweep the table region by region with the active regions in L2.
// Results are written in the split order: rv[i] = value (or NOT_FOUND), rk[i] = the
// query's input position qpos[i] with bit 31 set when found; a second split by position
// and a placement pass put them back in input order.
template <class L>
struct EmitSwept {
  const uint32_t* __restrict__ qpos;
  uint32_t* __restrict__ rk;
  typename L::Val* __restrict__ rv;
  const void* vals;
  __device__ void operator()(uint64_t i, bool hit, const typename L::Slot& s, uint64_t idx) const {
    rv[i] = hit ? slot_value<L>(s, vals, idx) : L::kNotFound;
    rk[i] = qpos[i] | (hit ? 0x80000000u : 0u);
  }
};

template <class L, int G, int S, int H = 1>
__global__ void __launch_bounds__(256) k_sv_retrieve_swept(TableDesc t, const typename L::Key* __restrict__ keys,
                                                           const uint32_t* __restrict__ qpos, uint64_t n,
                                                           unsigned long long* counter, uint32_t chunk,
                                                           uint32_t* __restrict__ rk,
                                                           typename L::Val* __restrict__ rv) {
  RangeSrc src(n, 0, counter, chunk);
  uint32_t flags = 0;
  EmitSwept<L> emit{qpos, rk, rv, t.vals};
  sv_retrieve_range<L, G, S, EmitSwept<L>, typename L::Key, false, H>(t, keys, src, emit, flags);
  flush_flags(t.status, flags);
}

// Placement of split-ordered results: out[pos] = value, found[pos] = bit 31 of rk.  The
// input is grouped by position region and the grid walks it front to back, so the
// scattered stores of a moment fall into one or two L2-sized output regions.
template <class V>
__global__ void __launch_bounds__(256) k_place_results(const uint32_t* __restrict__ rk, const V* __restrict__ rv,
                                                       uint64_t n, V* __restrict__ out, uint8_t* __restrict__ found) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t k = ldg_stream(rk + i);
    const V v = ldg_stream(rv + i);
    const uint32_t pos = k & 0x7fffffffu;
    out[pos] = v;
    if (found) found[pos] = static_cast<uint8_t>(k >> 31);
  }
}

// Exact per-region counts of the positions 0..n-1 (region r holds positions
// [r * per, (r + 1) * per), the last one the rest).
static __global__ void k_index_hist(unsigned int* __restrict__ hist, uint32_t R, uint32_t per, uint64_t n) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const uint64_t lo = static_cast<uint64_t>(r) * per;
    const uint64_t hi = r + 1 == R ? n : lo + per;
    hist[r] = static_cast<unsigned int>(hi > lo ? hi - lo : 0);
  }
}

// ---------------------------------------------------------------------------------------
// insert (Sec. IV-B2 steps 1-7, Sec. IV-B3).  Returns through `added` the number of new
// keys this lane's groups stored (counted by lane r == 0 of each group).
//
// A window of W = G * S * H slots is walked in H steps of G * S slots (the paper's fixed
// window walked by a smaller group, Sec. IV-B2): a step that finds the key or an empty
// slot ends the walk, so the rest of the window is read only when the part before it is
// full.  That is the same order the whole-window read gives: an insert claims the earliest
// candidate of its sequence, so no live key ever sits behind an empty slot of its own
// sequence, whatever the window's width.
template <class L, int G, int S, int H = 1>
__device__ __forceinline__ void sv_insert_range(const TableDesc& t, const typename L::Key* __restrict__ keys,
                                                const typename L::Val* __restrict__ vals, RangeSrc& src,
                                                uint32_t& flags, long long& added) {
  using Slot = typename L::Slot;
  using Key = typename L::Key;
  using Val = typename L::Val;
  const SvLane<L, G, S> ln;
  constexpr int SW = G * S;  // slots of one step
  constexpr int W = SW * H;
  Slot* slots = static_cast<Slot*>(t.slots);
  bool act = false;
  uint64_t pos = 0;
  Key k = 0;
  Val v = 0;
  uint32_t w = 0, step = 0, j = 0, tag = 0, h = 0;
  bool have_t = false;     // a tombstone earlier on the sequence is remembered
  uint64_t t_slot = 0;     // its slot index
  Slot t_word{};           // and the word read there
  Feed<Key> fk;
  Feed<Val> fv;
  const bool unit = vals == nullptr;  // counting tables without weights: every occurrence counts 1
  while (true) {
    const bool more = src.ensure();
    if (more && src.fresh) {
      fk.load(keys, src.next, src.end);
      if (!unit) fv.load(vals, src.next, src.end);
      src.fresh = false;
    }
    uint64_t np = 0;
    const bool got = more && take_next(!act, ln.r, ln.gbase, src.next, src.end, np);
    const Key kin = fk.get(np, got);
    const Val vin = unit ? Val(1) : fv.get(np, got);
    if (more) {
      fk.advance(src.next);
      if (!unit) fv.advance(src.next);
    }
    if (got) {
      pos = np;
      k = kin;
      if (is_sentinel(k)) {
        // counting inserts run on aggregated batches whose padding is key 0 (the
        // aggregation pass already flagged the caller's sentinel keys)
        if (!(L::kCount && k == Key(0))) flags |= kFlagInvalid;
      } else {
        v = vin;
        act = true;
        j = 0;
        h = 0;
        have_t = false;
        probe_init(static_cast<uint64_t>(k), t.seed, t.p, w, step, tag);
      }
    }
    if (__ballot_sync(kFull, act) == 0) {
      if (!more) break;
      continue;
    }
    Slot s[S];
    uint32_t mm = 0, me = 0, mt = 0;
    const uint64_t lane_slot = static_cast<uint64_t>(w) * W + Steps<H>::offset(h, SW) + ln.r * S;
    if (act) {
      load_slots<L, S>(slots + lane_slot, s);
      classify<L, S>(s, k, mm, me, mt);
    }
    const uint32_t bm = group_vote<G>(mm != 0, ln.gbase);
    const uint32_t be = group_vote<G>(me != 0, ln.gbase);
    const uint32_t bt = group_vote<G>(mt != 0, ln.gbase);
    const uint32_t bc = group_vote<G>((me | mt) != 0, ln.gbase);
    const bool last = j + 1 >= t.p && Steps<H>::last(h);
    const bool claim = bm == 0 && (be != 0 || last);

    // The key is present: overwrite its value (duplicate warning, Sec. IV-B3).
    if (act && bm && ln.r == __ffs(bm) - 1) slot_store_value<L>(slots, t.vals, lane_slot + (__ffs(mm) - 1), v);

    // Claim the earliest candidate: a remembered tombstone from an earlier window,
    // else the first empty-or-tombstone slot of this window (Sec. IV-B2 steps 4 and 6).
    bool ok = false;
    if (act && claim) {
      if (have_t) {
        if (ln.r == 0) {
          ok = L::cas(slots + t_slot, t_word, L::make(k, v));
          if constexpr (L::kSoA) {
            if (ok) slot_store_value<L>(slots, t.vals, t_slot, v);
          }
        }
      } else if (bc && ln.r == __ffs(bc) - 1) {
        const int sub = __ffs(me | mt) - 1;
        ok = L::cas(slots + lane_slot + sub, pick<L, S>(s, sub), L::make(k, v));
        if constexpr (L::kSoA) {
          if (ok) slot_store_value<L>(slots, t.vals, lane_slot + sub, v);
        }
      }
    }
    if constexpr (G > 1) ok = __shfl_sync(kFull, ok, ln.gbase + ((have_t || bc == 0) ? 0 : __ffs(bc) - 1));

    // Remember the first tombstone met before the terminating window.  The branch is
    // warp-uniform, so every lane reaches the same shuffles.
    uint64_t nt_slot = 0;
    Slot nt_word{};
    if (__any_sync(kFull, act && !claim && bt != 0 && !have_t)) {
      const int sub = mt ? __ffs(mt) - 1 : 0;
      nt_slot = lane_slot + sub;
      nt_word = pick<L, S>(s, sub);
      if constexpr (G > 1) {
        const int tl = ln.gbase + (bt ? __ffs(bt) - 1 : 0);
        nt_slot = __shfl_sync(kFull, nt_slot, tl);
        nt_word = L::shfl(nt_word, tl);
      }
    }

    if (act) {
      if (bm) {
        if constexpr (!L::kCount) flags |= kFlagDuplicate;
        act = false;
      } else if (claim) {
        if (ok) {
          if (ln.r == 0) ++added;
          act = false;
        } else if (have_t) {
          // the remembered tombstone was taken: probe again from the start
          have_t = false;
          j = 0;
          h = 0;
          probe_init(static_cast<uint64_t>(k), t.seed, t.p, w, step, tag);
        } else if (bc == 0) {
          flags |= kFlagProbeLimit;  // every window visited, nothing to claim
          act = false;
        }
        // else: lost the race for a slot of this window; read it again
      } else {
        if (bt && !have_t) {
          have_t = true;
          t_slot = nt_slot;
          t_word = nt_word;
        }
        if (Steps<H>::more(h)) {
          ++h;  // the rest of this window, in the next trip
        } else {
          if (t.ovf != nullptr && ln.r == 0) ovf_mark(t.ovf, w, tag);  // walking past a window without an empty slot
          h = 0;
          ++j;
          w = probe_next(w, step, t.p);
        }
      }
    }
  }
}

// counter != nullptr: warps pull chunks in order (input sorted by table region).
template <class L, int G, int S, int H = 1>
__global__ void __launch_bounds__(256) k_sv_insert(TableDesc t, const typename L::Key* __restrict__ keys,
                                                   const typename L::Val* __restrict__ vals, uint64_t n,
                                                   uint64_t per_warp, unsigned long long* counter, uint32_t chunk) {
  RangeSrc src(n, per_warp, counter, chunk);
  if (counter == nullptr && src.next >= src.end) return;
  uint32_t flags = 0;
  long long added = 0;
  sv_insert_range<L, G, S, H>(t, keys, vals, src, flags, added);
  flush_flags(t.status, flags);
  flush_delta(t.size, added);
}

// ---------------------------------------------------------------------------------------
// erase (Sec. IV-B5): the key's slot becomes a tombstone.  `removed` counts erased keys;
// on_erase(slot) sees the word that was replaced (multi-value tables use it to adjust
// their pair count).
template <class L, int G, int S, class OnErase, class KIn = typename L::Key, int H = 1>
__device__ __forceinline__ void sv_erase_range(const TableDesc& t, const KIn* __restrict__ keys, RangeSrc& src,
                                               uint32_t& flags, long long& removed, OnErase& on_erase) {
  using Slot = typename L::Slot;
  using Key = typename L::Key;
  const SvLane<L, G, S> ln;
  constexpr int SW = G * S;  // slots of one step; a window is walked in H steps
  constexpr int W = SW * H;
  Slot* slots = static_cast<Slot*>(t.slots);
  bool act = false;
  Key k = 0;
  uint32_t w = 0, step = 0, j = 0, tag = 0, h = 0;
  Feed<KIn> fk;
  while (true) {
    const bool more = src.ensure();
    if (more && src.fresh) {
      fk.load(keys, src.next, src.end);
      src.fresh = false;
    }
    uint64_t np = 0;
    const bool got = more && take_next(!act, ln.r, ln.gbase, src.next, src.end, np);
    const KIn kin = fk.get(np, got);
    if (more) fk.advance(src.next);
    if (got) {
      k = static_cast<Key>(kin);
      if (is_sentinel(kin)) {
        flags |= kFlagInvalid;
      } else {
        act = true;
        j = 0;
        h = 0;
        probe_init(static_cast<uint64_t>(k), t.seed, t.p, w, step, tag);
      }
    }
    if (__ballot_sync(kFull, act) == 0) {
      if (!more) break;
      continue;
    }
    Slot s[S];
    uint32_t mm = 0, me = 0, mt = 0;
    const uint64_t lane_slot = static_cast<uint64_t>(w) * W + Steps<H>::offset(h, SW) + ln.r * S;
    if (act) {
      load_slots<L, S>(slots + lane_slot, s);
      classify<L, S>(s, k, mm, me, mt);
    }
    const uint32_t bm = group_vote<G>(mm != 0, ln.gbase);
    const uint32_t be = group_vote<G>(me != 0, ln.gbase);
    uint32_t fw = 0xffffffffu;
    if (t.ovf != nullptr && act && !bm && !be && Steps<H>::last(h)) fw = ovf_word(t.ovf, w);
    bool ok = false;
    if (act && bm && ln.r == __ffs(bm) - 1) {
      const int sub = __ffs(mm) - 1;
      const Slot old = pick<L, S>(s, sub);
      ok = L::cas(slots + lane_slot + sub, old, L::tomb());
      if (ok) on_erase(old);
    }
    if constexpr (G > 1) ok = __shfl_sync(kFull, ok, ln.gbase + (bm ? __ffs(bm) - 1 : 0));
    if (act) {
      if (bm) {
        if (ok) {
          if (ln.r == 0) ++removed;
          act = false;
        }
        // else: another erase of the same key won; read the window again
      } else if (!be && Steps<H>::more(h)) {
        ++h;  // the rest of this window
      } else if (be || !ovf_bit(fw, w, tag) || ++j >= t.p) {
        act = false;  // absent: nothing to erase
      } else {
        h = 0;
        w = probe_next(w, step, t.p);
      }
    }
  }
}

struct NoOnErase {
  template <class Slot>
  __device__ void operator()(const Slot&) const {}
};

template <class L, int G, int S, int H = 1>
__global__ void __launch_bounds__(256) k_sv_erase(TableDesc t, const typename L::Key* __restrict__ keys, uint64_t n,
                                                  uint64_t per_warp) {
  RangeSrc src(n, per_warp, nullptr, 0);
  if (src.next >= src.end) return;
  uint32_t flags = 0;
  long long removed = 0;
  NoOnErase none;
  sv_erase_range<L, G, S, NoOnErase, typename L::Key, H>(t, keys, src, flags, removed, none);
  flush_flags(t.status, flags);
  flush_delta(t.size, -removed);
}

}  // namespace wc
