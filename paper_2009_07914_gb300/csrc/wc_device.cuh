// Device-side building blocks shared by every kernel of the library: slot layouts, the
// outer probing scheme, window loads, group votes and status accounting.
//
// Probing (Sec. IV-B2, cooperative probing scheme): the table is p windows of W slots,
// p prime.  A key visits windows w_j = (w_0 + j * step) mod p, j = 0..p-1 (outer
// double hashing; step in [1, p-1] and p prime make the sequence visit every window
// exactly once), and inside a window all W slots at once (inner linear probing).  A
// group of G lanes reads one window together: lane r holds slots [r*S, r*S + S) with
// S = W / G, so slot order inside a window is (lane, sub-slot) order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "wc_device_api.cuh"

namespace wc {

constexpr uint32_t kFull = 0xffffffffu;

// Device status-word bits (same values as WC_FLAG_* of the public header).
enum : uint32_t {
  kFlagDuplicate = 1u,
  kFlagInvalid = 2u,
  kFlagProbeLimit = 4u,
  kFlagPoolExhausted = 8u,
  kFlagCountOverflow = 16u,
  kFlagQueueTimeout = 32u,
};

// The probing sequence (fmix64 hash, first window and step, next window) is the one the
// public device API defines, so keys inserted by user kernels and by the bulk kernels
// follow the same sequences.
using wc_dev::fmix64;
using wc_dev::probe_init;
using wc_dev::probe_next;
using wc_dev::overflow_shift;

// ---- vector loads that bypass L1 (L2 is the coherence point for CAS) ----------------

__device__ __forceinline__ void ldcg1(const void* p, unsigned long long (&u)[1]) {
  asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(u[0]) : "l"(p));
}
__device__ __forceinline__ void ldcg2(const void* p, unsigned long long* u) {
  asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(u[0]), "=l"(u[1]) : "l"(p));
}
__device__ __forceinline__ void ldcg4(const void* p, unsigned long long* u) {
  asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(u[0]), "=l"(u[1]), "=l"(u[2]), "=l"(u[3])
               : "l"(p));
}

// Load N 64-bit words (N in 1, 2, 4, 8; address aligned to min(8N, 32) bytes).
template <int N>
__device__ __forceinline__ void load_words(const unsigned long long* p, unsigned long long (&u)[N]) {
  if constexpr (N == 1) {
    ldcg1(p, u);
  } else if constexpr (N == 2) {
    ldcg2(p, u);
  } else if constexpr (N == 4) {
    ldcg4(p, u);
  } else {
    static_assert(N % 4 == 0, "word count");
#pragma unroll
    for (int i = 0; i < N; i += 4) ldcg4(p + i, u + i);
  }
}

// Streamed input element (read once): loaded with an evict-first L2 cache policy, so
// batches flowing through L2 displace table lines as little as possible.
__device__ __forceinline__ unsigned long long evict_first_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint32_t ldg_stream(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
               : "=r"(v)
               : "l"(p), "l"(evict_first_policy()));
  return v;
}
__device__ __forceinline__ unsigned long long ldg_stream(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;"
               : "=l"(v)
               : "l"(p), "l"(evict_first_policy()));
  return v;
}

// ---- overflow bits --------------------------------------------------------------------
// Eight bits per window (one byte), indexed by a 3-bit tag of the key's hash: an insert
// that walks past a window because it holds no empty slot sets the bit of its own tag.
// Every key stored beyond a window on its own sequence has passed that window, so a lookup
// that meets a window without the key, without an empty slot and with its tag's bit clear
// may stop there: the key is absent.  With one bit per window an absent key walks on
// wherever any key overflowed; with eight, only where a key of its own tag did (W = 8,
// load 0.9: 2.07 -> 1.20 windows per absent key).  The bits only ever get set (a clear
// resets them), so they stay a superset of what lookups need after erases and re-inserts.
//
// The bulk kernels read and set the bits with an evict-last L2 policy: at one byte per
// window they are 1/64 of a table of 8-byte slots and are touched far more often than any
// one window (2^27 keys at load 0.9: bulk insert + retrieve 26.9 -> 27.5 G ops/s).  The
// public device API keeps plain accesses: its one-thread-per-key inserts CAS into the
// window they have just read, and lose more of those lines to the pinned bits than they
// gain (6.9 -> 6.4 G inserts/s with the hint).
__device__ __forceinline__ unsigned long long evict_last_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint32_t ovf_word(const uint32_t* ovf, uint32_t w) {
  uint32_t v;
  asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;"
               : "=r"(v)
               : "l"(ovf + (w >> 2)), "l"(evict_last_policy()));
  return v;
}
__device__ __forceinline__ bool ovf_bit(uint32_t word, uint32_t w, uint32_t tag) {
  return (word >> overflow_shift(w, tag)) & 1u;
}
__device__ __forceinline__ void ovf_mark(uint32_t* ovf, uint32_t w, uint32_t tag) {
  asm volatile("red.relaxed.gpu.global.or.L2::cache_hint.b32 [%0], %1, %2;"
               :
               : "l"(ovf + (w >> 2)), "r"(1u << overflow_shift(w, tag)), "l"(evict_last_policy())
               : "memory");
}

// ---- slot layouts ---------------------------------------------------------------------

// Packed array-of-structs slot (Sec. IV-B1): a uint32 key in the low half and a uint32
// value in the high half of one 64-bit word, so one 64-bit CAS stores both.
struct LayoutP32 {
  using Key = uint32_t;
  using Val = uint32_t;
  struct Slot {
    unsigned long long w;
  };
  static constexpr int kWords = 1;
  static constexpr bool kHalf = false;   // slots of 4 bytes, two per loaded 64-bit word
  static constexpr bool kCount = false;  // duplicates overwrite the value (single-value table)
  static constexpr bool kSoA = false;    // values in the slot word (not in a separate array)
  static constexpr Key kEmpty = 0u;
  static constexpr Key kTomb = 0xffffffffu;
  static constexpr Val kNotFound = 0xffffffffu;
  __device__ static Key key(const Slot& s) { return static_cast<uint32_t>(s.w); }
  __device__ static Val val(const Slot& s) { return static_cast<uint32_t>(s.w >> 32); }
  __device__ static Slot make(Key k, Val v) { return Slot{(static_cast<unsigned long long>(v) << 32) | k}; }
  __device__ static Slot tomb() { return Slot{0xffffffffull}; }
  __device__ static Slot from_words(const unsigned long long* u) { return Slot{u[0]}; }
  __device__ static bool cas(Slot* p, const Slot& e, const Slot& d) {
    return atomicCAS(&p->w, e.w, d.w) == e.w;
  }
  __device__ static void store_val(Slot* p, Val v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(reinterpret_cast<uint32_t*>(&p->w) + 1), "r"(v)
                 : "memory");
  }
  __device__ static Slot shfl(const Slot& s, int src) { return Slot{__shfl_sync(kFull, s.w, src)}; }
};


// 16-byte array-of-structs slot {uint64 key, uint64 value}, claimed with one 128-bit CAS
// (atom.cas.b128, sm_90 and later).  The paper's GV100 had only 64-bit CAS and had to
// swap the key first and store the value afterwards (Sec. II, hazard (1) of Sec. IV-D);
// one 16-byte CAS stores the pair at once.
struct LayoutP64 {
  using Key = unsigned long long;
  using Val = unsigned long long;
  struct Slot {
    unsigned long long k, v;
  };
  static constexpr int kWords = 2;
  static constexpr bool kHalf = false;
  static constexpr bool kCount = false;
  static constexpr bool kSoA = false;
  static constexpr Key kEmpty = 0ull;
  static constexpr Key kTomb = ~0ull;
  static constexpr Val kNotFound = ~0ull;
  __device__ static Key key(const Slot& s) { return s.k; }
  __device__ static Val val(const Slot& s) { return s.v; }
  __device__ static Slot make(Key k, Val v) { return Slot{k, v}; }
  __device__ static Slot tomb() { return Slot{~0ull, 0ull}; }
  __device__ static Slot from_words(const unsigned long long* u) { return Slot{u[0], u[1]}; }
  __device__ static bool cas(Slot* p, const Slot& e, const Slot& d) {
    unsigned long long olo, ohi;
    asm volatile(
        "{\n\t.reg .b128 e, d, o;\n\t"
        "mov.b128 e, {%2, %3};\n\t"
        "mov.b128 d, {%4, %5};\n\t"
        "atom.global.cas.b128 o, [%6], e, d;\n\t"
        "mov.b128 {%0, %1}, o;\n\t}"
        : "=l"(olo), "=l"(ohi)
        : "l"(e.k), "l"(e.v), "l"(d.k), "l"(d.v), "l"(p)
        : "memory");
    return olo == e.k && ohi == e.v;
  }
  __device__ static void store_val(Slot* p, Val v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(&p->v), "l"(v) : "memory");
  }
  __device__ static Slot shfl(const Slot& s, int src) {
    return Slot{__shfl_sync(kFull, s.k, src), __shfl_sync(kFull, s.v, src)};
  }
};

// Counting tables (the paper's CountingHashTable: counts key occurrences): the same slot
// words, but an insert of a stored key adds its weight to the stored count with one
// atomic add on the value word instead of overwriting it.
struct LayoutC32 : LayoutP32 {
  static constexpr bool kCount = true;
  __device__ static void store_val(Slot* p, Val v) { atomicAdd(reinterpret_cast<uint32_t*>(&p->w) + 1, v); }
};
struct LayoutC64 : LayoutP64 {
  static constexpr bool kCount = true;
  __device__ static void store_val(Slot* p, Val v) { atomicAdd(&p->v, v); }
};

// Hash sets (the paper's HashSet): a slot holds only a key.  "Values" read back are 1 for
// a stored key; inserting a stored key leaves it as it is (DUPLICATE_KEY is raised).
struct LayoutK64 {
  using Key = unsigned long long;
  using Val = unsigned long long;
  struct Slot {
    unsigned long long k;
  };
  static constexpr int kWords = 1;
  static constexpr bool kHalf = false;
  static constexpr bool kCount = false;
  static constexpr bool kSoA = false;
  static constexpr Key kEmpty = 0ull;
  static constexpr Key kTomb = ~0ull;
  static constexpr Val kNotFound = 0ull;
  __device__ static Key key(const Slot& s) { return s.k; }
  __device__ static Val val(const Slot&) { return 1ull; }
  __device__ static Slot make(Key k, Val) { return Slot{k}; }
  __device__ static Slot tomb() { return Slot{~0ull}; }
  __device__ static Slot from_words(const unsigned long long* u) { return Slot{u[0]}; }
  __device__ static bool cas(Slot* p, const Slot& e, const Slot& d) { return atomicCAS(&p->k, e.k, d.k) == e.k; }
  __device__ static void store_val(Slot*, Val) {}
  __device__ static Slot shfl(const Slot& s, int src) { return Slot{__shfl_sync(kFull, s.k, src)}; }
};
struct LayoutK32 {
  using Key = uint32_t;
  using Val = uint32_t;
  struct Slot {
    uint32_t k;
  };
  static constexpr int kWords = 1;       // per loaded word (two slots)
  static constexpr bool kHalf = true;
  static constexpr bool kCount = false;
  static constexpr bool kSoA = false;
  static constexpr Key kEmpty = 0u;
  static constexpr Key kTomb = 0xffffffffu;
  static constexpr Val kNotFound = 0u;
  __device__ static Key key(const Slot& s) { return s.k; }
  __device__ static Val val(const Slot&) { return 1u; }
  __device__ static Slot make(Key k, Val) { return Slot{k}; }
  __device__ static Slot tomb() { return Slot{0xffffffffu}; }
  __device__ static bool cas(Slot* p, const Slot& e, const Slot& d) { return atomicCAS(&p->k, e.k, d.k) == e.k; }
  __device__ static void store_val(Slot*, Val) {}
  __device__ static Slot shfl(const Slot& s, int src) { return Slot{__shfl_sync(kFull, s.k, src)}; }
};

// Struct-of-arrays single-value tables (Sec. IV-A: keys and values in two arrays of the
// same length): probing reads the key array only -- twice the keys per line for 4+4-byte
// pairs -- and a hit reads the value at the same index.  An insert claims the key slot
// with one CAS and then writes the value with a plain store; the value is complete when
// the insert call is (Sec. IV-D orders calls), the relaxed value write the paper notes.
struct LayoutS32 : LayoutK32 {
  static constexpr bool kSoA = true;
  static constexpr Val kNotFound = 0xffffffffu;
};
struct LayoutS64 : LayoutK64 {
  static constexpr bool kSoA = true;
  static constexpr Val kNotFound = ~0ull;
};

// Value of slot `idx` (whose word is s) and its update, for every layout: packed layouts
// keep the value in the slot word; struct-of-arrays layouts in the value array.
template <class L>
__device__ __forceinline__ typename L::Val slot_value(const typename L::Slot& s, const void* vals, uint64_t idx) {
  if constexpr (L::kSoA) {
    return static_cast<const typename L::Val*>(vals)[idx];
  } else {
    return L::val(s);
  }
}

template <class L>
__device__ __forceinline__ void slot_store_value(void* slots, void* vals, uint64_t idx, typename L::Val v) {
  if constexpr (L::kSoA) {
    static_cast<typename L::Val*>(vals)[idx] = v;
  } else {
    L::store_val(static_cast<typename L::Slot*>(slots) + idx, v);
  }
}

// S consecutive slots of one lane.
template <class L, int S>
__device__ __forceinline__ void load_slots(const typename L::Slot* p, typename L::Slot (&s)[S]) {
  if constexpr (L::kHalf) {  // 4-byte slots: S / 2 words, low half first (little-endian)
    static_assert(S % 2 == 0, "4-byte slots are loaded in pairs");
    unsigned long long u[S / 2];
    load_words<S / 2>(reinterpret_cast<const unsigned long long*>(p), u);
#pragma unroll
    for (int i = 0; i < S; ++i) s[i].k = static_cast<uint32_t>(u[i / 2] >> (32 * (i & 1)));
  } else {
    unsigned long long u[S * L::kWords];
    load_words<S * L::kWords>(reinterpret_cast<const unsigned long long*>(p), u);
#pragma unroll
    for (int i = 0; i < S; ++i) s[i] = L::from_words(u + i * L::kWords);
  }
}

// s[i] selected without dynamic register indexing.
template <class L, int S>
__device__ __forceinline__ typename L::Slot pick(const typename L::Slot (&s)[S], int i) {
  typename L::Slot x = s[0];
#pragma unroll
  for (int k = 1; k < S; ++k)
    if (i == k) x = s[k];
  return x;
}

// My group's G bits of a warp ballot.
template <int G>
__device__ __forceinline__ uint32_t group_bits(uint32_t ballot, int gbase) {
  if constexpr (G == 32) {
    return ballot;
  } else {
    return (ballot >> gbase) & ((1u << G) - 1u);
  }
}

template <int G>
__device__ __forceinline__ uint32_t group_vote(bool pred, int gbase) {
  if constexpr (G == 1) {
    return pred ? 1u : 0u;
  } else {
    return group_bits<G>(__ballot_sync(kFull, pred), gbase);
  }
}

// Hand each idle group of the warp the next input position of the warp's range
// [next, end).  `next` is warp-uniform and advances by the number of idle groups.
// Positions go to idle groups in lane order, so a warp reads its inputs nearly
// contiguously.  Returns true if this lane's group received a position.
__device__ __forceinline__ bool take_next(bool idle, int r, int gbase, uint64_t& next, uint64_t end,
                                          uint64_t& pos) {
  const uint32_t idle_leaders = __ballot_sync(kFull, idle && r == 0);
  const uint64_t mine = next + __popc(idle_leaders & ((1u << gbase) - 1u));
  next += __popc(idle_leaders);
  if (idle && mine < end) {
    pos = mine;
    return true;
  }
  return false;
}

// Warp-aggregated status and counter updates, once per warp at kernel end.
__device__ __forceinline__ void flush_flags(uint32_t* status, uint32_t flags) {
  flags = __reduce_or_sync(kFull, flags);
  if ((threadIdx.x & 31) == 0 && flags) atomicOr(status, flags);
}

__device__ __forceinline__ void flush_delta(unsigned long long* counter, long long delta) {
  // butterfly sum over the warp, then one atomic per warp
  long long d = delta;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
  if ((threadIdx.x & 31) == 0 && d != 0) atomicAdd(counter, static_cast<unsigned long long>(d));
}

}  // namespace wc
