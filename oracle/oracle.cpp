// CPU oracle for the bulk hash-table operations.  TEST INFRASTRUCTURE ONLY: the tests,
// the package's smoke check and the bench's CPU-baseline leg load it; the library
// itself never does.  It shares no code, header or constant generator with the CUDA
// path.
//
// What it computes is the plain definition of each operation, over the C++ standard
// library's associative containers (no blocking, no reordering):
//
//   * single-value table (Sec. IV, "SingleValueHashTable": each key occurs once)
//       insert   : key absent -> M[k] = v; key present -> M[k] = v and the duplicate-key
//                  warning of Sec. IV-B3 is raised (the stored value is overwritten).
//       retrieve : M[k] if present (Sec. IV-B4), else NOT_FOUND = all ones, found = 0.
//       erase    : removes k if present (Sec. IV-B5); an absent key is a no-op.
//       size     : number of live keys; load factor = size / capacity (Sec. II).
//   * multi-value table (Sec. IV, "MultiValueHashTable": a key may occur many times)
//       insert        : always appends (k, v) (multiset semantics).
//       count_values  : per query, the number of values of that key; offsets are the
//                       exclusive prefix sum with n+1 entries (Sec. IV-B4).
//       retrieve_multi: query i's values are written to out[offsets[i] .. offsets[i+1]);
//                       their order inside a segment is unspecified.
//       erase         : removes every value of the key.
//
// Sentinel keys (0 = empty marker k_e, all ones = tombstone k_t, Sec. IV-B1 and
// IV-B5) cannot be stored: they are skipped and reported with the INVALID_KEY flag.
// Flag bits match the meaning (not the code) of the library's device status word.
#include <cstdint>
#include <cstring>
#include <functional>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

constexpr uint32_t F_DUPLICATE = 1u;
constexpr uint32_t F_INVALID = 2u;

template <class K>
bool is_sentinel(K k) { return k == K(0) || k == K(~K(0)); }

template <class K, class V>
struct SV {
  using Key = K;
  using Val = V;
  std::unordered_map<K, V> m;

  uint32_t insert(const K* keys, const V* vals, uint64_t n) {
    uint32_t f = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (is_sentinel(keys[i])) { f |= F_INVALID; continue; }
      auto it = m.find(keys[i]);
      if (it == m.end()) {
        m.emplace(keys[i], vals[i]);
      } else {
        it->second = vals[i];
        f |= F_DUPLICATE;
      }
    }
    return f;
  }
  uint32_t retrieve(const K* keys, uint64_t n, V* out, uint8_t* found) const {
    uint32_t f = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (is_sentinel(keys[i])) f |= F_INVALID;
      auto it = is_sentinel(keys[i]) ? m.end() : m.find(keys[i]);
      bool hit = it != m.end();
      out[i] = hit ? it->second : V(~V(0));
      if (found) found[i] = hit ? 1 : 0;
    }
    return f;
  }
  uint32_t erase(const K* keys, uint64_t n) {
    uint32_t f = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (is_sentinel(keys[i])) { f |= F_INVALID; continue; }
      m.erase(keys[i]);
    }
    return f;
  }
};

template <class K, class V>
struct MV {
  std::unordered_multimap<K, V> m;

  uint32_t insert(const K* keys, const V* vals, uint64_t n) {
    uint32_t f = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (is_sentinel(keys[i])) { f |= F_INVALID; continue; }
      m.emplace(keys[i], vals[i]);
    }
    return f;
  }
  uint32_t count_values(const K* keys, uint64_t n, uint64_t* offsets) const {
    uint32_t f = 0;
    uint64_t run = 0;
    for (uint64_t i = 0; i < n; ++i) {
      offsets[i] = run;
      if (is_sentinel(keys[i])) { f |= F_INVALID; continue; }
      run += m.count(keys[i]);
    }
    offsets[n] = run;
    return f;
  }
  uint32_t retrieve_multi(const K* keys, uint64_t n, const uint64_t* offsets, V* out) const {
    uint32_t f = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (is_sentinel(keys[i])) { f |= F_INVALID; continue; }
      uint64_t o = offsets[i];
      auto range = m.equal_range(keys[i]);
      for (auto it = range.first; it != range.second; ++it) {
        if (o < offsets[i + 1]) out[o] = it->second;
        ++o;
      }
    }
    return f;
  }
  uint32_t erase(const K* keys, uint64_t n) {
    uint32_t f = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (is_sentinel(keys[i])) { f |= F_INVALID; continue; }
      m.erase(keys[i]);
    }
    return f;
  }
};

// A tagged handle so one C entry point serves every key/value width.
struct Handle {
  int kind;  // 0 = single-value, 1 = multi-value
  int kb, vb;
  void* impl;
};

template <template <class, class> class T, class F>
auto dispatch(Handle* h, F&& f) {
  if (h->kb == 4 && h->vb == 4) return f(static_cast<T<uint32_t, uint32_t>*>(h->impl));
  if (h->kb == 8 && h->vb == 8) return f(static_cast<T<uint64_t, uint64_t>*>(h->impl));
  if (h->kb == 8 && h->vb == 4) return f(static_cast<T<uint64_t, uint32_t>*>(h->impl));
  return f(static_cast<T<uint32_t, uint64_t>*>(h->impl));
}

template <template <class, class> class T>
void* make(int kb, int vb) {
  if (kb == 4 && vb == 4) return new T<uint32_t, uint32_t>();
  if (kb == 8 && vb == 8) return new T<uint64_t, uint64_t>();
  if (kb == 8 && vb == 4) return new T<uint64_t, uint32_t>();
  return new T<uint32_t, uint64_t>();
}

bool valid_widths(int kb, int vb) { return (kb == 4 || kb == 8) && (vb == 4 || vb == 8); }

}  // namespace

extern "C" {

void* oracle_create(int kind, int key_bytes, int value_bytes) {
  if (!valid_widths(key_bytes, value_bytes) || (kind != 0 && kind != 1)) return nullptr;
  auto* h = new Handle{kind, key_bytes, value_bytes, nullptr};
  h->impl = kind == 0 ? make<SV>(key_bytes, value_bytes) : make<MV>(key_bytes, value_bytes);
  return h;
}

void oracle_destroy(void* p) {
  auto* h = static_cast<Handle*>(p);
  if (!h) return;
  if (h->kind == 0) dispatch<SV>(h, [](auto* t) { delete t; return 0; });
  else dispatch<MV>(h, [](auto* t) { delete t; return 0; });
  delete h;
}

uint32_t oracle_insert(void* p, const void* keys, const void* vals, uint64_t n) {
  auto* h = static_cast<Handle*>(p);
  if (h->kind == 0)
    return dispatch<SV>(h, [&](auto* t) {
      using M = std::remove_pointer_t<decltype(t)>;
      using K = typename decltype(M::m)::key_type;
      using V = typename decltype(M::m)::mapped_type;
      return t->insert(static_cast<const K*>(keys), static_cast<const V*>(vals), n);
    });
  return dispatch<MV>(h, [&](auto* t) {
    using M = std::remove_pointer_t<decltype(t)>;
    using K = typename decltype(M::m)::key_type;
    using V = typename decltype(M::m)::mapped_type;
    return t->insert(static_cast<const K*>(keys), static_cast<const V*>(vals), n);
  });
}

// Single-value only.
uint32_t oracle_retrieve(void* p, const void* keys, uint64_t n, void* out, uint8_t* found) {
  auto* h = static_cast<Handle*>(p);
  if (h->kind != 0) return 0xFFFFFFFFu;
  return dispatch<SV>(h, [&](auto* t) {
    using M = std::remove_pointer_t<decltype(t)>;
    using K = typename decltype(M::m)::key_type;
    using V = typename decltype(M::m)::mapped_type;
    return t->retrieve(static_cast<const K*>(keys), n, static_cast<V*>(out), found);
  });
}

uint32_t oracle_erase(void* p, const void* keys, uint64_t n) {
  auto* h = static_cast<Handle*>(p);
  if (h->kind == 0)
    return dispatch<SV>(h, [&](auto* t) {
      using M = std::remove_pointer_t<decltype(t)>;
      using K = typename decltype(M::m)::key_type;
      return t->erase(static_cast<const K*>(keys), n);
    });
  return dispatch<MV>(h, [&](auto* t) {
    using M = std::remove_pointer_t<decltype(t)>;
    using K = typename decltype(M::m)::key_type;
    return t->erase(static_cast<const K*>(keys), n);
  });
}

// Multi-value only.
uint32_t oracle_count_values(void* p, const void* keys, uint64_t n, uint64_t* offsets) {
  auto* h = static_cast<Handle*>(p);
  if (h->kind != 1) return 0xFFFFFFFFu;
  return dispatch<MV>(h, [&](auto* t) {
    using M = std::remove_pointer_t<decltype(t)>;
    using K = typename decltype(M::m)::key_type;
    return t->count_values(static_cast<const K*>(keys), n, offsets);
  });
}

uint32_t oracle_retrieve_multi(void* p, const void* keys, uint64_t n, const uint64_t* offsets,
                               void* out) {
  auto* h = static_cast<Handle*>(p);
  if (h->kind != 1) return 0xFFFFFFFFu;
  return dispatch<MV>(h, [&](auto* t) {
    using M = std::remove_pointer_t<decltype(t)>;
    using K = typename decltype(M::m)::key_type;
    using V = typename decltype(M::m)::mapped_type;
    return t->retrieve_multi(static_cast<const K*>(keys), n, offsets, static_cast<V*>(out));
  });
}

uint64_t oracle_size(void* p) {
  auto* h = static_cast<Handle*>(p);
  if (h->kind == 0) return dispatch<SV>(h, [](auto* t) { return (uint64_t)t->m.size(); });
  return dispatch<MV>(h, [](auto* t) { return (uint64_t)t->m.size(); });
}

// Number of distinct live keys (equals size for a single-value table).
uint64_t oracle_num_keys(void* p) {
  auto* h = static_cast<Handle*>(p);
  if (h->kind == 0) return dispatch<SV>(h, [](auto* t) { return (uint64_t)t->m.size(); });
  return dispatch<MV>(h, [](auto* t) {
    uint64_t c = 0;
    for (auto it = t->m.begin(); it != t->m.end();) {
      auto r = t->m.equal_range(it->first);
      ++c;
      it = r.second;
    }
    return c;
  });
}

// Reserve buckets for n elements (a plain std::unordered_map::reserve); used by the
// CPU-baseline timing so rehashing is not what gets measured.
void oracle_reserve(void* p, uint64_t n) {
  auto* h = static_cast<Handle*>(p);
  if (h->kind == 0) dispatch<SV>(h, [&](auto* t) { t->m.reserve(n); return 0; });
  else dispatch<MV>(h, [&](auto* t) { t->m.reserve(n); return 0; });
}

}  // extern "C"

// ---- sharded single-value table (the multi-core form of the same definition) ----------
// T single-value maps; key k belongs to shard std::hash<K>()(k) mod T.  Thread t walks
// every batch in input order and applies the elements of its own shard to its own map,
// so every key sees its operations in batch order, in one map: the results are those of
// the single map above (every flag, value and found bit), only computed on T cores.
namespace {

template <class K, class V>
struct Sharded {
  std::vector<SV<K, V>> shards;
  explicit Sharded(int t) : shards(static_cast<size_t>(t)) {}
  int T() const { return static_cast<int>(shards.size()); }
  bool mine(K k, int t) const { return std::hash<K>()(k) % static_cast<size_t>(T()) == static_cast<size_t>(t); }

  template <class F>
  uint32_t each(F f) {
    std::vector<uint32_t> flags(shards.size(), 0u);
    std::vector<std::thread> th;
    for (int t = 0; t < T(); ++t) th.emplace_back([&, t] { flags[t] = f(t); });
    for (auto& x : th) x.join();
    uint32_t all = 0;
    for (uint32_t x : flags) all |= x;
    return all;
  }
  uint32_t insert(const K* keys, const V* vals, uint64_t n) {
    return each([&](int t) {
      uint32_t f = 0;
      for (uint64_t i = 0; i < n; ++i) {
        if (is_sentinel(keys[i])) { f |= F_INVALID; continue; }
        if (mine(keys[i], t)) f |= shards[t].insert(keys + i, vals + i, 1);
      }
      return f;
    });
  }
  uint32_t retrieve(const K* keys, uint64_t n, V* out, uint8_t* found) {
    return each([&](int t) {
      uint32_t f = 0;
      for (uint64_t i = 0; i < n; ++i) {
        if (is_sentinel(keys[i])) {
          if (t == 0) f |= shards[0].retrieve(keys + i, 1, out + i, found ? found + i : nullptr);
          continue;
        }
        if (mine(keys[i], t)) f |= shards[t].retrieve(keys + i, 1, out + i, found ? found + i : nullptr);
      }
      return f;
    });
  }
  uint32_t erase(const K* keys, uint64_t n) {
    return each([&](int t) {
      uint32_t f = 0;
      for (uint64_t i = 0; i < n; ++i) {
        if (is_sentinel(keys[i])) { f |= F_INVALID; continue; }
        if (mine(keys[i], t)) f |= shards[t].erase(keys + i, 1);
      }
      return f;
    });
  }
  uint64_t size() const {
    uint64_t s = 0;
    for (const auto& x : shards) s += x.m.size();
    return s;
  }
  void reserve(uint64_t n) {
    for (auto& x : shards) x.m.reserve(n / shards.size() + 1);
  }
};

template <class F>
auto sharded_dispatch(Handle* h, F&& f) {
  if (h->kb == 4 && h->vb == 4) return f(static_cast<Sharded<uint32_t, uint32_t>*>(h->impl));
  if (h->kb == 8 && h->vb == 8) return f(static_cast<Sharded<uint64_t, uint64_t>*>(h->impl));
  if (h->kb == 8 && h->vb == 4) return f(static_cast<Sharded<uint64_t, uint32_t>*>(h->impl));
  return f(static_cast<Sharded<uint32_t, uint64_t>*>(h->impl));
}

}  // namespace

extern "C" {

void* oracle_sharded_create(int key_bytes, int value_bytes, int threads) {
  if (!valid_widths(key_bytes, value_bytes) || threads < 1) return nullptr;
  auto* h = new Handle{2, key_bytes, value_bytes, nullptr};
  if (key_bytes == 4 && value_bytes == 4) h->impl = new Sharded<uint32_t, uint32_t>(threads);
  else if (key_bytes == 8 && value_bytes == 8) h->impl = new Sharded<uint64_t, uint64_t>(threads);
  else if (key_bytes == 8) h->impl = new Sharded<uint64_t, uint32_t>(threads);
  else h->impl = new Sharded<uint32_t, uint64_t>(threads);
  return h;
}

void oracle_sharded_destroy(void* p) {
  auto* h = static_cast<Handle*>(p);
  if (!h) return;
  sharded_dispatch(h, [](auto* t) { delete t; return 0; });
  delete h;
}

uint32_t oracle_sharded_insert(void* p, const void* keys, const void* vals, uint64_t n) {
  return sharded_dispatch(static_cast<Handle*>(p), [&](auto* t) {
    using M = std::remove_pointer_t<decltype(t)>;
    using K = typename decltype(M::shards)::value_type::Key;
    using V = typename decltype(M::shards)::value_type::Val;
    return t->insert(static_cast<const K*>(keys), static_cast<const V*>(vals), n);
  });
}

uint32_t oracle_sharded_retrieve(void* p, const void* keys, uint64_t n, void* out, uint8_t* found) {
  return sharded_dispatch(static_cast<Handle*>(p), [&](auto* t) {
    using M = std::remove_pointer_t<decltype(t)>;
    using K = typename decltype(M::shards)::value_type::Key;
    using V = typename decltype(M::shards)::value_type::Val;
    return t->retrieve(static_cast<const K*>(keys), n, static_cast<V*>(out), found);
  });
}

uint32_t oracle_sharded_erase(void* p, const void* keys, uint64_t n) {
  return sharded_dispatch(static_cast<Handle*>(p), [&](auto* t) {
    using M = std::remove_pointer_t<decltype(t)>;
    using K = typename decltype(M::shards)::value_type::Key;
    return t->erase(static_cast<const K*>(keys), n);
  });
}

uint64_t oracle_sharded_size(void* p) {
  return sharded_dispatch(static_cast<Handle*>(p), [](auto* t) { return t->size(); });
}

void oracle_sharded_reserve(void* p, uint64_t n) {
  sharded_dispatch(static_cast<Handle*>(p), [&](auto* t) { t->reserve(n); return 0; });
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Counting table (Sec. IV, "CountingHashTable": counts key occurrences) and hash set
// (Sec. IV, "HashSet": a set of keys, each once), by their plain definitions.
//   counting: add(k, w) -> C[k] += w (w = 1 when no weights), modulo 2^(8 * width);
//             get(k) -> C[k] or NOT_FOUND; erase(k) removes k.
//   set:      add(k) -> S += {k} (DUPLICATE_KEY when k was in S); contains(k); erase(k).
// Keys and counts have the same width (4 or 8 bytes).
namespace {

struct Counts {
  int kb;
  bool set;
  std::unordered_map<uint64_t, uint64_t> m;
};

uint64_t key_at(const void* keys, int kb, uint64_t i) {
  return kb == 4 ? static_cast<const uint32_t*>(keys)[i] : static_cast<const uint64_t*>(keys)[i];
}

bool sentinel_w(uint64_t k, int kb) { return k == 0 || k == (kb == 4 ? 0xffffffffull : ~0ull); }

}  // namespace

extern "C" {

void* oracle_counts_create(int key_bytes, int is_set) {
  if (key_bytes != 4 && key_bytes != 8) return nullptr;
  return new Counts{key_bytes, is_set != 0, {}};
}

void oracle_counts_destroy(void* p) { delete static_cast<Counts*>(p); }

uint32_t oracle_counts_add(void* p, const void* keys, const void* weights, uint64_t n) {
  auto* c = static_cast<Counts*>(p);
  const uint64_t mask = c->kb == 4 ? 0xffffffffull : ~0ull;
  uint32_t f = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t k = key_at(keys, c->kb, i);
    if (sentinel_w(k, c->kb)) { f |= F_INVALID; continue; }
    auto it = c->m.find(k);
    if (c->set) {
      if (it != c->m.end()) f |= F_DUPLICATE;
      else c->m.emplace(k, 0);
      continue;
    }
    const uint64_t w = weights ? key_at(weights, c->kb, i) : 1;
    if (it == c->m.end()) c->m.emplace(k, w & mask);
    else it->second = (it->second + w) & mask;
  }
  return f;
}

uint32_t oracle_counts_get(void* p, const void* keys, uint64_t n, void* out, uint8_t* found) {
  auto* c = static_cast<Counts*>(p);
  uint32_t f = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t k = key_at(keys, c->kb, i);
    if (sentinel_w(k, c->kb)) f |= F_INVALID;
    auto it = sentinel_w(k, c->kb) ? c->m.end() : c->m.find(k);
    const bool hit = it != c->m.end();
    const uint64_t v = hit ? it->second : ~0ull;
    if (out) {
      if (c->kb == 4) static_cast<uint32_t*>(out)[i] = static_cast<uint32_t>(v);
      else static_cast<uint64_t*>(out)[i] = v;
    }
    if (found) found[i] = hit ? 1 : 0;
  }
  return f;
}

uint32_t oracle_counts_erase(void* p, const void* keys, uint64_t n) {
  auto* c = static_cast<Counts*>(p);
  uint32_t f = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t k = key_at(keys, c->kb, i);
    if (sentinel_w(k, c->kb)) { f |= F_INVALID; continue; }
    c->m.erase(k);
  }
  return f;
}

uint64_t oracle_counts_size(void* p) { return static_cast<Counts*>(p)->m.size(); }

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Slot-dump invariant checker (layout, not values).  Given a host copy of a table's slot
// array it checks the two properties that make the early exit of Sec. IV-B4 correct:
//   * reachability: walking a live key's probing sequence window by window, the window
//     holding it comes no later than the first window that holds an empty slot (a slot
//     only moves empty -> key -> tombstone -> key, so nothing may sit behind an empty
//     window of its own sequence);
//   * uniqueness (single-value tables and key stores, Sec. IV: each key occurs once);
//   * with the table's overflow bits (optional; eight per window, one byte per window, bit
//     g = the key's tag, the low three bits of h below): every window a live key's sequence
//     passes before the key's own window has the bit of the key's tag set, since lookups
//     stop at a window without the key, without an empty slot and with that bit clear.
// The probing sequence is the table's definition restated here: h = fmix64(key ^ seed)
// (MurmurHash3's 64-bit finalizer), w_0 = floor(hi32(h) * p / 2^32),
// step = 1 + floor(lo32(h) * (p - 1) / 2^32), w_{j+1} = (w_j + step) mod p; windows are
// W consecutive slots.  The key is the first key_bytes of a slot (little-endian): 4-byte
// keys in 4- or 8-byte slots, 8-byte keys in 8- or 16-byte slots; empty = 0, tombstone =
// all ones of the key width.
namespace {

uint64_t chk_fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

uint64_t chk_key(const unsigned char* slots, uint64_t i, uint32_t slot_bytes, uint32_t key_bytes) {
  if (key_bytes == 4) {
    uint32_t k;
    std::memcpy(&k, slots + i * slot_bytes, 4);
    return k;
  }
  uint64_t k;
  std::memcpy(&k, slots + i * slot_bytes, 8);
  return k;
}

}  // namespace

extern "C" int oracle_check_slots(const void* dump, uint64_t p, uint32_t W, uint32_t slot_bytes, uint32_t key_bytes,
                                  uint64_t seed, int unique_keys, const uint8_t* ovf_or_null, uint64_t* out_live,
                                  uint64_t* out_dups, uint64_t* out_unreachable) {
  const bool shape_ok = (key_bytes == 4 && (slot_bytes == 4 || slot_bytes == 8)) ||
                        (key_bytes == 8 && (slot_bytes == 8 || slot_bytes == 16));
  if (dump == nullptr || p < 2 || W == 0 || !shape_ok) return -1;
  const unsigned char* s = static_cast<const unsigned char*>(dump);
  const uint64_t cap = p * W;
  const uint64_t tomb = key_bytes == 4 ? 0xffffffffull : ~0ull;
  std::vector<uint8_t> has_empty(p, 0);
  for (uint64_t i = 0; i < cap; ++i)
    if (chk_key(s, i, slot_bytes, key_bytes) == 0) has_empty[i / W] = 1;
  std::unordered_map<uint64_t, uint64_t> seen;
  uint64_t live = 0, dups = 0, unreachable = 0;
  for (uint64_t i = 0; i < cap; ++i) {
    const uint64_t k = chk_key(s, i, slot_bytes, key_bytes);
    if (k == 0 || k == tomb) continue;
    ++live;
    if (unique_keys && seen[k]++ > 0) ++dups;
    const uint64_t h = chk_fmix64(k ^ seed);
    uint64_t w = ((h >> 32) * p) >> 32;
    const uint64_t step = 1 + (((h & 0xffffffffull) * (p - 1)) >> 32);
    const unsigned tag = static_cast<unsigned>(h & 7u);
    const uint64_t home = i / W;
    bool ok = false;
    for (uint64_t j = 0; j < p; ++j) {
      if (w == home) { ok = true; break; }
      if (has_empty[w]) break;
      if (ovf_or_null != nullptr && !((ovf_or_null[w] >> tag) & 1u)) break;
      w = (w + step) % p;
    }
    if (!ok) ++unreachable;
  }
  if (out_live) *out_live = live;
  if (out_dups) *out_dups = dups;
  if (out_unreachable) *out_unreachable = unreachable;
  return 0;
}

// The overflow bits a table filled by inserts alone must hold: an insert sets bit tag(k) of
// every window it walks past, and walks past exactly the windows of its sequence before the
// one it is stored in, so the bits are the union over live keys of those windows' tag bits.
// out_bits: p bytes, one per window.  Keys that no walk reaches are skipped.
extern "C" int oracle_overflow_bits_of(const void* dump, uint64_t p, uint32_t W, uint32_t slot_bytes,
                                       uint32_t key_bytes, uint64_t seed, uint8_t* out_bits) {
  const bool shape_ok = (key_bytes == 4 && (slot_bytes == 4 || slot_bytes == 8)) ||
                        (key_bytes == 8 && (slot_bytes == 8 || slot_bytes == 16));
  if (dump == nullptr || out_bits == nullptr || p < 2 || W == 0 || !shape_ok) return -1;
  const unsigned char* s = static_cast<const unsigned char*>(dump);
  const uint64_t tomb = key_bytes == 4 ? 0xffffffffull : ~0ull;
  std::memset(out_bits, 0, p);
  std::vector<uint64_t> passed;
  for (uint64_t i = 0; i < p * W; ++i) {
    const uint64_t k = chk_key(s, i, slot_bytes, key_bytes);
    if (k == 0 || k == tomb) continue;
    const uint64_t h = chk_fmix64(k ^ seed);
    uint64_t w = ((h >> 32) * p) >> 32;
    const uint64_t step = 1 + (((h & 0xffffffffull) * (p - 1)) >> 32);
    passed.clear();
    bool ok = false;
    for (uint64_t j = 0; j < p; ++j) {
      if (w == i / W) { ok = true; break; }
      passed.push_back(w);
      w = (w + step) % p;
    }
    if (ok)
      for (uint64_t v : passed) out_bits[v] |= static_cast<uint8_t>(1u << (h & 7u));
  }
  return 0;
}

// Walk lengths on a slot dump (hash-quality statistics): for every live key, the number
// of windows its probing sequence visits up to and including the one that holds it; for
// every key of `absent` (keys not in the table), the number of windows a lookup visits
// before it may stop -- up to and including the first window holding an empty slot, or,
// with the overflow bits given, the first window that holds an empty slot or has the bit
// of the key's tag clear.  out[0..3] = sum over live keys, live keys counted, sum over
// absent keys, absent keys counted (keys whose walk never ends are left out of the sums).
extern "C" int oracle_walk_stats(const void* dump, uint64_t p, uint32_t W, uint32_t slot_bytes, uint32_t key_bytes,
                                 uint64_t seed, const uint8_t* ovf_or_null, const void* absent, uint64_t n_absent,
                                 uint64_t* out) {
  const bool shape_ok = (key_bytes == 4 && (slot_bytes == 4 || slot_bytes == 8)) ||
                        (key_bytes == 8 && (slot_bytes == 8 || slot_bytes == 16));
  if (dump == nullptr || out == nullptr || p < 2 || W == 0 || !shape_ok || (n_absent > 0 && absent == nullptr))
    return -1;
  const unsigned char* s = static_cast<const unsigned char*>(dump);
  const uint64_t tomb = key_bytes == 4 ? 0xffffffffull : ~0ull;
  std::vector<uint8_t> has_empty(p, 0);
  for (uint64_t i = 0; i < p * W; ++i)
    if (chk_key(s, i, slot_bytes, key_bytes) == 0) has_empty[i / W] = 1;
  uint64_t hit_sum = 0, hits = 0, miss_sum = 0, misses = 0;
  for (uint64_t i = 0; i < p * W; ++i) {
    const uint64_t k = chk_key(s, i, slot_bytes, key_bytes);
    if (k == 0 || k == tomb) continue;
    const uint64_t h = chk_fmix64(k ^ seed);
    uint64_t w = ((h >> 32) * p) >> 32;
    const uint64_t step = 1 + (((h & 0xffffffffull) * (p - 1)) >> 32);
    for (uint64_t j = 0; j < p; ++j) {
      if (w == i / W) {
        hit_sum += j + 1;
        ++hits;
        break;
      }
      w = (w + step) % p;
    }
  }
  for (uint64_t a = 0; a < n_absent; ++a) {
    uint64_t k;
    if (key_bytes == 4) {
      uint32_t k32;
      std::memcpy(&k32, static_cast<const unsigned char*>(absent) + a * 4, 4);
      k = k32;
    } else {
      std::memcpy(&k, static_cast<const unsigned char*>(absent) + a * 8, 8);
    }
    const uint64_t h = chk_fmix64(k ^ seed);
    uint64_t w = ((h >> 32) * p) >> 32;
    const uint64_t step = 1 + (((h & 0xffffffffull) * (p - 1)) >> 32);
    const unsigned tag = static_cast<unsigned>(h & 7u);
    for (uint64_t j = 0; j < p; ++j) {
      if (has_empty[w] || (ovf_or_null != nullptr && !((ovf_or_null[w] >> tag) & 1u))) {
        miss_sum += j + 1;
        ++misses;
        break;
      }
      w = (w + step) % p;
    }
  }
  out[0] = hit_sum;
  out[1] = hits;
  out[2] = miss_sum;
  out[3] = misses;
  return 0;
}

// A single-value table of packed 4+4-byte slots built by the paper's insertion applied to
// one key at a time (Sec. IV-B2: walk the key's windows, store the pair in the lowest empty
// slot of the first window that has one), with the overflow bits such an insert sets (bit
// tag(k) of every window it walks past).  Distinct keys, no erases.  out_slots: p * W
// packed words (key | value << 32); out_bits: p bytes.  Returns the number of keys that
// found no slot (0 below a full table).  Sequential order is one of the orders a parallel
// insert may produce; walk statistics of such tables predict those of the GPU's.
extern "C" int64_t oracle_build_packed_table(const uint32_t* keys, const uint32_t* vals, uint64_t n, uint64_t p,
                                             uint32_t W, uint64_t seed, uint64_t* out_slots, uint8_t* out_bits) {
  if (keys == nullptr || out_slots == nullptr || out_bits == nullptr || p < 2 || W == 0) return -1;
  std::memset(out_slots, 0, p * W * sizeof(uint64_t));
  std::memset(out_bits, 0, p);
  int64_t failed = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t k = keys[i];
    const uint64_t h = chk_fmix64(k ^ seed);
    uint64_t w = ((h >> 32) * p) >> 32;
    const uint64_t step = 1 + (((h & 0xffffffffull) * (p - 1)) >> 32);
    bool stored = false;
    for (uint64_t j = 0; j < p && !stored; ++j) {
      for (uint32_t q = 0; q < W; ++q) {
        uint64_t& slot = out_slots[w * W + q];
        if (static_cast<uint32_t>(slot) == 0) {
          slot = k | (static_cast<uint64_t>(vals ? vals[i] : 0) << 32);
          stored = true;
          break;
        }
      }
      if (!stored) {
        out_bits[w] |= static_cast<uint8_t>(1u << (h & 7u));
        w = (w + step) % p;
      }
    }
    if (!stored) ++failed;
  }
  return failed;
}

// ---------------------------------------------------------------------------------------
// Blocked Bloom filter (Sec. IV, "BloomFilter": set membership with false positives), by
// the definition the library documents: h = fmix64(key ^ seed); the key's block is
// floor(hi32(h) * blocks / 2^32) of `blocks` 256-bit blocks; its k bit positions are the
// bytes of g1 = fmix64(h ^ 0x9e3779b97f4a7c15), g2 = fmix64(g1), ... (position i = byte
// i % 8 of g_{i / 8 + 1}).  Insert sets the bits; a key is reported present when all of
// its bits are set.
namespace {

struct Bloom {
  int kb, k;
  uint64_t blocks, seed;
  std::vector<uint8_t> bits;  // blocks * 256 bits, one byte per bit
};

uint64_t bloom_fmix64(uint64_t x) { return chk_fmix64(x); }

void bloom_bits(const Bloom& b, uint64_t key, uint64_t* block, uint32_t* pos) {
  const uint64_t h = bloom_fmix64(key ^ b.seed);
  *block = ((h >> 32) * b.blocks) >> 32;
  uint64_t g = h ^ 0x9e3779b97f4a7c15ull;
  for (int i = 0; i < b.k; ++i) {
    if (i % 8 == 0) g = bloom_fmix64(g);
    pos[i] = static_cast<uint32_t>((g >> (8 * (i % 8))) & 255u);
  }
}

}  // namespace

extern "C" {

void* oracle_bloom_create(int key_bytes, uint64_t blocks, int k, uint64_t seed) {
  if ((key_bytes != 4 && key_bytes != 8) || blocks == 0 || k < 1 || k > 16) return nullptr;
  return new Bloom{key_bytes, k, blocks, seed, std::vector<uint8_t>(blocks * 256, 0)};
}

void oracle_bloom_destroy(void* p) { delete static_cast<Bloom*>(p); }

uint32_t oracle_bloom_insert(void* p, const void* keys, uint64_t n) {
  auto* b = static_cast<Bloom*>(p);
  uint32_t f = 0;
  uint32_t pos[16];
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t key = key_at(keys, b->kb, i);
    if (sentinel_w(key, b->kb)) { f |= F_INVALID; continue; }
    uint64_t blk;
    bloom_bits(*b, key, &blk, pos);
    for (int j = 0; j < b->k; ++j) b->bits[blk * 256 + pos[j]] = 1;
  }
  return f;
}

uint32_t oracle_bloom_contains(void* p, const void* keys, uint64_t n, uint8_t* found) {
  auto* b = static_cast<Bloom*>(p);
  uint32_t f = 0;
  uint32_t pos[16];
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t key = key_at(keys, b->kb, i);
    if (sentinel_w(key, b->kb)) { f |= F_INVALID; found[i] = 0; continue; }
    uint64_t blk;
    bloom_bits(*b, key, &blk, pos);
    bool all = true;
    for (int j = 0; j < b->k; ++j) all = all && b->bits[blk * 256 + pos[j]];
    found[i] = all ? 1 : 0;
  }
  return f;
}

}  // extern "C"
