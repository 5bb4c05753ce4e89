// The C ABI of include/wc.h: table lifecycle, geometry planning, argument checks and
// dispatch to the kernel families.  Host code only.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "wc.h"
#include "wc_internal.h"
#include "wc_tune.h"

namespace wc {

bool sv_p32_shape_ok(int W, int G);
bool sv_p64_shape_ok(int W, int G);
bool mv_shape_ok(int W, int G);
bool oa_p32_shape_ok(int W, int G);
bool count_shape_ok(int slot_bytes, int W, int G);
bool soa_shape_ok(int slot_bytes, int W, int G);
cudaError_t soa_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                       uint8_t* found, cudaStream_t s);
bool set_shape_ok(int slot_bytes, int W, int G);
cudaError_t set_launch(const wc_table* t, int op, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s);
cudaError_t bloom_launch(const wc_table* t, int op, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s);
cudaError_t count_insert(const wc_table* t, const void* keys, const void* weights, uint64_t n, cudaStream_t s);
bool oa_p64_shape_ok(int W, int G);
cudaError_t oa_p32_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, uint64_t* offs,
                          void* out, cudaStream_t s);
cudaError_t oa_p64_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, uint64_t* offs,
                          void* out, cudaStream_t s);
cudaError_t oa_p32_num_keys(const wc_table* t, cudaStream_t s);
cudaError_t oa_p64_num_keys(const wc_table* t, cudaStream_t s);
cudaError_t sv_p32_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                          uint8_t* found, cudaStream_t s);
cudaError_t sv_p64_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                          uint8_t* found, cudaStream_t s);

namespace {

constexpr uint64_t kAlign = 256;
constexpr uint64_t kMaxPool = 1ull << 35;
constexpr uint64_t kMaxBatch = (1ull << 32) - 1;
constexpr uint64_t kMaxMvBatch = 1ull << 31;  // per-call counts must stay below the poison bit
constexpr uint64_t kMaxCountHost = (1ull << 28) - 1;  // values per multi-value key

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Trial division: exact for every 64-bit input, fast for the < 2^32 range used here.
bool is_prime(uint64_t x) {
  if (x < 2) return false;
  if (x % 2 == 0) return x == 2;
  if (x % 3 == 0) return x == 3;
  for (uint64_t d = 5; d * d <= x; d += 6)
    if (x % d == 0 || x % (d + 2) == 0) return false;
  return true;
}

uint64_t next_prime(uint64_t x) {
  if (x <= 2) return 2;
  uint64_t c = x | 1;
  while (!is_prime(c)) c += 2;
  return c;
}

bool slot_layout(const wc_table_config& c, uint64_t* slot_bytes) {
  if (c.kind == WC_SINGLE_VALUE && (c.options & WC_OPT_SOA)) {  // key array; values in a second array
    if ((c.key_bytes == 4 && c.value_bytes == 4) || (c.key_bytes == 8 && c.value_bytes == 8)) {
      *slot_bytes = static_cast<uint64_t>(c.key_bytes);
      return true;
    }
    return false;
  }
  if (c.kind == WC_SINGLE_VALUE || c.kind == WC_MULTI_VALUE_OA || c.kind == WC_COUNTING) {
    if (c.key_bytes == 4 && c.value_bytes == 4) { *slot_bytes = 8; return true; }
    if (c.key_bytes == 8 && c.value_bytes == 8) { *slot_bytes = 16; return true; }
    return false;
  }
  if (c.kind == WC_HASH_SET) {
    if ((c.key_bytes == 4 || c.key_bytes == 8) && c.value_bytes == 0) {
      *slot_bytes = static_cast<uint64_t>(c.key_bytes);
      return true;
    }
    return false;
  }
  if (c.kind == WC_BLOOM_FILTER) {  // one 256-bit block per "slot"
    if ((c.key_bytes == 4 || c.key_bytes == 8) && c.value_bytes == 0) {
      *slot_bytes = 32;
      return true;
    }
    return false;
  }
  if (c.kind == WC_MULTI_VALUE) {
    if ((c.key_bytes == 4 || c.key_bytes == 8) && (c.value_bytes == 4 || c.value_bytes == 8)) {
      *slot_bytes = 16;
      return true;
    }
  }
  return false;
}

bool window_ok(int kind, uint64_t slot_bytes, int W) {
  if (kind == WC_MULTI_VALUE) return W == 2 || W == 4 || W == 8;
  if (slot_bytes == 4) return W == 8 || W == 16 || W == 32;
  if (slot_bytes == 8) return W == 4 || W == 8 || W == 16 || W == 32;
  return W == 2 || W == 4 || W == 8 || W == 16;
}

bool shape_ok(const wc_table* t, int op, int G) {
  const int W = static_cast<int>(t->W);
  if (t->cfg.kind == WC_MULTI_VALUE_OA) return t->slot_bytes == 8 ? oa_p32_shape_ok(W, G) : oa_p64_shape_ok(W, G);
  if (t->cfg.kind == WC_COUNTING && op == WC_OP_INSERT) return count_shape_ok(static_cast<int>(t->slot_bytes), W, G);
  if (t->cfg.kind == WC_HASH_SET) return set_shape_ok(static_cast<int>(t->slot_bytes), W, G);
  if (t->d_vals != nullptr) return soa_shape_ok(static_cast<int>(t->slot_bytes), W, G);
  if (t->slot_bytes == 8) return sv_p32_shape_ok(W, G);
  if (t->cfg.kind == WC_MULTI_VALUE) {
    if (op == WC_OP_INSERT || op == WC_OP_RETRIEVE) return G == 1;  // one thread per distinct key
    return mv_shape_ok(W, G);
  }
  return sv_p64_shape_ok(W, G);
}

// Default lanes per key, from launch-shape sweeps on GB300 (2^27 keys at load 0.9):
// probes are bound by random HBM traffic (direct) or by L2 round trips (blocked), so the
// shapes that keep the most keys in flight win.  Inserts use one lane per key (the
// blocked scheme's L2-resident probes favour it); lookups use 32 bytes of the window per
// lane (one 256-bit load).
int default_group(uint64_t slot_bytes, int W, int op) {
  if (op == WC_OP_INSERT && static_cast<uint64_t>(W) * slot_bytes <= 64) return 1;
  const int per_lane = static_cast<int>(32 / slot_bytes);
  return std::max(1, W / per_lane);
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

bool aligned(const void* p, uint64_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Testing hook (wc_debug_fail_allocations): allocations still to fail on purpose.
std::atomic<uint32_t> g_fail_allocs{0};

bool injected_alloc_failure() {
  uint32_t c = g_fail_allocs.load();
  while (c > 0)
    if (g_fail_allocs.compare_exchange_weak(c, c - 1)) return true;
  return false;
}

}  // namespace

TableDesc desc_of(const wc_table* t) {
  TableDesc d;
  d.slots = t->d_slots;
  d.seed = t->cfg.seed;
  d.status = t->d_status;
  d.size = t->d_size;
  d.nkeys = t->d_nkeys;
  d.ovf = t->d_ovf;
  d.vals = t->d_vals;
  d.p = static_cast<uint32_t>(t->windows);
  d.W = static_cast<uint32_t>(t->W);
  return d;
}

PoolDesc pool_of(const wc_table* t) {
  PoolDesc p;
  p.pool = t->d_pool;
  p.cursor = t->d_cursor;
  p.pending = t->d_pending;
  p.capacity = t->pool_capacity;
  p.value_bytes = t->cfg.value_bytes;
  p.growth = t->growth;
  p.nbuckets = t->nbuckets;
  p.s0 = t->cfg.bucket_first_size;
  p.foot0 = t->grow_foot0;
  p.foot = t->grow_foot;
  p.cum_size = t->d_growth;
  p.cum_foot = t->d_growth ? t->d_growth + t->nbuckets : nullptr;
  p.base = t->d_base;
  return p;
}

namespace {

// Bucket sizes of the growth strategy (Sec. IV-C): s_0 = s0, s_i = ceil(lambda * s_{i-1}).
// A product within a relative 1e-9 of an integer counts as that integer, so decimal
// factors such as 1.1 (not exact in binary) give the sizes their decimal value gives.
uint64_t next_bucket_size(double lambda, uint64_t s) {
  const double x = lambda * static_cast<double>(s);
  const double c = std::ceil(x - 1e-9 * x);
  return std::max<uint64_t>(s, static_cast<uint64_t>(c));
}

// Pool elements of bucket i: values plus (for i > 0) the header holding the previous
// handle, rounded to whole 8-byte words for 4-byte values.
uint64_t bucket_foot(uint64_t i, uint64_t s, int value_bytes) {
  const uint64_t e = s + (i ? 8u / static_cast<uint64_t>(value_bytes) : 0);
  return value_bytes == 4 ? (e + 1) & ~1ull : e;
}

}  // namespace

cudaLaunchAttribute* l2_attr(const wc_table* t, cudaLaunchAttribute* storage, unsigned* count) {
  if (t == nullptr || t->l2_window_bytes == 0) {
    *count = 0;
    return nullptr;
  }
  storage[0].id = cudaLaunchAttributeAccessPolicyWindow;
  storage[0].val.accessPolicyWindow.base_ptr = t->d_slots;
  storage[0].val.accessPolicyWindow.num_bytes = t->l2_window_bytes;
  storage[0].val.accessPolicyWindow.hitRatio = t->l2_hit_ratio;
  storage[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  storage[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  *count = 1;
  return storage;
}

int occupancy_cached(const void* kernel, int block, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(kernel, block, smem, dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, smem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cache[key] = nb;
  return nb;
}

cudaError_t ensure_scratch(const wc_table* t, uint64_t bytes, cudaStream_t s) {
  if (bytes <= t->scratch_bytes) return cudaSuccess;
  if (t->d_scratch != nullptr) {
    cudaError_t e = cudaFreeAsync(t->d_scratch, s);
    if (e != cudaSuccess) return e;
    t->d_scratch = nullptr;
    t->scratch_bytes = 0;
  }
  const uint64_t want = align_up(bytes + bytes / 8, kAlign);
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMallocAsync(&t->d_scratch, want, s);
  if (e != cudaSuccess) {
    t->d_scratch = nullptr;
    return e;
  }
  t->scratch_bytes = want;
  return cudaSuccess;
}

int scheme_for(const wc_table* t, int op, uint64_t n) {
  const int sc = t->launch[op].scheme;
  if (sc != WC_SCHEME_AUTO) return sc;
  if (op == WC_OP_INSERT && t->cfg.kind != WC_MULTI_VALUE && n >= (1ull << 18) && t->table_bytes > (64ull << 20))
    return WC_SCHEME_BLOCKED;
  return WC_SCHEME_DIRECT;
}

int sm_count_of(int device) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n < 1) n = 1;
  return n;
}

cudaError_t sv_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                      uint8_t* found, cudaStream_t s) {
  if (t->d_vals != nullptr) return soa_launch(t, op, keys, vals, n, out, found, s);
  if (t->slot_bytes == 8) return sv_p32_launch(t, op, keys, vals, n, out, found, s);
  return sv_p64_launch(t, op, keys, vals, n, out, found, s);
}

cudaError_t oa_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, uint64_t* offs,
                      void* out, cudaStream_t s) {
  if (t->slot_bytes == 8) return oa_p32_launch(t, op, keys, vals, n, offs, out, s);
  return oa_p64_launch(t, op, keys, vals, n, offs, out, s);
}

}  // namespace wc

using namespace wc;

extern "C" {

const char* wc_status_string(wc_status s) {
  switch (s) {
    case WC_OK: return "ok";
    case WC_ERR_INVALID_ARG: return "invalid argument";
    case WC_ERR_OUT_OF_MEMORY: return "out of device memory";
    case WC_ERR_FULL: return "table full (probe limit reached)";
    case WC_ERR_CUDA: return "CUDA runtime error";
    case WC_ERR_TIMEOUT: return "bounded device wait timed out";
    case WC_ERR_UNSUPPORTED: return "operation not supported for this table kind";
  }
  return "unknown status";
}

wc_status wc_debug_fail_allocations(uint32_t count) {
  g_fail_allocs.store(count);
  return WC_OK;
}

wc_status wc_plan_capacity(uint64_t min_capacity, int32_t window_width, uint64_t* h_windows,
                           uint64_t* h_capacity) {
  if (window_width < 1 || window_width > 64 || h_windows == nullptr || h_capacity == nullptr)
    return WC_ERR_INVALID_ARG;
  const uint64_t W = static_cast<uint64_t>(window_width);
  const uint64_t want = std::max<uint64_t>(1, (min_capacity + W - 1) / W);
  if (want >= (1ull << 32)) return WC_ERR_INVALID_ARG;
  const uint64_t p = next_prime(want);
  if (p >= (1ull << 32)) return WC_ERR_INVALID_ARG;
  *h_windows = p;
  *h_capacity = p * W;
  return WC_OK;
}

// The persisting-L2 carve-out (cudaLimitPersistingL2CacheSize) is a limit of the device's
// context, shared by every table with l2_persist.  The first such table on a device
// records the limit it found; when the last one is destroyed, the persisting lines are
// turned back into normal ones and the limit is put back, so later work in the process
// gets the whole L2 again.
namespace {
std::mutex g_l2_mu;
struct L2Hold {
  int tables = 0;
  size_t before = 0;
};
L2Hold g_l2_hold[64];
}  // namespace

static void l2_carveout_hold(wc_table* t, size_t limit_now) {
  if (t->device < 0 || t->device >= 64) return;
  std::lock_guard<std::mutex> lock(g_l2_mu);
  if (g_l2_hold[t->device].tables++ == 0) g_l2_hold[t->device].before = limit_now;
  t->l2_held = true;
}

static void l2_carveout_release(wc_table* t) {
  if (!t->l2_held) return;
  std::lock_guard<std::mutex> lock(g_l2_mu);
  t->l2_held = false;
  if (--g_l2_hold[t->device].tables > 0) return;
  cudaDeviceSynchronize();  // no kernel of this table still reads with the window
  cudaCtxResetPersistingL2Cache();
  cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_hold[t->device].before);
  cudaGetLastError();
}

wc_status wc_table_create(wc_table** out, const wc_table_config* cfg) {
  if (out == nullptr || cfg == nullptr) return WC_ERR_INVALID_ARG;
  *out = nullptr;
  uint64_t slot_bytes = 0;
  if (!slot_layout(*cfg, &slot_bytes)) return WC_ERR_INVALID_ARG;
  const bool bloom = cfg->kind == WC_BLOOM_FILTER;
  int W = cfg->window_width;
  int bloom_k = 0;
  wc_tuning tuning;
  bool tuned = false;
  if (bloom) {  // window_width carries k, the bits per key; a block is the unit of probing
    bloom_k = W == 0 ? 8 : W;
    if (bloom_k < 1 || bloom_k > 16) return WC_ERR_INVALID_ARG;
    W = 1;
  } else if (W == 0) {
    // autotuned (wc_tune.h) for the kinds the single-value engine serves in packed slots,
    // else (or when tuning is off or fails) the 64-byte window
    const bool tunable = (cfg->kind == WC_SINGLE_VALUE || cfg->kind == WC_COUNTING || cfg->kind == WC_HASH_SET) &&
                         !(cfg->options & WC_OPT_SOA);
    if (tunable && autotune_enabled() &&
        wc_autotune(cfg, 0.9, autotune_sample_for(*cfg), 1, &tuning) == WC_OK)
      tuned = true;
    W = tuned ? tuning.window_width : static_cast<int>(64 / slot_bytes);
    if (!window_ok(cfg->kind, slot_bytes, W)) return WC_ERR_INVALID_ARG;
  } else {
    if (!window_ok(cfg->kind, slot_bytes, W)) return WC_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return WC_ERR_CUDA;
  const bool mv = cfg->kind == WC_MULTI_VALUE;
  const bool oa = cfg->kind == WC_MULTI_VALUE_OA;
  if ((cfg->options & ~(WC_OPT_OVERFLOW_BITS | WC_OPT_SOA)) != 0 || cfg->reserved != 0) return WC_ERR_INVALID_ARG;
  if ((cfg->options & WC_OPT_SOA) && cfg->kind != WC_SINGLE_VALUE) return WC_ERR_INVALID_ARG;
  const bool soa = (cfg->options & WC_OPT_SOA) != 0;
  // bucket growth strategy (bucket multi-value tables)
  int growth = kGrowExact;
  std::vector<uint64_t> cum_size, cum_foot;
  uint64_t foot0 = 0, foot = 0;
  if (cfg->bucket_first_size != 0) {
    const double lam = cfg->bucket_growth;
    if (!mv || !(lam >= 1.0) || !(lam <= 1e6) || cfg->bucket_first_size > kMaxCountHost) return WC_ERR_INVALID_ARG;
    const uint64_t s0 = cfg->bucket_first_size;
    if (lam == 1.0) {
      growth = kGrowConst;
      foot0 = bucket_foot(0, s0, cfg->value_bytes);
      foot = bucket_foot(1, s0, cfg->value_bytes);
    } else {
      growth = kGrowTable;
      uint64_t s = s0, S = 0, F = 0;
      for (uint64_t i = 0;; ++i) {
        if (i >= kMaxGrowBuckets) return WC_ERR_INVALID_ARG;
        S += s;
        F += bucket_foot(i, s, cfg->value_bytes);
        cum_size.push_back(S);
        cum_foot.push_back(F);
        if (S >= kMaxCountHost) break;
        s = std::min<uint64_t>(next_bucket_size(lam, s), kMaxCountHost);
      }
    }
  }
  if ((cfg->options & WC_OPT_OVERFLOW_BITS) && cfg->kind != WC_SINGLE_VALUE && cfg->kind != WC_COUNTING &&
      cfg->kind != WC_HASH_SET)
    return WC_ERR_INVALID_ARG;
  if (mv && cfg->value_pool_capacity > kMaxPool) return WC_ERR_INVALID_ARG;

  uint64_t p = 0, cap = 0;
  const uint64_t want = bloom ? (cfg->min_capacity + 255) / 256 : cfg->min_capacity;  // Bloom: bits -> blocks
  if (wc_plan_capacity(want, W, &p, &cap) != WC_OK) return WC_ERR_INVALID_ARG;

  wc_table* t = new (std::nothrow) wc_table();
  if (t == nullptr) return WC_ERR_OUT_OF_MEMORY;
  t->cfg = *cfg;
  t->cfg.window_width = bloom ? bloom_k : W;
  t->device = cfg->device;
  t->windows = p;
  t->W = static_cast<uint64_t>(W);
  t->capacity = cap;
  t->slot_bytes = slot_bytes;
  t->table_bytes = cap * slot_bytes;
  const uint64_t soa_vals_off = align_up(t->table_bytes, kAlign);  // SoA: the value array follows the keys
  if (soa) t->table_bytes = soa_vals_off + cap * static_cast<uint64_t>(cfg->value_bytes);
  t->pool_capacity = mv ? cfg->value_pool_capacity : 0;

  DeviceGuard guard(t->device);
  t->sm_count = sm_count_of(t->device);

  // One allocation: [slots | meta 256 B | overflow bits (SV) | pending (MV) | scan partials (MV, OA) | pool (MV)]
  const bool sv = (cfg->kind == WC_SINGLE_VALUE || cfg->kind == WC_COUNTING || cfg->kind == WC_HASH_SET) &&
                  (cfg->options & WC_OPT_OVERFLOW_BITS);
  const uint64_t off_meta = align_up(t->table_bytes, kAlign);
  const uint64_t off_ovf = off_meta + kAlign;
  const uint64_t ovf_bytes = sv ? align_up((p + 3) / 4 * 4, kAlign) : 0;  // one byte per window
  const uint64_t off_pending = off_ovf + ovf_bytes;
  const uint64_t pending_bytes = mv ? align_up(cap * 4, kAlign) : 0;
  const uint64_t off_base = off_pending + pending_bytes;
  const uint64_t base_bytes = growth != kGrowExact ? align_up(cap * 4, kAlign) : 0;
  const uint64_t off_partials = off_base + base_bytes;
  t->partials_cap = mv || oa ? scan_partials_needed(kMaxBatch + 1) : 0;
  const uint64_t partial_bytes = align_up(t->partials_cap * 8, kAlign);
  const uint64_t off_pool = off_partials + partial_bytes;
  const uint64_t pool_bytes = align_up(t->pool_capacity * static_cast<uint64_t>(cfg->value_bytes), kAlign);
  const uint64_t off_growth = off_pool + pool_bytes;
  t->device_bytes = off_growth + align_up(cum_size.size() * 16, kAlign);
  t->growth = growth;
  t->nbuckets = static_cast<uint32_t>(cum_size.size());
  t->grow_foot0 = foot0;
  t->grow_foot = foot;

  if (injected_alloc_failure() || cudaMalloc(&t->d_block, t->device_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete t;
    return WC_ERR_OUT_OF_MEMORY;
  }
  char* base = static_cast<char*>(t->d_block);
  t->d_slots = base;
  t->d_status = reinterpret_cast<uint32_t*>(base + off_meta);
  t->d_size = reinterpret_cast<unsigned long long*>(base + off_meta + 8);
  t->d_nkeys = reinterpret_cast<unsigned long long*>(base + off_meta + 16);
  t->d_cursor = reinterpret_cast<unsigned long long*>(base + off_meta + 24);
  t->d_ovf = sv ? reinterpret_cast<uint32_t*>(base + off_ovf) : nullptr;
  t->d_vals = soa ? static_cast<void*>(base + soa_vals_off) : nullptr;
  t->d_pending = mv ? reinterpret_cast<uint32_t*>(base + off_pending) : nullptr;
  t->d_base = growth != kGrowExact ? reinterpret_cast<uint32_t*>(base + off_base) : nullptr;
  t->d_growth = growth == kGrowTable ? reinterpret_cast<uint64_t*>(base + off_growth) : nullptr;
  t->d_partials = mv || oa ? reinterpret_cast<uint64_t*>(base + off_partials) : nullptr;
  t->d_pool = mv ? static_cast<void*>(base + off_pool) : nullptr;

  for (int op = 0; op < WC_OP__N; ++op) {
    t->launch[op].group_size = default_group(slot_bytes, W, op);
    t->launch[op].block_threads = 256;
    t->launch[op].blocks_per_sm = 0;
    t->launch[op].scheme = WC_SCHEME_AUTO;
    t->launch[op].region_mib = 0;
    t->launch[op].keys_in_flight = 1;
  }
  // lookups of packed 4+4-byte single-value tables keep two keys per group in flight
  // (2^27 keys at load 0.9: 28.0 against 27.2 G lookups/s; +4 % at loads 0.5 and 0.99)
  if (cfg->kind == WC_SINGLE_VALUE && !soa && slot_bytes == 8) t->launch[WC_OP_RETRIEVE].keys_in_flight = 2;
  if (tuned) {
    for (int op = 0; op < 3; ++op)
      if (shape_ok(t, op, tuning.launch[op].group_size)) t->launch[op] = tuning.launch[op];
  }
  if (mv) {
    t->launch[WC_OP_INSERT].block_threads = 256;
    t->launch[WC_OP_INSERT].group_size = 1;
    t->launch[WC_OP_RETRIEVE].group_size = 1;
  }

  if (cfg->l2_persist) {
    int max_persist = 0, max_window = 0;
    cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, t->device);
    cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, t->device);
    if (max_persist > 0 && max_window > 0) {
      const size_t persist = std::min<size_t>(t->table_bytes, static_cast<size_t>(max_persist));
      size_t cur = 0;
      cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
      l2_carveout_hold(t, cur);
      if (cur < persist) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, persist);
      cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
      t->l2_window_bytes = std::min<size_t>(t->table_bytes, static_cast<size_t>(max_window));
      t->l2_hit_ratio = std::min(1.0f, static_cast<float>(cur) / static_cast<float>(t->l2_window_bytes));
    }
    cudaGetLastError();
  }

  t->clear_bytes = off_partials;
  cudaError_t ge = cudaSuccess;
  if (t->d_growth != nullptr) {
    ge = cudaMemcpy(t->d_growth, cum_size.data(), cum_size.size() * 8, cudaMemcpyHostToDevice);
    if (ge == cudaSuccess)
      ge = cudaMemcpy(t->d_growth + t->nbuckets, cum_foot.data(), cum_foot.size() * 8, cudaMemcpyHostToDevice);
  }
  if (ge != cudaSuccess || cudaMemset(t->d_block, 0, t->clear_bytes) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(t->d_block);
    delete t;
    return WC_ERR_CUDA;
  }
  *out = t;
  return WC_OK;
}

wc_status wc_table_destroy(wc_table* t) {
  if (t == nullptr) return WC_ERR_INVALID_ARG;
  DeviceGuard guard(t->device);
  host_pipe_free(t);
  l2_carveout_release(t);
  if (t->d_scratch != nullptr) {
    cudaDeviceSynchronize();
    cudaFree(t->d_scratch);
  }
  cudaError_t e = cudaFree(t->d_block);
  delete t;
  return cuda_status(e);
}

wc_status wc_table_clear(wc_table* t, void* stream) {
  TraceRange trace("wc_table_clear");
  if (t == nullptr) return WC_ERR_INVALID_ARG;
  DeviceGuard guard(t->device);
  return cuda_status(cudaMemsetAsync(t->d_block, 0, t->clear_bytes, as_stream(stream)));
}

wc_status wc_table_get_info(const wc_table* t, wc_table_info* h_out) {
  if (t == nullptr || h_out == nullptr) return WC_ERR_INVALID_ARG;
  h_out->capacity = t->capacity;
  h_out->windows = t->windows;
  h_out->slot_bytes = t->slot_bytes;
  h_out->table_bytes = t->table_bytes;
  h_out->pool_capacity = t->pool_capacity;
  h_out->device_bytes = t->device_bytes;
  h_out->window_width = t->cfg.kind == WC_BLOOM_FILTER ? t->cfg.window_width : static_cast<int32_t>(t->W);
  h_out->kind = t->cfg.kind;
  h_out->options = t->cfg.options;
  h_out->reserved = 0;
  h_out->work_bytes = t->scratch_bytes + host_pipe_bytes(t);
  return WC_OK;
}

wc_status wc_table_set_launch(wc_table* t, int32_t op, const wc_launch* launch) {
  if (t == nullptr || launch == nullptr || op < 0 || op >= WC_OP__N) return WC_ERR_INVALID_ARG;
  if (t->cfg.kind == WC_BLOOM_FILTER) return WC_ERR_UNSUPPORTED;  // one thread per key
  const int b = launch->block_threads;
  // the bucket table's insert runs its aggregation passes in blocks of 256 or 512 threads
  const bool mv_insert = t->cfg.kind == WC_MULTI_VALUE && op == WC_OP_INSERT;
  if (mv_insert ? (b != 256 && b != 512) : (b < 32 || b > 256 || b % 32 != 0)) return WC_ERR_INVALID_ARG;
  if (launch->blocks_per_sm < 0 || launch->blocks_per_sm > 64) return WC_ERR_INVALID_ARG;
  if (launch->keys_in_flight < 0 || launch->keys_in_flight > 2) return WC_ERR_INVALID_ARG;
  if (launch->scheme < WC_SCHEME_AUTO || launch->scheme > WC_SCHEME_DEDUP || launch->region_mib < 0 ||
      launch->region_mib > 4096)
    return WC_ERR_INVALID_ARG;
  if (launch->scheme == WC_SCHEME_BLOCKED &&
      !((op == WC_OP_INSERT && t->cfg.kind != WC_MULTI_VALUE) ||
        (op == WC_OP_RETRIEVE && (t->cfg.kind == WC_SINGLE_VALUE || t->cfg.kind == WC_COUNTING))))
    return WC_ERR_UNSUPPORTED;
  if (launch->scheme == WC_SCHEME_DEDUP &&
      !(op == WC_OP_RETRIEVE && (t->cfg.kind == WC_SINGLE_VALUE || t->cfg.kind == WC_COUNTING ||
                                 t->cfg.kind == WC_HASH_SET)))
    return WC_ERR_UNSUPPORTED;
  if (!shape_ok(t, op, launch->group_size)) return WC_ERR_INVALID_ARG;
  t->launch[op] = *launch;
  return WC_OK;
}

wc_status wc_table_get_launch(const wc_table* t, int32_t op, wc_launch* h_out) {
  if (t == nullptr || h_out == nullptr || op < 0 || op >= WC_OP__N) return WC_ERR_INVALID_ARG;
  *h_out = t->launch[op];
  return WC_OK;
}

static bool device_accessible(const wc_table* t, const void* p) { return wc::device_accessible(t->device, p); }

static wc_status check_buffer(const wc_table* t, const void* p, uint64_t n, uint64_t align) {
  if (n == 0) return WC_OK;
  if (p == nullptr || !aligned(p, align) || !device_accessible(t, p)) return WC_ERR_INVALID_ARG;
  return WC_OK;
}

static wc_status check_bulk(const wc_table* t, const void* keys, uint64_t n) {
  if (t == nullptr) return WC_ERR_INVALID_ARG;
  if (n > kMaxBatch) return WC_ERR_INVALID_ARG;
  return check_buffer(t, keys, n, static_cast<uint64_t>(t->cfg.key_bytes));
}

wc_status wc_insert(wc_table* t, const void* d_keys, const void* d_values, uint64_t n, void* stream) {
  TraceRange trace("wc_insert");
  wc_status st = check_bulk(t, d_keys, n);
  if (st != WC_OK) return st;
  const bool weights_optional =
      t->cfg.kind == WC_COUNTING || t->cfg.kind == WC_HASH_SET || t->cfg.kind == WC_BLOOM_FILTER;
  if (n > 0 && d_values == nullptr && !weights_optional) return WC_ERR_INVALID_ARG;
  if (d_values != nullptr && (t->cfg.kind == WC_HASH_SET || t->cfg.kind == WC_BLOOM_FILTER)) d_values = nullptr;
  if (d_values != nullptr) {
    st = check_buffer(t, d_values, n, static_cast<uint64_t>(t->cfg.value_bytes));
    if (st != WC_OK) return st;
  }
  if (n == 0) return WC_OK;
  if (t->cfg.kind == WC_COUNTING) {
    DeviceGuard guard(t->device);
    return cuda_status(count_insert(t, d_keys, d_values, n, as_stream(stream)));
  }
  if (t->cfg.kind == WC_HASH_SET || t->cfg.kind == WC_BLOOM_FILTER) {
    DeviceGuard guard(t->device);
    return cuda_status(t->cfg.kind == WC_HASH_SET ? set_launch(t, WC_OP_INSERT, d_keys, n, nullptr, as_stream(stream))
                                                  : bloom_launch(t, WC_OP_INSERT, d_keys, n, nullptr, as_stream(stream)));
  }
  if (t->cfg.kind == WC_MULTI_VALUE && n >= kMaxMvBatch) return WC_ERR_INVALID_ARG;
  DeviceGuard guard(t->device);
  if (t->cfg.kind == WC_MULTI_VALUE) return cuda_status(mv_insert(t, d_keys, d_values, n, as_stream(stream)));
  if (t->cfg.kind == WC_MULTI_VALUE_OA)
    return cuda_status(oa_launch(t, WC_OP_INSERT, d_keys, d_values, n, nullptr, nullptr, as_stream(stream)));
  return cuda_status(sv_launch(t, WC_OP_INSERT, d_keys, d_values, n, nullptr, nullptr, as_stream(stream)));
}

wc_status wc_retrieve(wc_table* t, const void* d_keys, uint64_t n, void* d_values_out, uint8_t* d_found_or_null,
                      void* stream) {
  TraceRange trace("wc_retrieve");
  wc_status st = check_bulk(t, d_keys, n);
  if (st != WC_OK) return st;
  if (t->cfg.kind != WC_SINGLE_VALUE && t->cfg.kind != WC_COUNTING) return WC_ERR_UNSUPPORTED;
  st = check_buffer(t, d_values_out, n, static_cast<uint64_t>(t->cfg.value_bytes));
  if (st == WC_OK && d_found_or_null != nullptr) st = check_buffer(t, d_found_or_null, n, 1);
  if (st != WC_OK) return st;
  if (n == 0) return WC_OK;
  DeviceGuard guard(t->device);
  return cuda_status(
      sv_launch(t, WC_OP_RETRIEVE, d_keys, nullptr, n, d_values_out, d_found_or_null, as_stream(stream)));
}

wc_status wc_erase(wc_table* t, const void* d_keys, uint64_t n, void* stream) {
  TraceRange trace("wc_erase");
  wc_status st = check_bulk(t, d_keys, n);
  if (st != WC_OK) return st;
  if (t->cfg.kind == WC_BLOOM_FILTER) return WC_ERR_UNSUPPORTED;  // bits are shared between keys
  if (n == 0) return WC_OK;
  DeviceGuard guard(t->device);
  if (t->cfg.kind == WC_MULTI_VALUE) return cuda_status(mv_erase(t, d_keys, n, as_stream(stream)));
  if (t->cfg.kind == WC_MULTI_VALUE_OA)
    return cuda_status(oa_launch(t, WC_OP_ERASE, d_keys, nullptr, n, nullptr, nullptr, as_stream(stream)));
  if (t->cfg.kind == WC_HASH_SET) return cuda_status(set_launch(t, WC_OP_ERASE, d_keys, n, nullptr, as_stream(stream)));
  return cuda_status(sv_launch(t, WC_OP_ERASE, d_keys, nullptr, n, nullptr, nullptr, as_stream(stream)));
}

wc_status wc_contains(wc_table* t, const void* d_keys, uint64_t n, uint8_t* d_found, void* stream) {
  TraceRange trace("wc_contains");
  wc_status st = check_bulk(t, d_keys, n);
  if (st != WC_OK) return st;
  st = check_buffer(t, d_found, n, 1);
  if (st != WC_OK) return st;
  const int kind = t->cfg.kind;
  if (kind != WC_SINGLE_VALUE && kind != WC_COUNTING && kind != WC_HASH_SET && kind != WC_BLOOM_FILTER)
    return WC_ERR_UNSUPPORTED;
  if (n == 0) return WC_OK;
  DeviceGuard guard(t->device);
  cudaStream_t s = as_stream(stream);
  if (kind == WC_HASH_SET) return cuda_status(set_launch(t, WC_OP_RETRIEVE, d_keys, n, d_found, s));
  if (kind == WC_BLOOM_FILTER) return cuda_status(bloom_launch(t, WC_OP_RETRIEVE, d_keys, n, d_found, s));
  return cuda_status(sv_launch(t, WC_OP_RETRIEVE, d_keys, nullptr, n, nullptr, d_found, s));
}

wc_status wc_count_values(wc_table* t, const void* d_keys, uint64_t n, uint64_t* d_offsets,
                          uint64_t* h_total_or_null, void* stream) {
  TraceRange trace("wc_count_values");
  wc_status st = check_bulk(t, d_keys, n);
  if (st != WC_OK) return st;
  if (t->cfg.kind != WC_MULTI_VALUE && t->cfg.kind != WC_MULTI_VALUE_OA) return WC_ERR_UNSUPPORTED;
  st = check_buffer(t, d_offsets, n + 1, 8);
  if (st != WC_OK) return st;
  DeviceGuard guard(t->device);
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaSuccess;
  if (t->cfg.kind == WC_MULTI_VALUE) {
    e = mv_count(t, d_keys, n, d_offsets, s);
  } else {
    if (n > 0) e = oa_launch(t, WC_OP_COUNT, d_keys, nullptr, n, d_offsets, nullptr, s);
    if (e == cudaSuccess) e = scan_exclusive_u64(d_offsets, n, t->d_partials, t->partials_cap, s);
  }
  if (e != cudaSuccess) return cuda_status(e);
  if (h_total_or_null != nullptr) {
    e = cudaMemcpyAsync(h_total_or_null, d_offsets + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return cuda_status(e);
}

wc_status wc_retrieve_multi(wc_table* t, const void* d_keys, uint64_t n, const uint64_t* d_offsets,
                            void* d_values_out, void* stream) {
  TraceRange trace("wc_retrieve_multi");
  wc_status st = check_bulk(t, d_keys, n);
  if (st != WC_OK) return st;
  if (t->cfg.kind != WC_MULTI_VALUE && t->cfg.kind != WC_MULTI_VALUE_OA) return WC_ERR_UNSUPPORTED;
  st = check_buffer(t, d_offsets, n + 1, 8);
  if (st == WC_OK) st = check_buffer(t, d_values_out, n, static_cast<uint64_t>(t->cfg.value_bytes));
  if (st != WC_OK) return st;
  if (n == 0) return WC_OK;
  DeviceGuard guard(t->device);
  if (t->cfg.kind == WC_MULTI_VALUE_OA)
    return cuda_status(oa_launch(t, WC_OP_RETRIEVE, d_keys, nullptr, n, const_cast<uint64_t*>(d_offsets),
                                 d_values_out, as_stream(stream)));
  return cuda_status(mv_retrieve_multi(t, d_keys, n, d_offsets, d_values_out, as_stream(stream)));
}

static wc_status read_counter(wc_table* t, const void* dptr, size_t bytes, void* host, void* stream) {
  if (t == nullptr || host == nullptr) return WC_ERR_INVALID_ARG;
  DeviceGuard guard(t->device);
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(host, dptr, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e);
}

wc_status wc_size(wc_table* t, uint64_t* h_out, void* stream) {
  if (t == nullptr) return WC_ERR_INVALID_ARG;
  return read_counter(t, t->d_size, sizeof(uint64_t), h_out, stream);
}

wc_status wc_num_keys(wc_table* t, uint64_t* h_out, void* stream) {
  if (t == nullptr || h_out == nullptr) return WC_ERR_INVALID_ARG;
  if (t->cfg.kind == WC_MULTI_VALUE_OA) {
    DeviceGuard guard(t->device);
    cudaError_t e = t->slot_bytes == 8 ? oa_p32_num_keys(t, as_stream(stream)) : oa_p64_num_keys(t, as_stream(stream));
    if (e != cudaSuccess) return cuda_status(e);
    return read_counter(t, t->d_nkeys, sizeof(uint64_t), h_out, stream);
  }
  return read_counter(t, t->cfg.kind == WC_MULTI_VALUE ? t->d_nkeys : t->d_size, sizeof(uint64_t), h_out, stream);
}

wc_status wc_value_pool_used(wc_table* t, uint64_t* h_out, void* stream) {
  if (t == nullptr || h_out == nullptr) return WC_ERR_INVALID_ARG;
  if (t->cfg.kind != WC_MULTI_VALUE) {
    *h_out = 0;
    return WC_OK;
  }
  return read_counter(t, t->d_cursor, sizeof(uint64_t), h_out, stream);
}

wc_status wc_load_factor(wc_table* t, double* h_out, void* stream) {
  if (t == nullptr || h_out == nullptr) return WC_ERR_INVALID_ARG;
  uint64_t live = 0;
  wc_status st = t->cfg.kind == WC_MULTI_VALUE_OA ? wc_size(t, &live, stream) : wc_num_keys(t, &live, stream);
  if (st != WC_OK) return st;
  *h_out = static_cast<double>(live) / static_cast<double>(t->capacity);
  return WC_OK;
}

wc_status wc_get_status(wc_table* t, uint32_t* h_flags, int32_t clear, void* stream) {
  if (t == nullptr || h_flags == nullptr) return WC_ERR_INVALID_ARG;
  wc_status st = read_counter(t, t->d_status, sizeof(uint32_t), h_flags, stream);
  if (st != WC_OK || !clear) return st;
  DeviceGuard guard(t->device);
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMemsetAsync(t->d_status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e);
}

}  // extern "C"
