// Autotuner (include/wc_tune.h): times the library's own bulk calls on a synthetic sample
// for every window width and launch shape, through the public C ABI only.  Host code plus
// one kernel that writes the sample.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "wc.h"
#include "wc_device_api.cuh"
#include "wc_internal.h"
#include "wc_tune.h"

namespace {

// The sample: key j = mix(j) for j = 1..n, values 1..n, n queries of which the even
// positions hold present keys and the odd ones the keys mix(n + 1 + i) (absent), and n "hot"
// queries over the first n / 64 keys only -- a set whose windows stay in L2, as the hot
// keys of a skewed query stream do.  mix is an invertible finalizer (MurmurHash3's fmix64 /
// fmix32, public domain), so the keys are distinct and look random in value and order (a
// sample of sequential keys measured a different best lookup shape than random keys do);
// mix(0) = 0, and the one j whose mix is all ones takes mix(3n + 7) instead, which no other
// sample key has.
__device__ __forceinline__ uint32_t tune_mix(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint64_t tune_mix(uint64_t h) { return wc_dev::fmix64(h); }

template <class K>
__device__ __forceinline__ K tune_key(uint64_t j, uint64_t n) {
  K x = tune_mix(static_cast<K>(j));
  if (x == K(~K(0))) x = tune_mix(static_cast<K>(3 * n + 7));
  return x;
}

template <class K, class V>
__global__ void k_tune_fill(K* keys, V* vals, K* queries, K* hot, uint64_t n) {
  const uint64_t hot_n = n / 64 > 0 ? n / 64 : 1;
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    keys[i] = tune_key<K>(i + 1, n);
    if (vals != nullptr) vals[i] = static_cast<V>(i + 1);
    queries[i] = tune_key<K>((i & 1) ? n + 1 + i : i + 1, n);
    hot[i] = tune_key<K>((i * 2654435761ull) % hot_n + 1, n);
  }
}

using CacheKey = std::tuple<int, int, int, int, int, int, int, uint64_t>;
std::mutex g_mu;
std::map<CacheKey, wc_tuning> g_cache;

struct Buffers {
  void* keys = nullptr;
  void* vals = nullptr;
  void* queries = nullptr;
  void* hot = nullptr;
  void* out = nullptr;
  uint8_t* found = nullptr;
  ~Buffers() {
    cudaFree(keys);
    cudaFree(vals);
    cudaFree(queries);
    cudaFree(hot);
    cudaFree(out);
    cudaFree(found);
  }
};

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Window widths tried for a slot width: 32- to 128-byte windows.
std::vector<int> window_candidates(int slot_bytes) {
  if (slot_bytes == 4) return {8, 16, 32};
  if (slot_bytes == 8) return {4, 8, 16};
  return {2, 4, 8};
}

// The library's window for window_width = 0 without tuning: 64 bytes.
int default_window(int slot_bytes) { return 64 / slot_bytes; }

int slot_bytes_of(const wc_table_config& c) {
  if (c.kind == WC_HASH_SET) return c.key_bytes;
  return c.key_bytes + c.value_bytes;
}

// A shape or window width replaces the library's default only when it is more than 10 %
// faster on the sample: the sample is smaller than most tables it stands for (a 256 MiB
// table for tables of gigabytes), and smaller margins measured on it did not carry over
// (2^27 keys: a 32-byte window 2-4 % ahead on the sample was 4 % behind on the table).
constexpr double kReplace = 0.90;

// One window width: the best shape of each operation, with the library default kept
// unless another shape is more than 10 % faster.
struct WindowResult {
  bool ok = false;
  wc_launch launch[3];
  double ms[3] = {0, 0, 0};
  int candidates = 0;
};

class Tuner {
 public:
  Tuner(const wc_table_config& cfg, double load, uint64_t n, cudaStream_t s, Buffers& b)
      : cfg_(cfg), load_(load), n_(n), s_(s), b_(b) {}

  wc_status run_window(int W, WindowResult& r) {
    wc_table_config c = cfg_;
    c.window_width = W;
    c.l2_persist = 0;
    c.min_capacity = static_cast<uint64_t>(std::ceil(static_cast<double>(n_) / load_));
    wc_table* t = nullptr;
    wc_status st = wc_table_create(&t, &c);
    if (st == WC_ERR_INVALID_ARG) return WC_OK;  // W not valid for this kind: skipped
    if (st != WC_OK) return st;
    st = tune_table(t, W, r);
    const wc_status d = wc_table_destroy(t);
    return st != WC_OK ? st : d;
  }

 private:
  const wc_table_config cfg_;
  const double load_;
  const uint64_t n_;
  cudaStream_t s_;
  Buffers& b_;
  Timer tm_;

  bool is_set() const { return cfg_.kind == WC_HASH_SET; }
  int slot_bytes() const { return slot_bytes_of(cfg_); }

  wc_status insert(wc_table* t) { return wc_insert(t, b_.keys, is_set() ? nullptr : b_.vals, n_, s_); }
  // a lookup is timed on both kinds of query stream: the uniform one (HBM-bound) and the
  // hot one (L2-bound), so a shape that only wins one of them does not take the table
  wc_status lookup(wc_table* t) {
    for (const void* q : {b_.queries, b_.hot}) {
      const wc_status st = is_set() ? wc_contains(t, q, n_, b_.found, s_)
                                    : wc_retrieve(t, q, n_, b_.out, b_.found, s_);
      if (st != WC_OK) return st;
    }
    return WC_OK;
  }
  wc_status erase(wc_table* t) { return wc_erase(t, b_.keys, n_, s_); }

  // Best of three timed calls of `timed`, each after `prep` (untimed); then the table's
  // status word, which must show no failure.
  template <class Prep, class Op>
  wc_status best_of(wc_table* t, Prep prep, Op timed, double& ms) {
    ms = 1e30;
    for (int rep = 0; rep < 3; ++rep) {
      wc_status st = prep();
      if (st != WC_OK) return st;
      if (cudaEventRecord(tm_.a, s_) != cudaSuccess) return WC_ERR_CUDA;
      st = timed();
      if (st != WC_OK) return st;
      if (cudaEventRecord(tm_.b, s_) != cudaSuccess || cudaEventSynchronize(tm_.b) != cudaSuccess)
        return WC_ERR_CUDA;
      float f = 0;
      if (cudaEventElapsedTime(&f, tm_.a, tm_.b) != cudaSuccess) return WC_ERR_CUDA;
      ms = std::min(ms, static_cast<double>(f));
    }
    uint32_t flags = 0;
    const wc_status st = wc_get_status(t, &flags, 1, s_);
    if (st != WC_OK) return st;
    // a sample at load <= 0.99 always fits, and no call here waits on a queue
    if (flags & (WC_FLAG_PROBE_LIMIT | WC_FLAG_QUEUE_TIMEOUT | WC_FLAG_INVALID_KEY)) return WC_ERR_CUDA;
    return WC_OK;
  }

  // Time the table's default shape of `op` and every other valid group size (and, for
  // lookups whose lanes hold at most 32 bytes of window, two keys in flight); keep the
  // default unless the fastest other shape beats it by more than 10 %.
  template <class Prep, class Op>
  wc_status sweep(wc_table* t, int W, int op, Prep prep, Op timed, WindowResult& r) {
    wc_launch def{};
    wc_status st = wc_table_get_launch(t, op, &def);
    if (st != WC_OK) return st;
    const int def_k = std::max(1, def.keys_in_flight);
    std::vector<wc_launch> cands{def};
    for (int g = 1; g <= W && g <= 32; g *= 2) {
      for (int k = 1; k <= 2; ++k) {
        if (k == 2 && (op != WC_OP_RETRIEVE || is_set() || (W / g) * slot_bytes() > 32)) continue;
        if (g == def.group_size && k == def_k) continue;
        wc_launch l = def;
        l.group_size = g;
        l.keys_in_flight = k;
        cands.push_back(l);
      }
    }
    double def_ms = 0, best_ms = 1e30;
    wc_launch best = def;
    for (size_t i = 0; i < cands.size(); ++i) {
      st = wc_table_set_launch(t, op, &cands[i]);
      if (st == WC_ERR_INVALID_ARG && i > 0) continue;  // group size not valid for W
      if (st != WC_OK) return st;
      double ms = 0;
      st = best_of(t, prep, timed, ms);
      if (st != WC_OK) return st;
      ++r.candidates;
      if (i == 0) {
        def_ms = ms;
      } else if (ms < best_ms) {
        best_ms = ms;
        best = cands[i];
      }
    }
    const bool keep = !(best_ms < kReplace * def_ms);
    r.launch[op] = keep ? def : best;
    r.ms[op] = keep ? def_ms : best_ms;
    return wc_table_set_launch(t, op, &r.launch[op]);
  }

  wc_status tune_table(wc_table* t, int W, WindowResult& r) {
    auto clear = [&]() { return wc_table_clear(t, s_); };
    auto fill = [&]() {
      wc_status st = wc_table_clear(t, s_);
      return st != WC_OK ? st : insert(t);
    };
    auto none = [&]() { return WC_OK; };
    wc_status st = sweep(t, W, WC_OP_INSERT, clear, [&]() { return insert(t); }, r);
    if (st == WC_OK) st = fill();
    if (st == WC_OK) st = sweep(t, W, WC_OP_RETRIEVE, none, [&]() { return lookup(t); }, r);
    if (st == WC_OK) st = sweep(t, W, WC_OP_ERASE, fill, [&]() { return erase(t); }, r);
    if (st == WC_OK) r.ok = true;
    return st;
  }
};

template <class K, class V>
cudaError_t fill_sample(Buffers& b, uint64_t n, cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(std::min<uint64_t>((n + 255) / 256, 4096));
  k_tune_fill<K, V><<<grid, 256, 0, s>>>(static_cast<K*>(b.keys), static_cast<V*>(b.vals), static_cast<K*>(b.queries),
                                         static_cast<K*>(b.hot), n);
  return cudaGetLastError();
}

wc_status autotune_uncached(const wc_table_config& cfg, double load, uint64_t n, wc_tuning& out) {
  const int sb = slot_bytes_of(cfg);
  const int kb = cfg.key_bytes, vb = cfg.value_bytes;
  Buffers b;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return WC_ERR_CUDA;
  auto done = [&](wc_status st) {
    if (s != nullptr) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    if (st != WC_OK) cudaGetLastError();
    return st;
  };
  const uint64_t vbytes = vb > 0 ? static_cast<uint64_t>(vb) : 4;
  if (cudaMalloc(&b.keys, n * kb) != cudaSuccess || cudaMalloc(&b.queries, n * kb) != cudaSuccess ||
      cudaMalloc(&b.hot, n * kb) != cudaSuccess ||
      cudaMalloc(&b.out, n * vbytes) != cudaSuccess || cudaMalloc(&b.found, n) != cudaSuccess ||
      (vb > 0 && cudaMalloc(&b.vals, n * vbytes) != cudaSuccess))
    return done(WC_ERR_OUT_OF_MEMORY);
  cudaError_t e = kb == 4 ? (vb == 8 ? fill_sample<uint32_t, uint64_t>(b, n, s) : fill_sample<uint32_t, uint32_t>(b, n, s))
                          : (vb == 4 ? fill_sample<uint64_t, uint32_t>(b, n, s) : fill_sample<uint64_t, uint64_t>(b, n, s));
  if (e != cudaSuccess) return done(WC_ERR_CUDA);

  std::vector<int> ws = cfg.window_width != 0 ? std::vector<int>{cfg.window_width} : window_candidates(sb);
  const int wdef = cfg.window_width != 0 ? cfg.window_width : default_window(sb);
  Tuner tuner(cfg, load, n, s, b);
  int candidates = 0;
  // the default window width is kept unless another one's insert + lookup time beats it
  // by more than 10 %
  bool have = false, have_def = false;
  double best = 1e30, def_score = 0;
  WindowResult pick, def_r;
  int pick_w = 0;
  for (int W : ws) {
    WindowResult r;
    const wc_status st = tuner.run_window(W, r);
    if (st != WC_OK) return done(st);
    candidates += r.candidates;
    if (!r.ok) continue;
    const double score = r.ms[WC_OP_INSERT] + r.ms[WC_OP_RETRIEVE];
    if (W == wdef) {
      have_def = true;
      def_score = score;
      def_r = r;
    } else if (score < best) {
      best = score;
      pick = r;
      pick_w = W;
      have = true;
    }
  }
  if (have_def && !(have && best < kReplace * def_score)) {
    pick = def_r;
    pick_w = wdef;
    have = true;
  }
  if (!have) return done(WC_ERR_UNSUPPORTED);
  std::memset(&out, 0, sizeof(out));
  out.window_width = pick_w;
  out.candidates = candidates;
  out.from_cache = 0;
  for (int op = 0; op < 3; ++op) {
    out.launch[op] = pick.launch[op];
    out.ms[op] = pick.ms[op];
  }
  out.sample_keys = n;
  out.load = load;
  return done(WC_OK);
}

}  // namespace

namespace wc {

// Sample size for window_width = 0 at table creation: tables of up to 32 MiB of slots
// live in L2 and are tuned on 2^20 keys; larger ones on a table of 256 MiB of slots (twice
// the L2) at load 0.9.
uint64_t autotune_sample_for(const wc_table_config& cfg) {
  const uint64_t sb = static_cast<uint64_t>(slot_bytes_of(cfg));
  if (cfg.min_capacity * sb <= (32ull << 20)) return 1ull << 20;
  return ((256ull << 20) / sb * 9 / 10) & ~1023ull;  // 30,198,784 keys of 8-byte slots
}

bool autotune_enabled() {
  const char* v = std::getenv("WC_AUTOTUNE");
  return v == nullptr || std::strcmp(v, "0") != 0;
}

}  // namespace wc

extern "C" {

wc_status wc_autotune(const wc_table_config* cfg, double load, uint64_t sample_keys, int32_t use_cache,
                      wc_tuning* h_out) {
  if (cfg == nullptr || h_out == nullptr) return WC_ERR_INVALID_ARG;
  if (!(load >= 0.05 && load <= 0.99) || sample_keys < (1ull << 10) || sample_keys > (1ull << 26))
    return WC_ERR_INVALID_ARG;
  if (cfg->kind != WC_SINGLE_VALUE && cfg->kind != WC_COUNTING && cfg->kind != WC_HASH_SET) return WC_ERR_UNSUPPORTED;
  if (cfg->options & WC_OPT_SOA) return WC_ERR_UNSUPPORTED;
  const bool widths_ok = cfg->kind == WC_HASH_SET
                             ? ((cfg->key_bytes == 4 || cfg->key_bytes == 8) && cfg->value_bytes == 0)
                             : ((cfg->key_bytes == 4 && cfg->value_bytes == 4) || (cfg->key_bytes == 8 && cfg->value_bytes == 8));
  if (!widths_ok) return WC_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return WC_ERR_CUDA;
  const CacheKey key{cfg->device, cfg->kind, cfg->key_bytes, cfg->value_bytes, cfg->options, cfg->window_width,
                     static_cast<int>(std::lround(load * 100)), sample_keys};
  std::lock_guard<std::mutex> lock(g_mu);
  if (use_cache) {
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *h_out = it->second;
      h_out->from_cache = 1;
      return WC_OK;
    }
  }
  wc::DeviceGuard guard(cfg->device);
  wc_tuning r;
  const wc_status st = autotune_uncached(*cfg, load, sample_keys, r);
  if (st != WC_OK) return st;
  if (use_cache) g_cache[key] = r;
  *h_out = r;
  return WC_OK;
}

uint64_t wc_autotune_sample_keys(const wc_table_config* cfg) {
  return cfg == nullptr ? 0 : wc::autotune_sample_for(*cfg);
}

wc_status wc_table_apply_tuning(wc_table* t, const wc_tuning* tuning) {
  if (t == nullptr || tuning == nullptr) return WC_ERR_INVALID_ARG;
  wc_table_info info;
  wc_status st = wc_table_get_info(t, &info);
  if (st != WC_OK) return st;
  if (info.window_width != tuning->window_width) return WC_ERR_INVALID_ARG;
  wc_launch old[3];
  for (int op = 0; op < 3; ++op) wc_table_get_launch(t, op, &old[op]);
  for (int op = 0; op < 3; ++op) {
    st = wc_table_set_launch(t, op, &tuning->launch[op]);
    if (st != WC_OK) {
      for (int o = 0; o < 3; ++o) wc_table_set_launch(t, o, &old[o]);
      return st;
    }
  }
  return WC_OK;
}

}  // extern "C"
