// Random-access roofline probes (include/wc_roofline.h).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "wc.h"
#include "wc_device.cuh"
#include "wc_internal.h"
#include "wc_launch.cuh"
#include "wc_roofline.h"
#include "wc_device_api.cuh"

namespace wc {
namespace {

// XOR of the chunk's words; `first` receives its first word.
template <int BYTES>
__device__ __forceinline__ unsigned long long read_chunk(const unsigned long long* p, unsigned long long& first) {
  unsigned long long acc = 0;
  if constexpr (BYTES == 8) {
    unsigned long long u[1];
    ldcg1(p, u);
    acc = first = u[0];
  } else if constexpr (BYTES == 16) {
    unsigned long long u[2];
    ldcg2(p, u);
    first = u[0];
    acc = u[0] ^ u[1];
  } else {
#pragma unroll
    for (int i = 0; i < BYTES / 8; i += 4) {
      unsigned long long u[4];
      ldcg4(p + i, u);
      if (i == 0) first = u[0];
      acc ^= u[0] ^ u[1] ^ u[2] ^ u[3];
    }
  }
  return acc;
}

// One access = BYTES contiguous bytes at a random BYTES-aligned position, read by a group
// of LANES adjacent threads (lane r reads bytes [r, r + 1) * BYTES / LANES: the window load
// of a probing group); every thread keeps U accesses in flight.  Every load feeds `acc`,
// which is compared with a runtime value the compiler cannot know, so no load is dead
// code.  In CAS mode lane 0 then CASes the first word of the access with the value it read
// (the claim of a slot read in the same window).
template <int BYTES, int LANES, int U, bool kCas>
__global__ void __launch_bounds__(256) k_rand_access(unsigned long long* buf, uint64_t chunks, uint64_t accesses,
                                                     uint64_t seed, unsigned long long* sink) {
  constexpr int PER = BYTES / LANES;
  static_assert(PER >= 8 && BYTES % LANES == 0, "each lane reads whole 8-byte words");
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t grp = tid / LANES;
  const int r = static_cast<int>(threadIdx.x % LANES);
  const uint64_t ngrp = static_cast<uint64_t>(gridDim.x) * blockDim.x / LANES;
  unsigned long long acc = 0;
  for (uint64_t base = grp; base < accesses; base += ngrp * U) {
    unsigned long long* p[U];
    unsigned long long v[U], f[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + static_cast<uint64_t>(u) * ngrp;
      const uint64_t h = fmix64(seed ^ i);
      const uint64_t c = __umul64hi(h, chunks);
      p[u] = buf + c * (BYTES / 8) + r * (PER / 8);
      f[u] = 0ull;
      v[u] = i < accesses ? read_chunk<PER>(p[u], f[u]) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + static_cast<uint64_t>(u) * ngrp;
      if (kCas && r == 0 && i < accesses) acc ^= atomicCAS(p[u], f[u], f[u] + 1);
      acc ^= v[u];
    }
  }
  if (acc == seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull) *sink = acc;  // practically never taken
}

// Random stores of BYTES (the scatter of results to their input positions): thread-
// varying data, no read of the target.
template <int BYTES>
__global__ void __launch_bounds__(256) k_rand_write(unsigned long long* buf, uint64_t chunks, uint64_t accesses,
                                                    uint64_t seed) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t nth = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = tid; i < accesses; i += nth) {
    const uint64_t h = fmix64(seed ^ i);
    const uint64_t c = __umul64hi(h, chunks);
    char* p = reinterpret_cast<char*>(buf) + c * BYTES;
    if constexpr (BYTES == 4) {
      *reinterpret_cast<uint32_t*>(p) = static_cast<uint32_t>(h);
    } else {
#pragma unroll
      for (int w = 0; w < BYTES / 8; ++w) reinterpret_cast<unsigned long long*>(p)[w] = h + w;
    }
  }
}

template <int BYTES>
cudaError_t run_write(void* buf, const wc_rand_access_config& c, cudaStream_t s) {
  const int block = c.block_threads ? static_cast<int>(c.block_threads) : 256;
  int dev = 0;
  cudaGetDevice(&dev);
  auto kern = k_rand_write<BYTES>;
  const int bps = c.blocks_per_sm ? static_cast<int>(c.blocks_per_sm) : occupancy(kern, block);
  kern<<<bps * sm_count_of(dev), block, 0, s>>>(static_cast<unsigned long long*>(buf), c.buffer_bytes / BYTES,
                                                c.accesses, c.seed);
  return cudaGetLastError();
}

template <int BYTES, int LANES, int U>
cudaError_t launch_read(unsigned long long* b, const wc_rand_access_config& c, unsigned long long* k, int sms,
                        cudaStream_t s) {
  const int block = c.block_threads ? static_cast<int>(c.block_threads) : 256;
  const uint64_t chunks = c.buffer_bytes / BYTES;
  auto kern = c.mode == 1 ? k_rand_access<BYTES, LANES, U, true> : k_rand_access<BYTES, LANES, U, false>;
  const int bps = c.blocks_per_sm ? static_cast<int>(c.blocks_per_sm) : occupancy(kern, block);
  kern<<<bps * sms, block, 0, s>>>(b, chunks, c.accesses, c.seed, k);
  return cudaGetLastError();
}

template <int BYTES, int LANES>
cudaError_t run_lanes(unsigned long long* b, const wc_rand_access_config& c, unsigned long long* k, int sms,
                      cudaStream_t s) {
  if constexpr (BYTES / LANES < 8) {
    return cudaErrorInvalidValue;
  } else {
    switch (c.in_flight ? c.in_flight : 4u) {
      case 1: return launch_read<BYTES, LANES, 1>(b, c, k, sms, s);
      case 2: return launch_read<BYTES, LANES, 2>(b, c, k, sms, s);
      case 4: return launch_read<BYTES, LANES, 4>(b, c, k, sms, s);
      case 8: return launch_read<BYTES, LANES, 8>(b, c, k, sms, s);
      case 16: return launch_read<BYTES, LANES, 16>(b, c, k, sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

template <int BYTES>
cudaError_t run(void* buf, const wc_rand_access_config& c, uint64_t* sink, cudaStream_t s) {
  if (c.mode == 2) return run_write<BYTES>(buf, c, s);
  int dev = 0;
  cudaGetDevice(&dev);
  const int sms = sm_count_of(dev);
  auto* b = static_cast<unsigned long long*>(buf);
  auto* k = reinterpret_cast<unsigned long long*>(sink);
  switch (c.lanes ? c.lanes : 1u) {
    case 1: return run_lanes<BYTES, 1>(b, c, k, sms, s);
    case 2: return run_lanes<BYTES, 2>(b, c, k, sms, s);
    case 4: return run_lanes<BYTES, 4>(b, c, k, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int W>
__global__ void __launch_bounds__(256) k_dev_insert(wc_device_view v, uint64_t n, uint32_t seed) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  long long added = 0;  // new keys of this thread, added to the size once at the end
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t k = static_cast<uint32_t>(i * 2654435761ull) ^ seed;
    if (!wc_dev::is_sentinel(k) && wc_dev::insert_w<uint32_t, W, false, false>(v, k, static_cast<uint32_t>(i)) == 0)
      ++added;
  }
  wc_dev::add_size(v, added);
}

template <int W>
__global__ void __launch_bounds__(256) k_dev_lookup(wc_device_view v, uint64_t n, uint32_t seed,
                                                    unsigned long long* sink) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  unsigned long long acc = 0;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t k = static_cast<uint32_t>(i * 2654435761ull) ^ seed;
    uint32_t x;
    if (!wc_dev::is_sentinel(k) && wc_dev::retrieve_w<uint32_t, W>(v, k, x)) acc += x;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sink, acc);
}

template <int W>
void dev_probe(const wc_device_view& v, int mode, uint64_t n, uint32_t seed, unsigned long long* sink, int sms,
               cudaStream_t s) {
  if (mode == 0) {
    const int bps = occupancy(k_dev_insert<W>, 256);
    k_dev_insert<W><<<bps * sms, 256, 0, s>>>(v, n, seed);
  } else {
    const int bps = occupancy(k_dev_lookup<W>, 256);
    k_dev_lookup<W><<<bps * sms, 256, 0, s>>>(v, n, seed, sink);
  }
}

// The fused producer with tiles of G threads per key (the device API's group-cooperative
// insert and lookup).
template <int W, int G>
__global__ void __launch_bounds__(256) k_dev_group(wc_device_view v, int mode, uint64_t n, uint32_t seed,
                                                   unsigned long long* sink) {
  namespace cg = cooperative_groups;
  const auto tile = cg::tiled_partition<G>(cg::this_thread_block());
  const uint64_t tiles = static_cast<uint64_t>(gridDim.x) * blockDim.x / G;
  unsigned long long acc = 0;
  long long added = 0;  // new keys stored by this tile (its rank-0 thread), added once at the end
  for (uint64_t i = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / G; i < n; i += tiles) {
    const uint32_t k = static_cast<uint32_t>(i * 2654435761ull) ^ seed;
    if (wc_dev::is_sentinel(k)) continue;
    if (mode == 0) {
      if (wc_dev::insert_group<uint32_t, W, G, false>(tile, v, k, static_cast<uint32_t>(i)) == 0 && tile.thread_rank() == 0)
        ++added;
    } else {
      uint32_t x;
      if (wc_dev::retrieve_group<uint32_t, W, G>(tile, v, k, x) && tile.thread_rank() == 0) acc += x;
    }
  }
  if (mode != 0) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sink, acc);
  } else {
    wc_dev::add_size(v, added);
  }
}

// One thread per pair appends (keys[i], values[i]) to a bucket multi-value table with the
// device API's per-element append (the concurrent bucket-list insert).
template <class K, class V>
__global__ void __launch_bounds__(256) k_dev_append(wc_device_view v, const K* __restrict__ keys,
                                                    const V* __restrict__ vals, uint64_t n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  wc_dev::bl::Counts c;  // the thread's appended values and new keys, added once at the end
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    wc_dev::append_uncounted<K, V>(v, keys[i], vals[i], c);
  wc_dev::add_counts(v, c);
}

}  // namespace
}  // namespace wc

extern "C" {

wc_status wc_bench_device_api_group(wc_table* t, int32_t mode, int32_t group, uint64_t n, uint32_t key_seed,
                                    uint64_t* d_sink, void* stream) {
  if (t == nullptr || (mode != 0 && mode != 1) || (mode == 1 && d_sink == nullptr)) return WC_ERR_INVALID_ARG;
  wc_device_view v;
  const wc_status st = wc_table_device_view(t, &v);
  if (st != WC_OK) return st;
  if (v.kind != WC_SINGLE_VALUE || v.key_bytes != 4) return WC_ERR_UNSUPPORTED;
  if (n == 0) return WC_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return WC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* sink = reinterpret_cast<unsigned long long*>(d_sink);
  const int sms = wc::sm_count_of(t->device);
#define WC_GRP(Wv, Gv)                                                                                   \
  if (static_cast<int>(v.window_width) == (Wv) && group == (Gv)) {                                       \
    const int bps = wc::occupancy(wc::k_dev_group<Wv, Gv>, 256);                                         \
    wc::k_dev_group<Wv, Gv><<<bps * sms, 256, 0, s>>>(v, mode, n, key_seed, sink);                      \
    return cudaGetLastError() == cudaSuccess ? WC_OK : WC_ERR_CUDA;                                    \
  }
  WC_GRP(8, 1) WC_GRP(8, 2) WC_GRP(8, 4) WC_GRP(16, 2) WC_GRP(16, 4)
#undef WC_GRP
  return WC_ERR_INVALID_ARG;
}

wc_status wc_bench_mv_append(wc_table* t, const void* d_keys, const void* d_values, uint64_t n, void* stream) {
  if (t == nullptr || (n > 0 && (d_keys == nullptr || d_values == nullptr))) return WC_ERR_INVALID_ARG;
  wc_device_view v;
  const wc_status st = wc_table_device_view(t, &v);
  if (st != WC_OK) return st;
  if (v.kind != WC_MULTI_VALUE) return WC_ERR_UNSUPPORTED;
  if (n == 0) return WC_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return WC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned blocks = static_cast<unsigned>(wc::occupancy(wc::k_dev_append<uint32_t, uint32_t>, 256) *
                                                wc::sm_count_of(t->device));
  if (v.key_bytes == 4 && v.value_bytes == 4)
    wc::k_dev_append<uint32_t, uint32_t><<<blocks, 256, 0, s>>>(v, static_cast<const uint32_t*>(d_keys),
                                                               static_cast<const uint32_t*>(d_values), n);
  else if (v.key_bytes == 8 && v.value_bytes == 4)
    wc::k_dev_append<unsigned long long, uint32_t><<<blocks, 256, 0, s>>>(
        v, static_cast<const unsigned long long*>(d_keys), static_cast<const uint32_t*>(d_values), n);
  else if (v.key_bytes == 8)
    wc::k_dev_append<unsigned long long, unsigned long long><<<blocks, 256, 0, s>>>(
        v, static_cast<const unsigned long long*>(d_keys), static_cast<const unsigned long long*>(d_values), n);
  else
    wc::k_dev_append<uint32_t, unsigned long long><<<blocks, 256, 0, s>>>(
        v, static_cast<const uint32_t*>(d_keys), static_cast<const unsigned long long*>(d_values), n);
  return cudaGetLastError() == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}

wc_status wc_bench_device_api(wc_table* t, int32_t mode, uint64_t n, uint32_t key_seed, uint64_t* d_sink,
                              void* stream) {
  if (t == nullptr || (mode != 0 && mode != 1) || (mode == 1 && d_sink == nullptr)) return WC_ERR_INVALID_ARG;
  wc_device_view v;
  wc_status st = wc_table_device_view(t, &v);
  if (st != WC_OK) return st;
  if (v.kind != WC_SINGLE_VALUE || v.key_bytes != 4) return WC_ERR_UNSUPPORTED;
  if (n == 0) return WC_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return WC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int sms = wc::sm_count_of(t->device);
  auto* sink = reinterpret_cast<unsigned long long*>(d_sink);
  switch (v.window_width) {
    case 4: wc::dev_probe<4>(v, mode, n, key_seed, sink, sms, s); break;
    case 8: wc::dev_probe<8>(v, mode, n, key_seed, sink, sms, s); break;
    case 16: wc::dev_probe<16>(v, mode, n, key_seed, sink, sms, s); break;
    default: wc::dev_probe<32>(v, mode, n, key_seed, sink, sms, s); break;
  }
  return cudaGetLastError() == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}

wc_status wc_bench_random_access(void* d_buffer, const wc_rand_access_config* cfg, uint64_t* d_sink,
                                 void* stream) {
  if (d_buffer == nullptr || cfg == nullptr || d_sink == nullptr) return WC_ERR_INVALID_ARG;
  const uint32_t a = cfg->access_bytes;
  if (!(a == 8 || a == 16 || a == 32 || a == 64 || a == 128 || (a == 4 && cfg->mode == 2)) ||
      cfg->buffer_bytes < a || cfg->buffer_bytes % a != 0 || cfg->mode > 2)
    return WC_ERR_INVALID_ARG;
  if (cfg->block_threads && (cfg->block_threads > 256 || cfg->block_threads % 32)) return WC_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_buffer) % 256) return WC_ERR_INVALID_ARG;
  const uint32_t lanes = cfg->lanes ? cfg->lanes : 1u, inflight = cfg->in_flight ? cfg->in_flight : 4u;
  if (cfg->mode != 2 && ((lanes != 1 && lanes != 2 && lanes != 4) || a / lanes < 8 ||
                         (inflight != 1 && inflight != 2 && inflight != 4 && inflight != 8 && inflight != 16)))
    return WC_ERR_INVALID_ARG;
  if (cfg->accesses == 0) return WC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (a) {
    case 4: e = wc::run_write<4>(d_buffer, *cfg, s); break;
    case 8: e = wc::run<8>(d_buffer, *cfg, d_sink, s); break;
    case 16: e = wc::run<16>(d_buffer, *cfg, d_sink, s); break;
    case 32: e = wc::run<32>(d_buffer, *cfg, d_sink, s); break;
    case 64: e = wc::run<64>(d_buffer, *cfg, d_sink, s); break;
    default: e = wc::run<128>(d_buffer, *cfg, d_sink, s); break;
  }
  return e == cudaSuccess ? WC_OK : (e == cudaErrorInvalidValue ? WC_ERR_INVALID_ARG : WC_ERR_CUDA);
}

wc_status wc_set_l2_fetch_granularity(int32_t bytes) {
  if (bytes < 0 || bytes > 128) return WC_ERR_INVALID_ARG;
  return cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, static_cast<size_t>(bytes)) == cudaSuccess
             ? WC_OK
             : WC_ERR_CUDA;
}

wc_status wc_get_l2_fetch_granularity(int32_t* h_bytes) {
  if (h_bytes == nullptr) return WC_ERR_INVALID_ARG;
  size_t v = 0;
  if (cudaDeviceGetLimit(&v, cudaLimitMaxL2FetchGranularity) != cudaSuccess) return WC_ERR_CUDA;
  *h_bytes = static_cast<int32_t>(v);
  return WC_OK;
}

}  // extern "C"
