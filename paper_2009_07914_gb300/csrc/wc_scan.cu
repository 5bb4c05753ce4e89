// Device-wide exclusive prefix sum of uint64 (reduce, scan of tile sums, down-sweep).
// Used by the multi-value counting pass to turn per-query counts into the n+1 output
// offsets of Sec. IV-B4.
#include <cuda_runtime.h>

#include <cstdint>

#include "wc_device.cuh"
#include "wc_internal.h"

namespace wc {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr uint64_t kTile = kThreads * kItems;
constexpr int kPartThreads = 1024;

__device__ __forceinline__ uint64_t warp_inclusive(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; `total` gets the sum.
template <int kT>
__device__ __forceinline__ uint64_t block_exclusive(uint64_t x, uint64_t& total) {
  __shared__ uint64_t s_w[kT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t inc = warp_inclusive(x);
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t v = lane < kT / 32 ? s_w[lane] : 0;
    v = warp_inclusive(v);
    if (lane < kT / 32) s_w[lane] = v;
  }
  __syncthreads();
  total = s_w[kT / 32 - 1];
  const uint64_t before = warp ? s_w[warp - 1] : 0;
  __syncthreads();
  return before + inc - x;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint64_t* __restrict__ d, uint64_t n,
                                                          uint64_t* __restrict__ partials) {
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kTile;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const uint64_t i = base + static_cast<uint64_t>(k) * kThreads + threadIdx.x;
    if (i < n) s += d[i];
  }
  uint64_t total;
  block_exclusive<kThreads>(s, total);
  if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// One block: exclusive scan of the tile sums in place, partials[nt] = grand total.
__global__ void __launch_bounds__(kPartThreads) k_scan_partials(uint64_t* __restrict__ partials, uint64_t nt) {
  uint64_t carry = 0;
  for (uint64_t base = 0; base < nt; base += kPartThreads) {
    const uint64_t i = base + threadIdx.x;
    const uint64_t x = i < nt ? partials[i] : 0;
    uint64_t total;
    const uint64_t ex = block_exclusive<kPartThreads>(x, total);
    if (i < nt) partials[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) partials[nt] = carry;
}

// Each thread owns kItems consecutive values of the tile.
__global__ void __launch_bounds__(kThreads) k_scan_down(uint64_t* __restrict__ d, uint64_t n,
                                                        const uint64_t* __restrict__ partials, uint64_t nt) {
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kTile + static_cast<uint64_t>(threadIdx.x) * kItems;
  uint64_t v[kItems];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = base + k < n ? d[base + k] : 0;
    s += v[k];
  }
  uint64_t total;
  uint64_t run = partials[blockIdx.x] + block_exclusive<kThreads>(s, total);
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if (base + k < n) d[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == nt - 1 && threadIdx.x == 0) d[n] = partials[nt];
}

}  // namespace

uint64_t scan_partials_needed(uint64_t n) { return (n + kTile - 1) / kTile + 1; }

cudaError_t scan_exclusive_u64(uint64_t* d, uint64_t n, uint64_t* partials, uint64_t partials_cap,
                               cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(d, 0, sizeof(uint64_t), s);
  const uint64_t nt = (n + kTile - 1) / kTile;
  if (nt + 1 > partials_cap) return cudaErrorInvalidValue;
  k_scan_reduce<<<static_cast<unsigned>(nt), kThreads, 0, s>>>(d, n, partials);
  k_scan_partials<<<1, kPartThreads, 0, s>>>(partials, nt);
  k_scan_down<<<static_cast<unsigned>(nt), kThreads, 0, s>>>(d, n, partials, nt);
  return cudaGetLastError();
}

}  // namespace wc
