// Multi-split of a batch by table region (the partition step of the paper's distributed
// mode, Sec. IV-E, applied to L2-sized regions of one table instead of to GPUs).
//
// Region of a key = (first window of its probing sequence) / windows_per_region.  After
// the split the batch is ordered by region, so a probe kernel that sweeps it front to
// back touches one table region (a few tens of MB) at a time: its window loads and CAS
// claims hit L2 instead of HBM, and every region is read from and written back to HBM
// about once.  The order of keys inside a region is unspecified (bulk operations are
// sets of independent element operations).
#pragma once

#include <algorithm>

#include "wc_device.cuh"
#include "wc_internal.h"
#include "wc_launch.cuh"

namespace wc {

constexpr int kPartThreads = 512;
constexpr int kPartItems = 8;
constexpr int kPartTile = kPartThreads * kPartItems;
constexpr int kMaxRegions = 1024;

struct RegionMap {
  uint64_t seed;
  uint32_t p;    // windows of the table
  uint32_t wpr;  // windows per region
  uint32_t R;    // regions
};

template <class K>
__device__ __forceinline__ uint32_t region_of(const RegionMap& m, K key) {
  uint32_t w, step;
  probe_init(static_cast<uint64_t>(key), m.seed, m.p, w, step);
  const uint32_t r = w / m.wpr;
  return r < m.R ? r : m.R - 1;
}

// Per-region counts of the batch (hist[R], zeroed by the caller).  Each warp keeps its
// own shared-memory histogram, so atomics only collide inside a warp.
constexpr int kHistWarps = kPartThreads / 32;

template <class K>
__global__ void __launch_bounds__(kPartThreads) k_part_hist(const K* __restrict__ keys, uint64_t n, RegionMap m,
                                                            unsigned int* __restrict__ hist) {
  extern __shared__ unsigned int s_hw[];  // kHistWarps * R
  for (uint32_t i = threadIdx.x; i < kHistWarps * m.R; i += kPartThreads) s_hw[i] = 0;
  __syncthreads();
  unsigned int* mine = s_hw + (threadIdx.x >> 5) * m.R;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kPartThreads;
  for (uint64_t e = static_cast<uint64_t>(blockIdx.x) * kPartThreads + threadIdx.x; e < n; e += stride)
    atomicAdd(mine + region_of(m, ldg_stream(keys + e)), 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < m.R; i += kPartThreads) {
    unsigned int c = 0;
#pragma unroll
    for (int w = 0; w < kHistWarps; ++w) c += s_hw[w * m.R + i];
    if (c) atomicAdd(hist + i, c);
  }
}

// Exclusive scan of cnt[0..R) into off[0..R) by the whole block (R <= kMaxRegions);
// returns the total.  Every thread handles kMaxRegions / kPartThreads consecutive entries.
template <class T>
__device__ __forceinline__ T block_scan_regions(const T* cnt, T* off, uint32_t R, T* s_w) {
  constexpr int kPer = kMaxRegions / kPartThreads;
  const uint32_t b0 = threadIdx.x * kPer;
  T v[kPer];
  T sum = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    v[k] = b0 + k < R ? cnt[b0 + k] : T(0);
    sum += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  T before = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kPartThreads / 32; ++w) {
    if (w < warp) before += s_w[w];
    total += s_w[w];
  }
  T run = before + inc - sum;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (b0 + k < R) off[b0 + k] = run;
    run += v[k];
  }
  __syncthreads();
  return total;
}

// Scatter (keys, vals) into region order.  Per tile: rank every element inside its
// region with shared-memory atomics, reserve one run per region in the output with one
// global atomic on cursor[r] (zeroed by the caller), stage the tile in shared memory
// grouped by region, then copy the runs out with consecutive threads on consecutive
// addresses.
template <class K, class V>
struct ScatterSmem {
  K keys[kPartTile];
  V vals[kPartTile];
  unsigned short reg[kPartTile];
  unsigned int cnt[kMaxRegions];
  unsigned int toff[kMaxRegions];
  unsigned long long base[kMaxRegions];
  unsigned long long pos[kMaxRegions];
  unsigned long long w64[kPartThreads / 32];
  unsigned int w32[kPartThreads / 32];
};

template <class K, class V>
__global__ void __launch_bounds__(kPartThreads) k_part_scatter(const K* __restrict__ keys, const V* __restrict__ vals,
                                                               uint64_t n, RegionMap m,
                                                               const unsigned int* __restrict__ hist,
                                                               unsigned long long* __restrict__ cursor,
                                                               K* __restrict__ okeys, V* __restrict__ ovals) {
  extern __shared__ unsigned long long scatter_smem[];
  ScatterSmem<K, V>& S = *reinterpret_cast<ScatterSmem<K, V>*>(scatter_smem);
  // region bases: exclusive prefix of the histogram (every block recomputes it)
  for (uint32_t i = threadIdx.x; i < m.R; i += kPartThreads) S.pos[i] = hist[i];
  __syncthreads();
  block_scan_regions<unsigned long long>(S.pos, S.base, m.R, S.w64);
  const uint64_t ntiles = (n + kPartTile - 1) / kPartTile;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (uint32_t i = threadIdx.x; i < m.R; i += kPartThreads) S.cnt[i] = 0;
    __syncthreads();
    const uint64_t t0 = tile * kPartTile;
    const uint32_t tn = static_cast<uint32_t>(n - t0 < kPartTile ? n - t0 : kPartTile);
    K kk[kPartItems];
    V vv[kPartItems];
    uint32_t rr[kPartItems], rank[kPartItems];
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
      const uint32_t i = k * kPartThreads + threadIdx.x;
      rr[k] = 0xffffffffu;
      if (i < tn) {
        kk[k] = ldg_stream(keys + t0 + i);
        vv[k] = ldg_stream(vals + t0 + i);
        rr[k] = region_of(m, kk[k]);
        rank[k] = atomicAdd(S.cnt + rr[k], 1u);
      }
    }
    __syncthreads();
    block_scan_regions<unsigned int>(S.cnt, S.toff, m.R, S.w32);
    for (uint32_t r = threadIdx.x; r < m.R; r += kPartThreads)
      if (S.cnt[r]) S.pos[r] = S.base[r] + atomicAdd(cursor + r, static_cast<unsigned long long>(S.cnt[r]));
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
      if (rr[k] == 0xffffffffu) continue;
      const uint32_t o = S.toff[rr[k]] + rank[k];
      S.keys[o] = kk[k];
      S.vals[o] = vv[k];
      S.reg[o] = static_cast<unsigned short>(rr[k]);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tn; i += kPartThreads) {
      const uint32_t r = S.reg[i];
      const uint64_t o = S.pos[r] + (i - S.toff[r]);
      okeys[o] = S.keys[i];
      ovals[o] = S.vals[i];
    }
    __syncthreads();
  }
}

template <class K, class V>
constexpr size_t scatter_smem_bytes() {
  return sizeof(ScatterSmem<K, V>);
}

// ---- host side -------------------------------------------------------------------------
// A batch split by table region in the table's scratch buffer, plus kSplitCounters zeroed
// chunk counters for the ordered sweeps of the kernels that consume it.
constexpr int kSplitCounters = 32;

template <class K, class V>
struct RegionSplit {
  const K* keys;
  const V* vals;
  unsigned long long* counters;
};

// Regions of about region_mib MiB of slots (at most kMaxRegions of them).  Scratch layout:
// [hist 8 KiB | cursor 8 KiB | counters 256 B | keys | vals], grown on demand.
template <class K, class V>
cudaError_t region_split(const wc_table* t, int region_mib, const K* keys, const V* vals, uint64_t n, cudaStream_t s,
                         RegionSplit<K, V>& out) {
  static_assert(kMaxRegions * sizeof(unsigned long long) <= 8192, "cursor area");
  RegionMap m;
  m.seed = t->cfg.seed;
  m.p = static_cast<uint32_t>(t->windows);
  const uint64_t region_bytes = static_cast<uint64_t>(region_mib > 0 ? region_mib : 32) << 20;
  uint64_t wpr = std::max<uint64_t>(1, region_bytes / (t->W * t->slot_bytes));
  if ((t->windows + wpr - 1) / wpr > static_cast<uint64_t>(kMaxRegions)) wpr = (t->windows + kMaxRegions - 1) / kMaxRegions;
  m.wpr = static_cast<uint32_t>(wpr);
  m.R = static_cast<uint32_t>((t->windows + wpr - 1) / wpr);
  const uint64_t cur_off = 8192, cnt_off = cur_off + 8192, keys_off = cnt_off + 256;
  const uint64_t vals_off = keys_off + (n * sizeof(K) + 255) / 256 * 256;
  cudaError_t e = ensure_scratch(t, vals_off + n * sizeof(V), s);
  if (e != cudaSuccess) return e;
  char* sc = static_cast<char*>(t->d_scratch);
  auto* hist = reinterpret_cast<unsigned int*>(sc);
  auto* cursor = reinterpret_cast<unsigned long long*>(sc + cur_off);
  K* pk = reinterpret_cast<K*>(sc + keys_off);
  V* pv = reinterpret_cast<V*>(sc + vals_off);
  e = cudaMemsetAsync(sc, 0, keys_off, s);
  if (e != cudaSuccess) return e;
  auto hk = k_part_hist<K>;
  auto sk = k_part_scatter<K, V>;
  const size_t hsm = static_cast<size_t>(kHistWarps) * m.R * sizeof(unsigned int);
  const size_t ssm = scatter_smem_bytes<K, V>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kHistWarps * kMaxRegions * 4));
    cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(ssm));
    attr = true;
  }
  const uint64_t ntiles = (n + kPartTile - 1) / kPartTile;
  const unsigned hg = static_cast<unsigned>(std::min<uint64_t>(
      (n + kPartThreads - 1) / kPartThreads, static_cast<uint64_t>(occupancy_smem(hk, kPartThreads, hsm)) * t->sm_count));
  const unsigned sg = static_cast<unsigned>(
      std::min<uint64_t>(ntiles, static_cast<uint64_t>(occupancy_smem(sk, kPartThreads, ssm)) * t->sm_count));
  hk<<<hg, kPartThreads, hsm, s>>>(keys, n, m, hist);
  sk<<<sg, kPartThreads, ssm, s>>>(keys, vals, n, m, hist, cursor, pk, pv);
  e = cudaGetLastError();
  out.keys = pk;
  out.vals = pv;
  out.counters = reinterpret_cast<unsigned long long*>(sc + cnt_off);
  return e;
}

}  // namespace wc
