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
  uint32_t p;      // windows of the table
  uint32_t shift;  // 2^shift windows per region
  uint32_t R;      // regions
  template <class K>
  __device__ __forceinline__ uint32_t of(K key) const {
    uint32_t w, step;
    probe_init(static_cast<uint64_t>(key), seed, p, w, step);
    const uint32_t r = w >> shift;
    return r < R ? r : R - 1;
  }
};

// Regions of a table: a power of two of windows each (a shift instead of a division per
// key), the largest one within region_mib MiB (0 = 32), doubled until there are at most
// kMaxRegions of them.
inline RegionMap region_map(const wc_table* t, int region_mib) {
  const uint64_t region_bytes = static_cast<uint64_t>(region_mib > 0 ? region_mib : 32) << 20;
  const uint64_t window_bytes = t->W * t->slot_bytes;
  uint32_t shift = 0;
  while ((window_bytes << (shift + 1)) <= region_bytes && shift < 31) ++shift;
  while (((t->windows + (1ull << shift) - 1) >> shift) > static_cast<uint64_t>(kMaxRegions)) ++shift;
  RegionMap m;
  m.seed = t->cfg.seed;
  m.p = static_cast<uint32_t>(t->windows);
  m.shift = shift;
  m.R = static_cast<uint32_t>((t->windows + (1ull << shift) - 1) >> shift);
  return m;
}

// Region of an output position: `per` consecutive positions per region.  Bit 31 of the
// word carries a flag (the found bit of a retrieve result) and is not part of the
// position.
struct IndexMap {
  uint32_t per;
  uint32_t R;
  __device__ __forceinline__ uint32_t of(uint32_t x) const {
    const uint32_t r = (x & 0x7fffffffu) / per;
    return r < R ? r : R - 1;
  }
};

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
  // kPartItems independent loads in flight per thread (block b takes elements
  // [b * kPartTile, (b + 1) * kPartTile) of every grid-wide stride, one per thread per item)
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kPartTile;
  for (uint64_t e0 = static_cast<uint64_t>(blockIdx.x) * kPartTile + threadIdx.x; e0 < n; e0 += stride) {
    K x[kPartItems];
#pragma unroll
    for (int u = 0; u < kPartItems; ++u) {
      const uint64_t e = e0 + static_cast<uint64_t>(u) * kPartThreads;
      x[u] = e < n ? ldg_stream(keys + e) : K(0);
    }
#pragma unroll
    for (int u = 0; u < kPartItems; ++u)
      if (e0 + static_cast<uint64_t>(u) * kPartThreads < n) atomicAdd(mine + m.of(x[u]), 1u);
  }
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
// addresses.  For pairs of at most 8 bytes the next tile's input is copied into shared
// memory with cp.async while the current tile is ranked and written out, so the input
// stream never stops (wider pairs would halve the resident blocks and read directly).
template <class K, class V>
constexpr bool scatter_prefetch() {
  return sizeof(K) + sizeof(V) <= 8;
}

template <class K, class V>
struct ScatterSmem {
  static constexpr int kIn = scatter_prefetch<K, V>() ? kPartTile : 1;
  K keys[kPartTile];
  V vals[kPartTile];
  unsigned short reg[kPartTile];
  unsigned int cnt[kMaxRegions];
  unsigned int toff[kMaxRegions];
  unsigned long long base[kMaxRegions];
  unsigned long long pos[kMaxRegions];
  unsigned long long w64[kPartThreads / 32];
  unsigned int w32[kPartThreads / 32];
  K in_keys[kIn];  // the next tile's input (prefetching layouts only)
  V in_vals[kIn];
};

// Asynchronous global -> shared copy of one 4- or 8-byte element (cp.async, L1 bypassed
// for the streamed input with an evict-first L2 policy), and the wait for all of them.
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gmem_src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3;"
               :
               : "r"(d), "l"(gmem_src), "n"(static_cast<int>(sizeof(T))), "l"(evict_first_policy())
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Where the values of a split come from: read from `vals`, element i's input position i,
// or 1 (vals is not read in the last two).
enum { kValsRead = 0, kValsIota = 1, kValsOne = 2 };

template <class K, class V, class M = RegionMap, int kVals = kValsRead>
__global__ void __launch_bounds__(kPartThreads) k_part_scatter(const K* __restrict__ keys, const V* __restrict__ vals,
                                                               uint64_t n, M m,
                                                               const unsigned int* __restrict__ hist,
                                                               unsigned long long* __restrict__ cursor,
                                                               K* __restrict__ okeys, V* __restrict__ ovals) {
  extern __shared__ unsigned long long scatter_smem[];
  ScatterSmem<K, V>& S = *reinterpret_cast<ScatterSmem<K, V>*>(scatter_smem);
  constexpr bool kPre = scatter_prefetch<K, V>();
  const uint64_t ntiles = (n + kPartTile - 1) / kPartTile;
  // copy tile `tl`'s input into S.in_keys / S.in_vals (prefetching layouts)
  auto prefetch = [&](uint64_t tl) {
    const uint64_t b = tl * kPartTile;
    const uint32_t cnt = static_cast<uint32_t>(n - b < kPartTile ? n - b : kPartTile);
    for (uint32_t i = threadIdx.x; i < cnt; i += kPartThreads) {
      cp_async_elem(S.in_keys + i, keys + b + i);
      if constexpr (kVals == kValsRead) cp_async_elem(S.in_vals + i, vals + b + i);
    }
  };
  if constexpr (kPre) {
    if (blockIdx.x < ntiles) prefetch(blockIdx.x);
  }
  // region bases: exclusive prefix of the histogram (every block recomputes it)
  for (uint32_t i = threadIdx.x; i < m.R; i += kPartThreads) S.pos[i] = hist[i];
  __syncthreads();
  block_scan_regions<unsigned long long>(S.pos, S.base, m.R, S.w64);
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (uint32_t i = threadIdx.x; i < m.R; i += kPartThreads) S.cnt[i] = 0;
    if constexpr (kPre) cp_async_wait_all();  // this tile's input is in shared memory
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
        if constexpr (kPre) {
          kk[k] = S.in_keys[i];
        } else {
          kk[k] = ldg_stream(keys + t0 + i);
        }
        if constexpr (kVals == kValsIota) {
          vv[k] = static_cast<V>(t0 + i);
        } else if constexpr (kVals == kValsOne) {
          vv[k] = V(1);
        } else if constexpr (kPre) {
          vv[k] = S.in_vals[i];
        } else {
          vv[k] = ldg_stream(vals + t0 + i);
        }
        rr[k] = m.of(kk[k]);
        rank[k] = atomicAdd(S.cnt + rr[k], 1u);
      }
    }
    __syncthreads();
    // the input buffer is free again: start copying the block's next tile
    if constexpr (kPre) {
      if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x);
    }
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
      if (o < n) {  // always true when hist holds this batch's counts
        okeys[o] = S.keys[i];
        ovals[o] = S.vals[i];
      }
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
// chunk counters for the ordered sweeps of the kernels that consume it, and a zeroed
// area for a second split (hist2 / cursor2) and `extra` bytes the caller asked for.
constexpr int kSplitCounters = 32;
constexpr uint64_t kSplitHist = 0, kSplitCursor = 8192, kSplitCnt = 16384, kSplitHist2 = 16640,
                   kSplitCursor2 = 20736, kSplitHeader = 29184;
static_assert(kMaxRegions * sizeof(unsigned int) <= kSplitCursor2 - kSplitHist2, "hist2 area");
static_assert(kMaxRegions * sizeof(unsigned long long) <= kSplitHeader - kSplitCursor2, "cursor2 area");

template <class K, class V>
struct RegionSplit {
  const K* keys;
  const V* vals;
  unsigned long long* counters;
  unsigned int* hist2;          // second split: per-region counts (zeroed)
  unsigned long long* cursor2;  // second split: per-region cursors (zeroed)
  char* extra;                  // `extra` bytes, 256-byte aligned (not zeroed)
};

inline uint64_t align256(uint64_t x) { return (x + 255) / 256 * 256; }

// Regions of region_map(t, region_mib).  Scratch layout:
// [header kSplitHeader B | keys | vals | extra], grown on demand.  kVals: where the values
// come from (kValsIota: the input positions as uint32; kValsOne: all 1).
template <class K, class V, int kVals = kValsRead>
cudaError_t region_split(const wc_table* t, int region_mib, const K* keys, const V* vals, uint64_t n, cudaStream_t s,
                         RegionSplit<K, V>& out, uint64_t extra = 0) {
  static_assert(kMaxRegions * sizeof(unsigned long long) <= kSplitCnt - kSplitCursor, "cursor area");
  const RegionMap m = region_map(t, region_mib);
  const uint64_t keys_off = kSplitHeader;
  const uint64_t vals_off = keys_off + align256(n * sizeof(K));
  const uint64_t extra_off = vals_off + align256(n * sizeof(V));
  cudaError_t e = ensure_scratch(t, extra_off + extra, s);
  if (e != cudaSuccess) return e;
  char* sc = static_cast<char*>(t->d_scratch);
  auto* hist = reinterpret_cast<unsigned int*>(sc + kSplitHist);
  auto* cursor = reinterpret_cast<unsigned long long*>(sc + kSplitCursor);
  K* pk = reinterpret_cast<K*>(sc + keys_off);
  V* pv = reinterpret_cast<V*>(sc + vals_off);
  e = cudaMemsetAsync(sc, 0, kSplitHeader, s);
  if (e != cudaSuccess) return e;
  auto hk = k_part_hist<K>;
  auto sk = k_part_scatter<K, V, RegionMap, kVals>;
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
      (n + kPartTile - 1) / kPartTile, static_cast<uint64_t>(occupancy_smem(hk, kPartThreads, hsm)) * t->sm_count));
  const unsigned sg = static_cast<unsigned>(
      std::min<uint64_t>(ntiles, static_cast<uint64_t>(occupancy_smem(sk, kPartThreads, ssm)) * t->sm_count));
  hk<<<hg, kPartThreads, hsm, s>>>(keys, n, m, hist);
  sk<<<sg, kPartThreads, ssm, s>>>(keys, vals, n, m, hist, cursor, pk, pv);
  e = cudaGetLastError();
  out.keys = pk;
  out.vals = pv;
  out.counters = reinterpret_cast<unsigned long long*>(sc + kSplitCnt);
  out.hist2 = reinterpret_cast<unsigned int*>(sc + kSplitHist2);
  out.cursor2 = reinterpret_cast<unsigned long long*>(sc + kSplitCursor2);
  out.extra = sc + extra_off;
  return e;
}

}  // namespace wc
