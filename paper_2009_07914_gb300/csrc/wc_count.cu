// Counting tables (the paper's CountingHashTable): the single-value engine with the
// counting slot layouts -- a stored key's count grows by the insert's weight (1 when no
// weights are given).  Lookups and erases use the single-value kernels (same slots).
#include "wc_partition.cuh"
#include "wc_sv_dispatch.cuh"

namespace wc {

bool count_shape_ok(int slot_bytes, int W, int G) {
  if (slot_bytes == 8) {
    switch (W) {
      case 4: return G == 1 || G == 2;
      case 8: return G == 1 || G == 2;
      case 16: return G == 2 || G == 4;
      case 32: return G == 4 || G == 8;
      default: return false;
    }
  }
  switch (W) {
    case 2: return G == 1;
    case 4: return G == 1 || G == 2;
    case 8: return G == 2 || G == 4;
    case 16: return G == 4 || G == 8;
    default: return false;
  }
}

namespace {

// Pass before the insert: each block sums the weights of equal keys inside a tile of
// kCntTile inputs in a shared-memory table and writes the tile's distinct keys with their
// sums to the front of the tile's range of the output, key 0 (skipped by the counting
// insert) behind them -- a hot key then costs one atomic add per tile instead of one per
// occurrence.  Sentinel inputs raise INVALID_KEY here.
constexpr int kCntThreads = 512;
constexpr int kCntItems = 8;
constexpr int kCntTile = kCntThreads * kCntItems;
constexpr int kCntSlots = 2 * kCntTile;

template <class K, class V>
constexpr size_t count_agg_smem() {
  return static_cast<size_t>(kCntSlots) * (sizeof(K) + sizeof(V));
}

template <class K, class V>
__global__ void __launch_bounds__(kCntThreads) k_count_aggregate(const K* __restrict__ keys, const V* __restrict__ w,
                                                                 uint64_t n, K* __restrict__ ok, V* __restrict__ ov,
                                                                 uint32_t* status) {
  extern __shared__ unsigned long long cnt_smem[];
  K* s_key = reinterpret_cast<K*>(cnt_smem);
  V* s_sum = reinterpret_cast<V*>(s_key + kCntSlots);
  __shared__ uint32_t s_warp[kCntThreads / 32];
  uint32_t flags = 0;
  const uint64_t ntiles = (n + kCntTile - 1) / kCntTile;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int e = threadIdx.x; e < kCntSlots; e += kCntThreads) {
      s_key[e] = K(0);
      s_sum[e] = V(0);
    }
    __syncthreads();
    const uint64_t t0 = tile * kCntTile;
    const uint32_t tn = static_cast<uint32_t>(n - t0 < kCntTile ? n - t0 : kCntTile);
#pragma unroll
    for (int it = 0; it < kCntItems; ++it) {
      const uint32_t i = it * kCntThreads + threadIdx.x;
      if (i >= tn) continue;
      const K k = ldg_stream(keys + t0 + i);
      if (k == K(0) || k == K(~K(0))) {
        flags |= kFlagInvalid;
        continue;
      }
      const V wt = w ? ldg_stream(w + t0 + i) : V(1);
      uint32_t h = static_cast<uint32_t>(fmix64(static_cast<uint64_t>(k)) >> 40) & (kCntSlots - 1);
      while (true) {  // at most kCntTile keys in 2 * kCntTile slots
        const K cur = atomicCAS(s_key + h, K(0), k);
        if (cur == K(0) || cur == k) break;
        h = (h + 1) & (kCntSlots - 1);
      }
      atomicAdd(s_sum + h, wt);
    }
    __syncthreads();
    // compact: thread t owns slots t, t + kCntThreads, ... (a warp reads consecutive slots;
    // the order of the aggregated keys is of no consequence)
    constexpr int per = kCntSlots / kCntThreads;
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) c += s_key[q * kCntThreads + threadIdx.x] != K(0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t pos = inc - c, total = 0;
#pragma unroll
    for (int q = 0; q < kCntThreads / 32; ++q) {
      if (q < warp) pos += s_warp[q];
      total += s_warp[q];
    }
#pragma unroll
    for (int q = 0; q < per; ++q) {
      const int e = q * kCntThreads + threadIdx.x;
      if (s_key[e] != K(0)) {
        ok[t0 + pos] = s_key[e];
        ov[t0 + pos] = s_sum[e];
        ++pos;
      }
    }
    for (uint32_t i = total + threadIdx.x; i < tn; i += kCntThreads) ok[t0 + i] = K(0);  // padding
    __syncthreads();
  }
  if (flags) atomicOr(status, flags);
}

template <class K, class V>
cudaError_t aggregate(const wc_table* t, const void* keys, const void* weights, uint64_t n, uint64_t skip_bytes,
                      const void** akeys, const void** avals, cudaStream_t s) {
  const uint64_t kbytes = (n * sizeof(K) + 255) / 256 * 256;
  cudaError_t e = ensure_scratch(t, skip_bytes + kbytes + n * sizeof(V), s);
  if (e != cudaSuccess) return e;
  K* ok = reinterpret_cast<K*>(static_cast<char*>(t->d_scratch) + skip_bytes);
  V* ov = reinterpret_cast<V*>(reinterpret_cast<char*>(ok) + kbytes);
  auto kern = k_count_aggregate<K, V>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(count_agg_smem<K, V>()));
    attr = true;
  }
  const uint64_t ntiles = (n + kCntTile - 1) / kCntTile;
  const uint64_t most = static_cast<uint64_t>(occupancy_smem(kern, kCntThreads, count_agg_smem<K, V>())) * t->sm_count;
  kern<<<static_cast<unsigned>(ntiles < most ? ntiles : most), kCntThreads, count_agg_smem<K, V>(), s>>>(
      static_cast<const K*>(keys), static_cast<const V*>(weights), n, ok, ov, t->d_status);
  *akeys = ok;
  *avals = ov;
  return cudaGetLastError();
}

}  // namespace

#define WC_COUNT_CASE(L, Wv, Gv) \
  if (W == (Wv) && G == (Gv)) return sv_insert_op<L, (Gv), (Wv) / (Gv)>(t, keys, weights, n, s);

// Insert of the aggregated batch (keys, per-tile sums; key 0 = padding).
static cudaError_t count_insert_agg(const wc_table* t, const void* keys, const void* weights, uint64_t n,
                                    cudaStream_t s) {
  const int W = static_cast<int>(t->W);
  const int G = t->launch[WC_OP_INSERT].group_size;
  if (t->slot_bytes == 8) {
    WC_COUNT_CASE(LayoutC32, 4, 1) WC_COUNT_CASE(LayoutC32, 4, 2)
    WC_COUNT_CASE(LayoutC32, 8, 1) WC_COUNT_CASE(LayoutC32, 8, 2)
    WC_COUNT_CASE(LayoutC32, 16, 2) WC_COUNT_CASE(LayoutC32, 16, 4)
    WC_COUNT_CASE(LayoutC32, 32, 4) WC_COUNT_CASE(LayoutC32, 32, 8)
  } else {
    WC_COUNT_CASE(LayoutC64, 2, 1)
    WC_COUNT_CASE(LayoutC64, 4, 1) WC_COUNT_CASE(LayoutC64, 4, 2)
    WC_COUNT_CASE(LayoutC64, 8, 2) WC_COUNT_CASE(LayoutC64, 8, 4)
    WC_COUNT_CASE(LayoutC64, 16, 4) WC_COUNT_CASE(LayoutC64, 16, 8)
  }
  return cudaErrorInvalidValue;
}

cudaError_t count_insert(const wc_table* t, const void* keys, const void* weights, uint64_t n, cudaStream_t s) {
  // The aggregated arrays sit behind the region split's area (when the insert splits), so
  // the split reads them without moving the scratch buffer.
  const uint64_t kb = static_cast<uint64_t>(t->cfg.key_bytes);
  const bool split = scheme_for(t, WC_OP_INSERT, n) == WC_SCHEME_BLOCKED;
  const uint64_t skip = split ? kSplitHeader + 2 * ((n * kb + 255) / 256 * 256) : 0;
  const void* ak = nullptr;
  const void* av = nullptr;
  cudaError_t e = kb == 4 ? aggregate<uint32_t, uint32_t>(t, keys, weights, n, skip, &ak, &av, s)
                          : aggregate<unsigned long long, unsigned long long>(t, keys, weights, n, skip, &ak, &av, s);
  if (e != cudaSuccess) return e;
  return count_insert_agg(t, ak, av, n, s);
}

}  // namespace wc
