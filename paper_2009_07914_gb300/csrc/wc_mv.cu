// Multi-value bulk insert: dispatch of the count / allocate / scatter passes.
#include <algorithm>

#include "wc_launch.cuh"
#include "wc_mv_kernels.cuh"
#include "wc_partition.cuh"

namespace wc {

namespace {

template <class KIn, int VB, int W, int kThreads>
cudaError_t insert_passes(const wc_table* t, const void* keys, const void* vals, uint64_t n, cudaStream_t s) {
  using V = typename PoolT<VB>::T;
  using A = Agg<kThreads>;
  const TableDesc d = desc_of(t);
  const PoolDesc pd = pool_of(t);
  const KIn* k = static_cast<const KIn*>(keys);
  auto count = k_mv_aggregate<KIn, VB, W, false, kThreads>;
  auto scatter = k_mv_aggregate<KIn, VB, W, true, kThreads>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(count, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(A::smem_bytes(false, sizeof(KIn))));
    cudaFuncSetAttribute(scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(A::smem_bytes(true, sizeof(KIn))));
    attr_done = true;
  }
  // Large batches into a key store larger than L2 are first split by key-store region
  // (the region split of the single-value insert): the passes then probe one L2-resident
  // region of the key store at a time, and pass 3 writes one range of the pool at a time
  // (pass 2 lays buckets out in key-store order).
  unsigned long long* counters = nullptr;
  cudaError_t e = cudaSuccess;
  if (n >= (1ull << 20) && t->table_bytes > (64ull << 20)) {
    RegionSplit<KIn, V> sp;
    e = region_split(t, 32, k, static_cast<const V*>(vals), n, s, sp);
    if (e != cudaSuccess) return e;
    k = sp.keys;
    vals = sp.vals;
    counters = sp.counters;
  }
  const uint64_t ntiles = (n + A::kTile - 1) / A::kTile;
  const int bps_c = occupancy_smem(count, kThreads, A::smem_bytes(false, sizeof(KIn)));
  const int bps_s = occupancy_smem(scatter, kThreads, A::smem_bytes(true, sizeof(KIn)));
  const unsigned g_c = static_cast<unsigned>(std::min<uint64_t>(ntiles, static_cast<uint64_t>(bps_c) * t->sm_count));
  const unsigned g_s = static_cast<unsigned>(std::min<uint64_t>(ntiles, static_cast<uint64_t>(bps_s) * t->sm_count));
  e = cudaMemsetAsync(pd.pending, 0, t->capacity * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  e = launch_k(t, count, g_c, kThreads, A::smem_bytes(false, sizeof(KIn)), s, d, pd, k, vals, n, counters);
  if (e != cudaSuccess) return e;
  const uint64_t per_block = static_cast<uint64_t>(kAllocThreads) * kAllocItems;
  const unsigned g_a = static_cast<unsigned>((t->capacity + per_block - 1) / per_block);
  e = launch_k(t, t->growth == kGrowExact ? k_mv_alloc<VB> : k_mv_alloc_growth<VB>, g_a, kAllocThreads, 0, s, d, pd,
               t->capacity);
  if (e != cudaSuccess) return e;
  return launch_k(t, scatter, g_s, kThreads, A::smem_bytes(true, sizeof(KIn)), s, d, pd, k, vals, n,
                  counters ? counters + 1 : counters);
}

// The aggregation passes run blocks of the insert launch's block_threads (256 or 512;
// 2^28 Zipf inserts over 2^24 keys: 16.5 G/s with 256, 15.4 with 512 -- smaller shared
// tables fit more blocks per SM, whose probe phases overlap).
template <class KIn, int VB, int W>
cudaError_t insert_block(const wc_table* t, const void* keys, const void* vals, uint64_t n, cudaStream_t s) {
  if (t->launch[WC_OP_INSERT].block_threads == 512) return insert_passes<KIn, VB, W, 512>(t, keys, vals, n, s);
  return insert_passes<KIn, VB, W, 256>(t, keys, vals, n, s);
}

template <class KIn, int VB>
cudaError_t insert_w(const wc_table* t, const void* keys, const void* vals, uint64_t n, cudaStream_t s) {
  switch (t->W) {
    case 2: return insert_block<KIn, VB, 2>(t, keys, vals, n, s);
    case 4: return insert_block<KIn, VB, 4>(t, keys, vals, n, s);
    case 8: return insert_block<KIn, VB, 8>(t, keys, vals, n, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t mv_insert(const wc_table* t, const void* keys, const void* vals, uint64_t n, cudaStream_t s) {
  const int kb = t->cfg.key_bytes, vb = t->cfg.value_bytes;
  if (kb == 4 && vb == 4) return insert_w<uint32_t, 4>(t, keys, vals, n, s);
  if (kb == 4 && vb == 8) return insert_w<uint32_t, 8>(t, keys, vals, n, s);
  if (kb == 8 && vb == 4) return insert_w<unsigned long long, 4>(t, keys, vals, n, s);
  return insert_w<unsigned long long, 8>(t, keys, vals, n, s);
}

}  // namespace wc
