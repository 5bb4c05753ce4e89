// Multi-value bulk insert: dispatch of the count / allocate / place passes.
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
  auto count = k_mv_aggregate<KIn, W, kThreads>;
  auto place = k_mv_place<VB, kThreads>;
  const size_t smem_c = A::smem_bytes(sizeof(KIn));
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(count, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_c));
    attr_done = true;
  }
  // The counting pass's record for the placing pass (TileRecord): a (slot, count) entry
  // per distinct key of a tile and one word per element.
  const uint64_t ntiles = (n + A::kTile - 1) / A::kTile;
  const uint64_t list_bytes = align256(ntiles * A::kTile * sizeof(uint2));
  const uint64_t elem_bytes = align256(n * sizeof(uint32_t));
  const uint64_t rec_bytes = list_bytes + elem_bytes + align256(ntiles * sizeof(uint32_t));
  // Large batches into a key store larger than L2 are first split by key-store region
  // (the region split of the single-value insert): the passes then probe one L2-resident
  // region of the key store at a time, and pass 3 writes one range of the pool at a time
  // (pass 2 lays buckets out in key-store order).
  unsigned long long* counters = nullptr;
  char* rec_base = nullptr;
  cudaError_t e = cudaSuccess;
  if (n >= (1ull << 20) && t->table_bytes > (64ull << 20)) {
    RegionSplit<KIn, V> sp;
    e = region_split(t, 32, k, static_cast<const V*>(vals), n, s, sp, rec_bytes);
    if (e != cudaSuccess) return e;
    k = sp.keys;
    vals = sp.vals;
    counters = sp.counters;
    rec_base = sp.extra;
  } else {
    e = ensure_scratch(t, rec_bytes, s);
    if (e != cudaSuccess) return e;
    rec_base = static_cast<char*>(t->d_scratch);
  }
  TileRecord rec;
  rec.list = reinterpret_cast<uint2*>(rec_base);
  rec.elem = reinterpret_cast<uint32_t*>(rec_base + list_bytes);
  rec.len = reinterpret_cast<uint32_t*>(rec_base + list_bytes + elem_bytes);
  const int bps_c = occupancy_smem(count, kThreads, smem_c);
  const int bps_p = occupancy(place, kThreads);
  const unsigned g_c = static_cast<unsigned>(std::min<uint64_t>(ntiles, static_cast<uint64_t>(bps_c) * t->sm_count));
  const unsigned g_p = static_cast<unsigned>(std::min<uint64_t>(ntiles, static_cast<uint64_t>(bps_p) * t->sm_count));
  e = cudaMemsetAsync(pd.pending, 0, t->capacity * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  e = launch_k(t, count, g_c, kThreads, smem_c, s, d, pd, k, n, counters, rec);
  if (e != cudaSuccess) return e;
  const uint64_t per_block = static_cast<uint64_t>(kAllocThreads) * kAllocItems;
  const unsigned g_a = static_cast<unsigned>((t->capacity + per_block - 1) / per_block);
  e = launch_k(t, t->growth == kGrowExact ? k_mv_alloc<VB> : k_mv_alloc_growth<VB>, g_a, kAllocThreads, 0, s, d, pd,
               t->capacity);
  if (e != cudaSuccess) return e;
  return launch_k(t, place, g_p, kThreads, 0, s, d, pd, rec, vals, n, counters ? counters + 1 : counters);
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
