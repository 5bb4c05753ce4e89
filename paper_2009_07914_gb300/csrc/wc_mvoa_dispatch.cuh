// Instantiation and dispatch of the open-addressing multi-value kernels for one slot
// layout.  Ops: WC_OP_INSERT (append), WC_OP_COUNT (per-query counts; the caller scans),
// WC_OP_RETRIEVE (CSR write of the matches), WC_OP_ERASE (tombstone every copy).
#pragma once

#include "wc_launch.cuh"
#include "wc_mvoa_kernels.cuh"
#include "wc_partition.cuh"

namespace wc {

template <class L, int G, int S>
cudaError_t oa_run(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, uint64_t* offs,
                   void* out, cudaStream_t s) {
  using Key = typename L::Key;
  using Val = typename L::Val;
  const wc_launch& lc = t->launch[op];
  const int block = lc.block_threads;
  const TableDesc d = desc_of(t);
  const Key* k = static_cast<const Key*>(keys);
  if (op == WC_OP_INSERT) {
    auto kern = k_oa_insert<L, G, S>;
    const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
    const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
    if (scheme_for(t, op, n) != WC_SCHEME_BLOCKED)
      return launch_k(t, kern, g.blocks, block, 0, s, d, k, static_cast<const Val*>(vals), n, g.per_warp,
                      static_cast<unsigned long long*>(nullptr), 0u);
    RegionSplit<Key, Val> sp;
    cudaError_t e = region_split(t, lc.region_mib, k, static_cast<const Val*>(vals), n, s, sp);
    if (e != cudaSuccess) return e;
    const unsigned grid = static_cast<unsigned>(bps) * static_cast<unsigned>(t->sm_count);
    return launch_k(t, kern, grid, block, 0, s, d, sp.keys, sp.vals, n, static_cast<uint64_t>(0), sp.counters, 512u);
  }
  if (op == WC_OP_COUNT || op == WC_OP_RETRIEVE) {
    auto kern = op == WC_OP_COUNT ? k_oa_walk<L, G, S, false> : k_oa_walk<L, G, S, true>;
    const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
    const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
    return launch_k(t, kern, g.blocks, block, 0, s, d, k, n, offs, static_cast<Val*>(out));
  }
  auto kern = k_oa_erase<L, G, S>;
  const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
  const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
  return launch_k(t, kern, g.blocks, block, 0, s, d, k, n);
}

// Distinct live keys into the table's nkeys word (zeroed first).
template <class L>
cudaError_t oa_count_keys(const wc_table* t, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(t->d_nkeys, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  auto kern = k_oa_num_keys<L>;
  const uint64_t want = (t->capacity + 255) / 256;
  const uint64_t most = static_cast<uint64_t>(occupancy(kern, 256)) * t->sm_count;
  const unsigned grid = static_cast<unsigned>(want < most ? want : most);
  return launch_k(t, kern, grid, 256u, 0, s, desc_of(t), t->capacity);
}

}  // namespace wc

#define WC_OA_CASE(L, Wv, Gv) \
  if (W == (Wv) && G == (Gv)) return oa_run<L, (Gv), (Wv) / (Gv)>(t, op, keys, vals, n, offs, out, s);
