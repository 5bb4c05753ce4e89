// Instantiation and dispatch of the single-value kernels for one slot layout.
#pragma once

#include "wc_launch.cuh"
#include "wc_partition.cuh"
#include "wc_sv_kernels.cuh"

namespace wc {

template <class L, int G, int S>
cudaError_t sv_run(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                   uint8_t* found, cudaStream_t s) {
  using Key = typename L::Key;
  using Val = typename L::Val;
  const wc_launch& lc = t->launch[op];
  const int block = lc.block_threads;
  const TableDesc d = desc_of(t);
  const Key* k = static_cast<const Key*>(keys);
  if (op == WC_OP_INSERT) {
    auto kern = k_sv_insert<L, G, S>;
    const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
    const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
    if (scheme_for(t, op, n) != WC_SCHEME_BLOCKED)
      return launch_k(t, kern, g.blocks, block, 0, s, d, k, static_cast<const Val*>(vals), n, g.per_warp,
                      static_cast<unsigned long long*>(nullptr), 0u);
    // blocked scheme: split the batch by table region, then insert it region by region
    RegionSplit<Key, Val> sp;
    cudaError_t e = region_split(t, lc.region_mib, k, static_cast<const Val*>(vals), n, s, sp);
    if (e != cudaSuccess) return e;
    const unsigned grid = static_cast<unsigned>(bps) * static_cast<unsigned>(t->sm_count);
    return launch_k(t, kern, grid, block, 0, s, d, sp.keys, sp.vals, n, static_cast<uint64_t>(0), sp.counters, 512u);
  }
  if (op == WC_OP_RETRIEVE) {
    auto kern = k_sv_retrieve<L, G, S>;
    const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
    const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
    return launch_k(t, kern, g.blocks, block, 0, s, d, k, n, g.per_warp, static_cast<Val*>(out), found);
  }
  auto kern = k_sv_erase<L, G, S>;
  const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
  const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
  return launch_k(t, kern, g.blocks, block, 0, s, d, k, n, g.per_warp);
}

}  // namespace wc

#define WC_SV_CASE(L, Wv, Gv)                                               \
  if (W == (Wv) && G == (Gv)) return sv_run<L, (Gv), (Wv) / (Gv)>(t, op, keys, vals, n, out, found, s);
