// Instantiation and dispatch of the single-value kernels for one slot layout.
#pragma once

#include <algorithm>

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
    RegionMap m;
    m.seed = t->cfg.seed;
    m.p = static_cast<uint32_t>(t->windows);
    const uint64_t region_bytes = static_cast<uint64_t>(lc.region_mib > 0 ? lc.region_mib : 32) << 20;
    uint64_t wpr = std::max<uint64_t>(1, region_bytes / (t->W * t->slot_bytes));
    if ((t->windows + wpr - 1) / wpr > static_cast<uint64_t>(kMaxRegions)) wpr = (t->windows + kMaxRegions - 1) / kMaxRegions;
    m.wpr = static_cast<uint32_t>(wpr);
    m.R = static_cast<uint32_t>((t->windows + wpr - 1) / wpr);
    const uint64_t hist_off = 0, cur_off = 8192, work_off = cur_off + 8192;
    const uint64_t keys_off = work_off + 256;
    const uint64_t vals_off = keys_off + ((n * sizeof(Key) + 255) / 256) * 256;
    const uint64_t need = vals_off + n * sizeof(Val);
    cudaError_t e = ensure_scratch(t, need, s);
    if (e != cudaSuccess) return e;
    char* sc = static_cast<char*>(t->d_scratch);
    auto* hist = reinterpret_cast<unsigned int*>(sc + hist_off);
    auto* cursor = reinterpret_cast<unsigned long long*>(sc + cur_off);
    auto* work = reinterpret_cast<unsigned long long*>(sc + work_off);
    Key* pk = reinterpret_cast<Key*>(sc + keys_off);
    Val* pv = reinterpret_cast<Val*>(sc + vals_off);
    e = cudaMemsetAsync(sc, 0, keys_off, s);
    if (e != cudaSuccess) return e;
    const uint64_t ntiles = (n + kPartTile - 1) / kPartTile;
    auto hk = k_part_hist<Key>;
    auto sk = k_part_scatter<Key, Val>;
    const size_t hsm = static_cast<size_t>(kHistWarps) * m.R * sizeof(unsigned int);
    const size_t ssm = scatter_smem_bytes<Key, Val>();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kHistWarps * kMaxRegions * 4));
      cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(ssm));
      attr = true;
    }
    const unsigned hg = static_cast<unsigned>(std::min<uint64_t>((n + kPartThreads - 1) / kPartThreads,
                                                                 static_cast<uint64_t>(occupancy_smem(hk, kPartThreads, hsm)) * t->sm_count));
    const unsigned sg = static_cast<unsigned>(std::min<uint64_t>(ntiles,
                                                                 static_cast<uint64_t>(occupancy_smem(sk, kPartThreads, ssm)) * t->sm_count));
    hk<<<hg, kPartThreads, hsm, s>>>(k, n, m, hist);
    sk<<<sg, kPartThreads, ssm, s>>>(k, static_cast<const Val*>(vals), n, m, hist, cursor, pk, pv);
    const unsigned grid = static_cast<unsigned>(bps) * static_cast<unsigned>(t->sm_count);
    return launch_k(t, kern, grid, block, 0, s, d, static_cast<const Key*>(pk), static_cast<const Val*>(pv), n,
                    static_cast<uint64_t>(0), work, 512u);
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
