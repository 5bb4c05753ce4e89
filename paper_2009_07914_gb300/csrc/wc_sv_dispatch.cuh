// Instantiation and dispatch of the single-value kernels for one slot layout.
#pragma once

#include "wc_launch.cuh"
#include "wc_partition.cuh"
#include "wc_sv_kernels.cuh"

namespace wc {

// Retrieve by the blocked scheme: (1) split the queries by table region, keeping each
// query's input position; (2) probe region by region in L2, writing results in split
// order; (3) split the results by output-position region (the counts are known: every
// position occurs once); (4) place them, each moment's stores falling into one or two
// L2-sized output regions.  Needs n < 2^31 (bit 31 of a position word carries "found").
template <class L, int G, int S, int H = 1>
cudaError_t sv_retrieve_blocked(const wc_table* t, const wc_launch& lc, const typename L::Key* k, uint64_t n,
                                typename L::Val* out, uint8_t* found, cudaStream_t s) {
  using Key = typename L::Key;
  using Val = typename L::Val;
  uint64_t per = std::max<uint64_t>(1, (32ull << 20) / (sizeof(Val) + 1));
  if ((n + per - 1) / per > static_cast<uint64_t>(kMaxRegions)) per = (n + kMaxRegions - 1) / kMaxRegions;
  const IndexMap im{static_cast<uint32_t>(per), static_cast<uint32_t>((n + per - 1) / per)};
  const uint64_t rv_off = align256(n * sizeof(uint32_t));
  const uint64_t extra = rv_off + align256(n * sizeof(Val));
  RegionSplit<Key, uint32_t> sp;
  cudaError_t e = region_split<Key, uint32_t, kValsIota>(t, lc.region_mib, k, nullptr, n, s, sp, extra);
  if (e != cudaSuccess) return e;
  auto* rk = reinterpret_cast<uint32_t*>(sp.extra);
  auto* rv = reinterpret_cast<Val*>(sp.extra + rv_off);
  // the split queries are dead after the probe pass: the position split reuses them
  auto* ck = reinterpret_cast<uint32_t*>(const_cast<Key*>(sp.keys));
  auto* cv = reinterpret_cast<Val*>(reinterpret_cast<char*>(ck) + align256(n * sizeof(uint32_t)));
  const int block = lc.block_threads;
  auto kern = k_sv_retrieve_swept<L, G, S, H>;
  const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
  e = launch_k(t, kern, static_cast<unsigned>(bps) * static_cast<unsigned>(t->sm_count), block, 0, s, desc_of(t),
               sp.keys, sp.vals, n, sp.counters, 512u, rk, rv);
  if (e != cudaSuccess) return e;
  k_index_hist<<<(im.R + 255) / 256, 256, 0, s>>>(sp.hist2, im.R, im.per, n);
  auto sk = k_part_scatter<uint32_t, Val, IndexMap, kValsRead>;
  const size_t ssm = scatter_smem_bytes<uint32_t, Val>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(ssm));
    attr = true;
  }
  const uint64_t ntiles = (n + kPartTile - 1) / kPartTile;
  const unsigned sg = static_cast<unsigned>(
      std::min<uint64_t>(ntiles, static_cast<uint64_t>(occupancy_smem(sk, kPartThreads, ssm)) * t->sm_count));
  sk<<<sg, kPartThreads, ssm, s>>>(rk, rv, n, im, sp.hist2, sp.cursor2, ck, cv);
  auto pk = k_place_results<Val>;
  const unsigned pg = static_cast<unsigned>(std::min<uint64_t>(
      (n + 255) / 256, static_cast<uint64_t>(occupancy(pk, 256)) * t->sm_count));
  pk<<<pg, 256, 0, s>>>(ck, cv, n, out, found);
  return cudaGetLastError();
}

// Insert (direct, or the blocked scheme: split the batch by table region, then insert it
// region by region).  vals == nullptr (counting tables): every key counts 1.
template <class L, int G, int S, int H = 1>
cudaError_t sv_insert_op(const wc_table* t, const void* keys, const void* vals, uint64_t n, cudaStream_t s) {
  using Key = typename L::Key;
  using Val = typename L::Val;
  const wc_launch& lc = t->launch[WC_OP_INSERT];
  const int block = lc.block_threads;
  const TableDesc d = desc_of(t);
  const Key* k = static_cast<const Key*>(keys);
  auto kern = k_sv_insert<L, G, S, H>;
  const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
  const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
  if (scheme_for(t, WC_OP_INSERT, n) != WC_SCHEME_BLOCKED)
    return launch_k(t, kern, g.blocks, block, 0, s, d, k, static_cast<const Val*>(vals), n, g.per_warp,
                    static_cast<unsigned long long*>(nullptr), 0u);
  RegionSplit<Key, Val> sp;
  cudaError_t e = vals != nullptr ? region_split(t, lc.region_mib, k, static_cast<const Val*>(vals), n, s, sp)
                                  : region_split<Key, Val, kValsOne>(t, lc.region_mib, k, nullptr, n, s, sp);
  if (e != cudaSuccess) return e;
  const unsigned grid = static_cast<unsigned>(bps) * static_cast<unsigned>(t->sm_count);
  return launch_k(t, kern, grid, block, 0, s, d, sp.keys, sp.vals, n, static_cast<uint64_t>(0), sp.counters, 512u);
}

// H > 1: a window of G * S * H slots is walked in H steps of G * S slots.
template <class L, int G, int S, int H = 1>
cudaError_t sv_run(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                   uint8_t* found, cudaStream_t s) {
  using Key = typename L::Key;
  using Val = typename L::Val;
  if (op == WC_OP_INSERT) return sv_insert_op<L, G, S, H>(t, keys, vals, n, s);
  const wc_launch& lc = t->launch[op];
  const int block = lc.block_threads;
  const TableDesc d = desc_of(t);
  const Key* k = static_cast<const Key*>(keys);
  if (op == WC_OP_RETRIEVE) {
    const int scheme = scheme_for(t, op, n);
    if (scheme == WC_SCHEME_BLOCKED && n < (1ull << 31) && out != nullptr)
      return sv_retrieve_blocked<L, G, S, H>(t, lc, k, n, static_cast<Val*>(out), found, s);
    auto kern = scheme == WC_SCHEME_DEDUP ? k_sv_retrieve_dedup<L, G, S, H> : k_sv_retrieve<L, G, S, H>;
    // two keys per group: windows of at most 32 bytes per lane (register budget)
    if constexpr (S * L::kWords * 8 <= 32 || (L::kHalf && S * 4 <= 32))
      if (scheme != WC_SCHEME_DEDUP && lc.keys_in_flight == 2) kern = k_sv_retrieve2<L, G, S, H>;
    const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
    const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
    return launch_k(t, kern, g.blocks, block, 0, s, d, k, n, g.per_warp, static_cast<Val*>(out), found);
  }
  auto kern = k_sv_erase<L, G, S, H>;
  const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(kern, block);
  const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
  return launch_k(t, kern, g.blocks, block, 0, s, d, k, n, g.per_warp);
}

}  // namespace wc

#define WC_SV_CASE(L, Wv, Gv)                                               \
  if (W == (Wv) && G == (Gv)) return sv_run<L, (Gv), (Wv) / (Gv)>(t, op, keys, vals, n, out, found, s);
// A window of Wv slots walked by Gv lanes in Hv steps.
#define WC_SV_CASE_H(L, Wv, Gv, Hv) \
  if (W == (Wv) && G == (Gv)) return sv_run<L, (Gv), (Wv) / (Gv) / (Hv), (Hv)>(t, op, keys, vals, n, out, found, s);
