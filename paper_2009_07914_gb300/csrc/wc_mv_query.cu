// Multi-value queries: count_values (+ scan), retrieve_multi, erase.
#include "wc_launch.cuh"
#include "wc_mv_kernels.cuh"

namespace wc {

bool mv_shape_ok(int W, int G) {
  switch (W) {
    case 2: return G == 1 || G == 2;
    case 4: return G == 1 || G == 2 || G == 4;
    case 8: return G == 2 || G == 4 || G == 8;
    default: return false;
  }
}

namespace {

template <class KIn, int G, int S>
cudaError_t probe_op(const wc_table* t, int op, const void* keys, uint64_t n, uint64_t* offs, cudaStream_t s) {
  const TableDesc d = desc_of(t);
  const KIn* k = static_cast<const KIn*>(keys);
  const int block = t->launch[op].block_threads;
  if (op == WC_OP_COUNT) {
    auto kern = k_mv_count<KIn, G, S>;
    const int bps = t->launch[op].blocks_per_sm > 0 ? t->launch[op].blocks_per_sm : occupancy(kern, block);
    const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
    return launch_k(t, kern, g.blocks, block, 0, s, d, k, n, g.per_warp, offs);
  }
  auto kern = k_mv_erase<KIn, G, S>;
  const int bps = t->launch[op].blocks_per_sm > 0 ? t->launch[op].blocks_per_sm : occupancy(kern, block);
  const EngineGrid g = engine_grid(n, G, block, bps, t->sm_count);
  return launch_k(t, kern, g.blocks, block, 0, s, d, k, n, g.per_warp);
}

#define WC_MV_CASE(Wv, Gv) \
  if (W == (Wv) && G == (Gv)) return probe_op<KIn, (Gv), (Wv) / (Gv)>(t, op, keys, n, offs, s);

template <class KIn>
cudaError_t probe_dispatch(const wc_table* t, int op, const void* keys, uint64_t n, uint64_t* offs, cudaStream_t s) {
  const int W = static_cast<int>(t->W);
  const int G = t->launch[op].group_size;
  WC_MV_CASE(2, 1) WC_MV_CASE(2, 2)
  WC_MV_CASE(4, 1) WC_MV_CASE(4, 2) WC_MV_CASE(4, 4)
  WC_MV_CASE(8, 2) WC_MV_CASE(8, 4) WC_MV_CASE(8, 8)
  return cudaErrorInvalidValue;
}

template <class KIn, int VB, int W>
cudaError_t gather(const wc_table* t, const void* keys, uint64_t n, const uint64_t* offs, void* out, cudaStream_t s) {
  auto kern = t->growth == kGrowExact ? k_mv_retrieve_multi<KIn, VB, W, false> : k_mv_retrieve_multi<KIn, VB, W, true>;
  const int bps = occupancy(kern, kRmThreads);
  const unsigned grid = static_cast<unsigned>(bps * t->sm_count);
  return launch_k(t, kern, grid, kRmThreads, 0, s, desc_of(t), pool_of(t), static_cast<const KIn*>(keys), n, offs,
                  out);
}

template <class KIn, int VB>
cudaError_t gather_w(const wc_table* t, const void* keys, uint64_t n, const uint64_t* offs, void* out,
                     cudaStream_t s) {
  switch (t->W) {
    case 2: return gather<KIn, VB, 2>(t, keys, n, offs, out, s);
    case 4: return gather<KIn, VB, 4>(t, keys, n, offs, out, s);
    case 8: return gather<KIn, VB, 8>(t, keys, n, offs, out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t mv_count(const wc_table* t, const void* keys, uint64_t n, uint64_t* offsets, cudaStream_t s) {
  if (n > 0) {
    cudaError_t e = t->cfg.key_bytes == 4
                        ? probe_dispatch<uint32_t>(t, WC_OP_COUNT, keys, n, offsets, s)
                        : probe_dispatch<unsigned long long>(t, WC_OP_COUNT, keys, n, offsets, s);
    if (e != cudaSuccess) return e;
  }
  return scan_exclusive_u64(offsets, n, t->d_partials, t->partials_cap, s);
}

cudaError_t mv_erase(const wc_table* t, const void* keys, uint64_t n, cudaStream_t s) {
  return t->cfg.key_bytes == 4 ? probe_dispatch<uint32_t>(t, WC_OP_ERASE, keys, n, nullptr, s)
                               : probe_dispatch<unsigned long long>(t, WC_OP_ERASE, keys, n, nullptr, s);
}

cudaError_t mv_retrieve_multi(const wc_table* t, const void* keys, uint64_t n, const uint64_t* offsets, void* out,
                              cudaStream_t s) {
  const int kb = t->cfg.key_bytes, vb = t->cfg.value_bytes;
  if (kb == 4 && vb == 4) return gather_w<uint32_t, 4>(t, keys, n, offsets, out, s);
  if (kb == 4 && vb == 8) return gather_w<uint32_t, 8>(t, keys, n, offsets, out, s);
  if (kb == 8 && vb == 4) return gather_w<unsigned long long, 4>(t, keys, n, offsets, out, s);
  return gather_w<unsigned long long, 8>(t, keys, n, offsets, out, s);
}

}  // namespace wc
