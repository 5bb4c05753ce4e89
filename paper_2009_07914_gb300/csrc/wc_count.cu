// Counting tables (the paper's CountingHashTable): the single-value engine with the
// counting slot layouts -- a stored key's count grows by the insert's weight (1 when no
// weights are given).  Lookups and erases use the single-value kernels (same slots).
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

#define WC_COUNT_CASE(L, Wv, Gv) \
  if (W == (Wv) && G == (Gv)) return sv_insert_op<L, (Gv), (Wv) / (Gv)>(t, keys, weights, n, s);

cudaError_t count_insert(const wc_table* t, const void* keys, const void* weights, uint64_t n, cudaStream_t s) {
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

}  // namespace wc
