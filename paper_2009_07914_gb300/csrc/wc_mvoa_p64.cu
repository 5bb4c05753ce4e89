// Open-addressing multi-value kernels over 16-byte slots (uint64 key, uint64 value).
#include "wc_mvoa_dispatch.cuh"

namespace wc {

// One lane per key for narrow windows, else 32 bytes of the window per lane.
bool oa_p64_shape_ok(int W, int G) {
  switch (W) {
    case 2: return G == 1;
    case 4: return G == 1 || G == 2;
    case 8: return G == 2 || G == 4;
    case 16: return G == 4 || G == 8;
    default: return false;
  }
}

cudaError_t oa_p64_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, uint64_t* offs,
                          void* out, cudaStream_t s) {
  const int W = static_cast<int>(t->W);
  const int G = t->launch[op].group_size;
  WC_OA_CASE(LayoutP64, 2, 1)
  WC_OA_CASE(LayoutP64, 4, 1) WC_OA_CASE(LayoutP64, 4, 2)
  WC_OA_CASE(LayoutP64, 8, 2) WC_OA_CASE(LayoutP64, 8, 4)
  WC_OA_CASE(LayoutP64, 16, 4) WC_OA_CASE(LayoutP64, 16, 8)
  return cudaErrorInvalidValue;
}

cudaError_t oa_p64_num_keys(const wc_table* t, cudaStream_t s) { return oa_count_keys<LayoutP64>(t, s); }

}  // namespace wc
