// Single-value kernels over 16-byte slots (uint64 key, uint64 value; 128-bit CAS).
#include "wc_sv_dispatch.cuh"

namespace wc {

bool sv_p64_shape_ok(int W, int G) {
  switch (W) {
    case 2: return G == 1 || G == 2;
    case 4: return G == 1 || G == 2 || G == 4;
    case 8: return G == 1 || G == 2 || G == 4 || G == 8;
    case 16: return G == 4 || G == 8 || G == 16;
    default: return false;
  }
}

cudaError_t sv_p64_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                          uint8_t* found, cudaStream_t s) {
  const int W = static_cast<int>(t->W);
  const int G = t->launch[op].group_size;
  WC_SV_CASE(LayoutP64, 2, 1) WC_SV_CASE(LayoutP64, 2, 2)
  WC_SV_CASE(LayoutP64, 4, 1) WC_SV_CASE(LayoutP64, 4, 2) WC_SV_CASE(LayoutP64, 4, 4)
  // one lane per key walks a 128-byte window (one L2 line) in two 64-byte steps
  WC_SV_CASE_H(LayoutP64, 8, 1, 2)
  WC_SV_CASE(LayoutP64, 8, 2) WC_SV_CASE(LayoutP64, 8, 4) WC_SV_CASE(LayoutP64, 8, 8)
  WC_SV_CASE(LayoutP64, 16, 4) WC_SV_CASE(LayoutP64, 16, 8) WC_SV_CASE(LayoutP64, 16, 16)
  return cudaErrorInvalidValue;
}

}  // namespace wc
