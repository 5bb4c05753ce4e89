// Single-value kernels over packed 64-bit slots (uint32 key | uint32 value).
#include "wc_sv_dispatch.cuh"

namespace wc {

bool sv_p32_shape_ok(int W, int G) {
  switch (W) {
    case 4: return G == 1 || G == 2 || G == 4;
    case 8: return G == 1 || G == 2 || G == 4 || G == 8;
    case 16: return G == 1 || G == 2 || G == 4 || G == 8 || G == 16;
    case 32: return G == 4 || G == 8 || G == 16 || G == 32;
    default: return false;
  }
}

cudaError_t sv_p32_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                          uint8_t* found, cudaStream_t s) {
  const int W = static_cast<int>(t->W);
  const int G = t->launch[op].group_size;
  WC_SV_CASE(LayoutP32, 4, 1) WC_SV_CASE(LayoutP32, 4, 2) WC_SV_CASE(LayoutP32, 4, 4)
  WC_SV_CASE(LayoutP32, 8, 1) WC_SV_CASE(LayoutP32, 8, 2) WC_SV_CASE(LayoutP32, 8, 4) WC_SV_CASE(LayoutP32, 8, 8)
  // one lane per key walks a 128-byte window (one L2 line) in two 64-byte steps
  WC_SV_CASE_H(LayoutP32, 16, 1, 2)
  WC_SV_CASE(LayoutP32, 16, 2) WC_SV_CASE(LayoutP32, 16, 4) WC_SV_CASE(LayoutP32, 16, 8)
  WC_SV_CASE(LayoutP32, 16, 16)
  WC_SV_CASE(LayoutP32, 32, 4) WC_SV_CASE(LayoutP32, 32, 8) WC_SV_CASE(LayoutP32, 32, 16)
  WC_SV_CASE(LayoutP32, 32, 32)
  return cudaErrorInvalidValue;
}

}  // namespace wc
