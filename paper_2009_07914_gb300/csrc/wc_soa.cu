// Struct-of-arrays single-value tables (WC_OPT_SOA): the single-value engine over key-only
// slots (4 or 8 bytes) with the values in a second array of the same length.
#include "wc_sv_dispatch.cuh"

namespace wc {

bool soa_shape_ok(int slot_bytes, int W, int G) {
  if (slot_bytes == 4) {
    switch (W) {
      case 8: return G == 1 || G == 2;
      case 16: return G == 1 || G == 2 || G == 4;
      case 32: return G == 4 || G == 8;
      default: return false;
    }
  }
  switch (W) {
    case 4: return G == 1 || G == 2;
    case 8: return G == 1 || G == 2;
    case 16: return G == 2 || G == 4;
    case 32: return G == 4 || G == 8;
    default: return false;
  }
}

cudaError_t soa_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n, void* out,
                       uint8_t* found, cudaStream_t s) {
  const int W = static_cast<int>(t->W);
  const int G = t->launch[op].group_size;
  if (t->slot_bytes == 4) {
    WC_SV_CASE(LayoutS32, 8, 1) WC_SV_CASE(LayoutS32, 8, 2)
    WC_SV_CASE(LayoutS32, 16, 1) WC_SV_CASE(LayoutS32, 16, 2) WC_SV_CASE(LayoutS32, 16, 4)
    WC_SV_CASE(LayoutS32, 32, 4) WC_SV_CASE(LayoutS32, 32, 8)
  } else {
    WC_SV_CASE(LayoutS64, 4, 1) WC_SV_CASE(LayoutS64, 4, 2)
    WC_SV_CASE(LayoutS64, 8, 1) WC_SV_CASE(LayoutS64, 8, 2)
    WC_SV_CASE(LayoutS64, 16, 2) WC_SV_CASE(LayoutS64, 16, 4)
    WC_SV_CASE(LayoutS64, 32, 4) WC_SV_CASE(LayoutS64, 32, 8)
  }
  return cudaErrorInvalidValue;
}

}  // namespace wc
