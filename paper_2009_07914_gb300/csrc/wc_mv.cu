#include "wc_internal.h"
namespace wc {
cudaError_t mv_insert(const wc_table*, const void*, const void*, uint64_t, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t mv_count(const wc_table*, const void*, uint64_t, uint64_t*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t mv_retrieve_multi(const wc_table*, const void*, uint64_t, const uint64_t*, void*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t mv_erase(const wc_table*, const void*, uint64_t, cudaStream_t) { return cudaErrorNotSupported; }
uint64_t scan_partials_needed(uint64_t n) { return n / 8192 + 2; }
}
