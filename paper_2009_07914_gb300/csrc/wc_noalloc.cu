// wc_insert_noalloc: the blocked (region-split) single-value insert with its scratch in a
// fixed device array of this library instead of memory the table allocates on demand.
//
// Who needs it: callers that must not allocate device memory while they run -- e.g. a
// serving process that reserves its whole memory budget up front, code that runs between
// the steps of another framework's caching allocator and must not grow it, or an
// embedding whose allocation is done by someone else.  wc_insert's blocked scheme
// allocates its scratch (stream-ordered) the first time a large batch needs it; this
// entry point never allocates: it splits the batch inside a static buffer of
// WC_NOALLOC_SCRATCH_BYTES that exists in every context that loads the library.
//
// The buffer is shared by all calls on a device and keeps whatever the last call left in
// it; the counters a call needs zeroed are cleared by that call.  Two calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on the buffer
// and give wrong results: order them (same stream, or events).
#include <cuda.h>  // driver API types; the two driver calls are reached through the runtime
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "wc.h"
#include "wc_internal.h"
#include "wc_launch.cuh"
#include "wc_partition.cuh"
#include "wc_sv_kernels.cuh"

namespace wc {
namespace {

constexpr uint64_t kHeadBytes = 64ull << 10;  // hist (4 KiB) | cursors (8 KiB) | work counter
constexpr uint64_t kCursorOff = 8192, kWorkOff = 16384;
constexpr uint64_t kScratchBytes = kHeadBytes + WC_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Identity of the CUDA context current on this thread (cuCtxGetId: unique for the life of
// the process), through the runtime's driver entry-point query, so that the library needs
// no link against the driver library.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

cudaError_t current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (get_current == nullptr || get_id == nullptr) {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorNotSupported;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return cudaErrorDeviceUninitialized;
  if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Device address of g_noalloc_scratch in the current context of each device (host code
// cannot use the symbol itself as an address: in host code it names a host-side shadow).
// Looked up once per device, with that device current, and looked up again if the device's
// context changed since (after cudaDeviceReset the old address is gone).
std::mutex g_mu;
struct Cached {
  unsigned long long ctx;
  void* addr;
};
Cached g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned long long ctx = 0;
  cudaError_t e = current_context_id(&ctx);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[device].addr == nullptr || g_addr[device].ctx != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // loads this file's module on first use
    if (e != cudaSuccess) return e;
    g_addr[device] = Cached{ctx, p};
  }
  *out = g_addr[device].addr;
  return cudaSuccess;
}

template <class L, int G, int S, int H = 1>
cudaError_t run(const wc_table* t, const void* keys, const void* vals, uint64_t n, char* sc, cudaStream_t s) {
  using Key = typename L::Key;
  using Val = typename L::Val;
  const wc_launch& lc = t->launch[WC_OP_INSERT];
  const RegionMap m = region_map(t, lc.region_mib);
  auto* hist = reinterpret_cast<unsigned int*>(sc);
  auto* cursor = reinterpret_cast<unsigned long long*>(sc + kCursorOff);
  auto* work = reinterpret_cast<unsigned long long*>(sc + kWorkOff);
  Key* pk = reinterpret_cast<Key*>(sc + kHeadBytes);
  Val* pv = reinterpret_cast<Val*>(sc + kHeadBytes + (n * sizeof(Key) + 255) / 256 * 256);
  cudaError_t e = cudaMemsetAsync(sc, 0, kWorkOff + 8, s);
  if (e != cudaSuccess) return e;
  auto hk = k_part_hist<Key>;
  auto sk = k_part_scatter<Key, Val>;
  auto ik = k_sv_insert<L, G, S, H>;
  const size_t hsm = static_cast<size_t>(kHistWarps) * m.R * sizeof(unsigned int);
  const size_t ssm = scatter_smem_bytes<Key, Val>();
  e = cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kHistWarps * kMaxRegions * 4));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(ssm));
  if (e != cudaSuccess) return e;
  const uint64_t ntiles = (n + kPartTile - 1) / kPartTile;
  const unsigned hg = static_cast<unsigned>(std::min<uint64_t>(
      (n + kPartTile - 1) / kPartTile, static_cast<uint64_t>(occupancy_smem(hk, kPartThreads, hsm)) * t->sm_count));
  const unsigned sg = static_cast<unsigned>(
      std::min<uint64_t>(ntiles, static_cast<uint64_t>(occupancy_smem(sk, kPartThreads, ssm)) * t->sm_count));
  hk<<<hg, kPartThreads, hsm, s>>>(static_cast<const Key*>(keys), n, m, hist);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sk<<<sg, kPartThreads, ssm, s>>>(static_cast<const Key*>(keys), static_cast<const Val*>(vals), n, m, hist, cursor,
                                   pk, pv);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;  // no insert over a split that was never written
  const int block = lc.block_threads;
  const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : occupancy(ik, block);
  return launch_k(t, ik, static_cast<unsigned>(bps) * static_cast<unsigned>(t->sm_count), block, 0, s, desc_of(t),
                  static_cast<const Key*>(pk), static_cast<const Val*>(pv), n, static_cast<uint64_t>(0), work, 512u);
}

#define WC_NA_CASE(L, Wv, Gv) \
  if (W == (Wv) && G == (Gv)) return run<L, (Gv), (Wv) / (Gv)>(t, keys, vals, n, sc, s);
#define WC_NA_CASE_H(L, Wv, Gv, Hv) \
  if (W == (Wv) && G == (Gv)) return run<L, (Gv), (Wv) / (Gv) / (Hv), (Hv)>(t, keys, vals, n, sc, s);

cudaError_t dispatch(const wc_table* t, const void* keys, const void* vals, uint64_t n, char* sc, cudaStream_t s) {
  const int W = static_cast<int>(t->W);
  const int G = t->launch[WC_OP_INSERT].group_size;
  if (t->slot_bytes == 8) {
    WC_NA_CASE(LayoutP32, 4, 1) WC_NA_CASE(LayoutP32, 4, 2) WC_NA_CASE(LayoutP32, 4, 4)
    WC_NA_CASE(LayoutP32, 8, 1) WC_NA_CASE(LayoutP32, 8, 2) WC_NA_CASE(LayoutP32, 8, 4) WC_NA_CASE(LayoutP32, 8, 8)
    WC_NA_CASE_H(LayoutP32, 16, 1, 2)
    WC_NA_CASE(LayoutP32, 16, 2) WC_NA_CASE(LayoutP32, 16, 4) WC_NA_CASE(LayoutP32, 16, 8)
    WC_NA_CASE(LayoutP32, 16, 16)
    WC_NA_CASE(LayoutP32, 32, 4) WC_NA_CASE(LayoutP32, 32, 8) WC_NA_CASE(LayoutP32, 32, 16)
    WC_NA_CASE(LayoutP32, 32, 32)
  } else {
    WC_NA_CASE(LayoutP64, 2, 1) WC_NA_CASE(LayoutP64, 2, 2)
    WC_NA_CASE(LayoutP64, 4, 1) WC_NA_CASE(LayoutP64, 4, 2) WC_NA_CASE(LayoutP64, 4, 4)
    WC_NA_CASE_H(LayoutP64, 8, 1, 2)
    WC_NA_CASE(LayoutP64, 8, 2) WC_NA_CASE(LayoutP64, 8, 4) WC_NA_CASE(LayoutP64, 8, 8)
    WC_NA_CASE(LayoutP64, 16, 4) WC_NA_CASE(LayoutP64, 16, 8) WC_NA_CASE(LayoutP64, 16, 16)
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace wc

extern "C" wc_status wc_insert_noalloc(wc_table* t, const void* d_keys, const void* d_values, uint64_t n,
                                       void* stream) {
  wc::TraceRange trace("wc_insert_noalloc");
  if (t == nullptr || t->cfg.kind != WC_SINGLE_VALUE || t->d_vals != nullptr)
    return t == nullptr ? WC_ERR_INVALID_ARG : WC_ERR_UNSUPPORTED;
  const uint64_t pair = static_cast<uint64_t>(t->cfg.key_bytes) + static_cast<uint64_t>(t->cfg.value_bytes);
  // keys and values each start on a 256-byte boundary inside the buffer
  if (n > (WC_NOALLOC_SCRATCH_BYTES - 512) / pair) return WC_ERR_INVALID_ARG;
  if (n == 0) return WC_OK;
  if (d_keys == nullptr || d_values == nullptr) return WC_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_keys) % static_cast<uint64_t>(t->cfg.key_bytes) ||
      reinterpret_cast<uintptr_t>(d_values) % static_cast<uint64_t>(t->cfg.value_bytes))
    return WC_ERR_INVALID_ARG;
  // buffers the kernels cannot reach (pageable host memory, another GPU's memory) would
  // fault on the device: refused here, as wc_insert refuses them
  if (!wc::device_accessible(t->device, d_keys) || !wc::device_accessible(t->device, d_values))
    return WC_ERR_INVALID_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return WC_ERR_CUDA;
  // made current even when it already is: that also makes its primary context current
  if (cudaSetDevice(t->device) != cudaSuccess) return WC_ERR_CUDA;
  void* sc = nullptr;
  cudaError_t e = wc::scratch_address(t->device, &sc);
  if (e == cudaSuccess)
    e = wc::dispatch(t, d_keys, d_values, n, static_cast<char*>(sc), static_cast<cudaStream_t>(stream));
  if (prev != t->device) cudaSetDevice(prev);
  return wc::cuda_status(e);  // an out-of-memory error keeps its own code
}
