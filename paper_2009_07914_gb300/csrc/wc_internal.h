// Host-side internals shared by the library's translation units: the table object
// behind the opaque wc_table handle, the by-value descriptors kernels receive, and the
// launcher entry points of each kernel family.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "wc.h"

#include <nvtx3/nvToolsExt.h>

namespace wc {

// Named range on the NVTX timeline around a host call of the C ABI (a no-op unless a
// profiler is attached), so profiles show which call launched which kernels.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Host calls run on the table's device and give the caller's device back afterwards.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// wc_status of a CUDA runtime result (allocation failures: WC_ERR_OUT_OF_MEMORY).
inline wc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return WC_OK;
  if (e == cudaErrorMemoryAllocation) return WC_ERR_OUT_OF_MEMORY;
  return WC_ERR_CUDA;
}

// A buffer the kernels of a table on `device` may read or write: device memory of that
// device (or managed memory), or host memory mapped into the device's address space at
// the same address (pinned with cudaHostAlloc / cudaMallocHost, or registered mapped) --
// on GB300 the kernels then move it over NVLink-C2C themselves.  Anything else would
// fault on the device and is refused by the host calls.
inline bool device_accessible(int device, const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type == cudaMemoryTypeDevice) return a.device == device;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer == p;
  return false;  // unregistered host memory
}

// What every single-value / key-store kernel needs, passed by value.
struct TableDesc {
  void* slots;                       // p * W slots, 256-byte aligned
  uint64_t seed;                     // hash seed
  uint32_t* status;                  // device status word (WC_FLAG_* bits)
  unsigned long long* size;          // SV: live keys; MV: stored pairs
  unsigned long long* nkeys;         // MV: distinct live keys
  uint32_t* ovf;                     // SV: eight overflow bits per window (see wc_device.cuh); else null
  void* vals;                        // SoA tables: the value array (slot i's value); else null
  uint32_t p;                        // windows (prime)
  uint32_t W;                        // slots per window
};

// Multi-value extras.
struct PoolDesc {
  void* pool;                        // value elements (value_bytes each)
  unsigned long long* cursor;        // next free pool element
  uint32_t* pending;                 // per key-store slot: this call's count / cursor
  uint64_t capacity;                 // pool elements
  int32_t value_bytes;               // 4 or 8
  // bucket growth strategy (kGrowExact: one exact bucket per call and key)
  int32_t growth;                    // kGrowExact, kGrowConst (lambda = 1) or kGrowTable
  uint32_t nbuckets;                 // kGrowTable: entries of cum_size / cum_foot
  uint64_t s0;                       // first bucket size (kGrowConst: every bucket's)
  uint64_t foot0, foot;              // kGrowConst: pool elements of bucket 0 / of later buckets
  const uint64_t* cum_size;          // kGrowTable: values in buckets 0..i
  const uint64_t* cum_foot;          // kGrowTable: pool elements of buckets 0..i
  uint32_t* base;                    // growth: per key-store slot, the key's count before this call
};

enum { kGrowExact = 0, kGrowConst = 1, kGrowTable = 2 };
constexpr uint32_t kMaxGrowBuckets = 1024;

struct HostPipe;  // staging of wc_insert_host / wc_retrieve_host (wc_host.cu)

// Shape of one launch after the table's tuning was applied.
struct LaunchShape {
  int group;           // lanes per key
  int block;           // threads per block
  int blocks_per_sm;   // 0 = occupancy limit
};

}  // namespace wc

struct wc_table {
  wc_table_config cfg;
  int device;
  int sm_count;
  uint64_t windows;      // p
  uint64_t W;
  uint64_t capacity;     // p * W
  uint64_t slot_bytes;
  uint64_t table_bytes;
  uint64_t pool_capacity;
  uint64_t device_bytes;
  uint64_t clear_bytes;  // prefix of d_block zeroed by a clear (slots, meta, pending)
  void* d_block;         // the single allocation holding everything below
  void* d_slots;
  uint32_t* d_status;
  unsigned long long* d_size;
  unsigned long long* d_nkeys;
  unsigned long long* d_cursor;
  uint32_t* d_ovf;       // SV: overflow bits, one byte per window
  void* d_vals;          // SoA single-value tables: value array (capacity entries)
  uint32_t* d_pending;   // MV: capacity entries
  uint32_t* d_base;      // MV with bucket growth: capacity entries
  uint64_t* d_growth;    // MV with kGrowTable: cum_size[nbuckets] then cum_foot[nbuckets]
  int32_t growth;
  uint32_t nbuckets;
  uint64_t grow_foot0, grow_foot;
  uint64_t* d_partials;  // MV: scan partial sums
  uint64_t partials_cap;
  void* d_pool;
  wc_launch launch[WC_OP__N];
  size_t l2_window_bytes;  // > 0: launch with an L2 access-policy window over the slots
  float l2_hit_ratio;
  bool l2_held = false;    // counted in its device's persisting-L2 carve-out (released on destroy)
  // scratch for the blocked scheme, grown on demand (stream-ordered allocation)
  mutable void* d_scratch;
  mutable uint64_t scratch_bytes;
  wc::HostPipe* host = nullptr;  // host-buffer pipeline, created on first use
};

namespace wc {

TableDesc desc_of(const wc_table* t);
PoolDesc pool_of(const wc_table* t);

// Launch with the table's L2 access-policy window when it has one.
cudaLaunchAttribute* l2_attr(const wc_table* t, cudaLaunchAttribute* storage, unsigned* count);

// Single-value families (wc_sv.cu): op is WC_OP_INSERT / RETRIEVE / ERASE.
cudaError_t sv_launch(const wc_table* t, int op, const void* keys, const void* vals, uint64_t n,
                      void* out, uint8_t* found, cudaStream_t s);
bool sv_shape_ok(int slot_bytes, int W, int G);

// Multi-value families (wc_mv.cu).
cudaError_t mv_insert(const wc_table* t, const void* keys, const void* vals, uint64_t n, cudaStream_t s);
cudaError_t mv_count(const wc_table* t, const void* keys, uint64_t n, uint64_t* offsets, cudaStream_t s);
cudaError_t mv_retrieve_multi(const wc_table* t, const void* keys, uint64_t n, const uint64_t* offsets,
                              void* out, cudaStream_t s);
cudaError_t mv_erase(const wc_table* t, const void* keys, uint64_t n, cudaStream_t s);

// Exclusive scan of n uint64 in place, d[n] = total (wc_scan.cu).
cudaError_t scan_exclusive_u64(uint64_t* d, uint64_t n, uint64_t* partials, uint64_t partials_cap,
                               cudaStream_t s);
uint64_t scan_partials_needed(uint64_t n);

int sm_count_of(int device);

// Scratch of at least `bytes` on stream s (grows the table's buffer if needed).
cudaError_t ensure_scratch(const wc_table* t, uint64_t bytes, cudaStream_t s);

// Release the table's host-buffer pipeline (streams, events, staging).
void host_pipe_free(wc_table* t);

// Device bytes of the table's host-buffer staging (0 before the first host-buffer call).
uint64_t host_pipe_bytes(const wc_table* t);

// window_width = 0 at table creation (wc_tune.cu): the sample size the autotuner runs for a
// table of this configuration, and whether tuning is on (environment WC_AUTOTUNE != 0).
uint64_t autotune_sample_for(const wc_table_config& cfg);
bool autotune_enabled();

// Scheme the table uses for `op` on a batch of n keys.
int scheme_for(const wc_table* t, int op, uint64_t n);

}  // namespace wc
