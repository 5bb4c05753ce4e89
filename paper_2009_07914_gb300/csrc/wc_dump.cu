// Host copies of a table: the slot array alone (for inspection and the slot-dump
// invariant checks), and whole-table snapshots that a table of the same geometry can be
// restored from (checkpoint and resume).  Plus the status check that folds the device
// status word into a wc_status.  Host code only.
#include <cuda_runtime.h>

#include <cstring>

#include "wc.h"
#include "wc_internal.h"

namespace {

constexpr uint64_t kMagic = 0x31544e5350414e53ull;  // "SNAPSNT1"

// Snapshot header: the geometry a restore must match, then the table's device block.
struct SnapHeader {
  uint64_t magic;
  int32_t kind, key_bytes, value_bytes, window_width;
  uint64_t windows, pool_capacity, seed, device_bytes, clear_bytes;
  uint64_t bucket_first_size, bucket_growth_bits;
};
static_assert(sizeof(SnapHeader) == 80, "snapshot header layout");

SnapHeader header_of(const wc_table* t) {
  SnapHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kMagic;
  h.kind = t->cfg.kind;
  h.key_bytes = t->cfg.key_bytes;
  h.value_bytes = t->cfg.value_bytes;
  h.window_width = static_cast<int32_t>(t->W);
  h.windows = t->windows;
  h.pool_capacity = t->pool_capacity;
  h.seed = t->cfg.seed;
  h.device_bytes = t->device_bytes;
  h.clear_bytes = t->clear_bytes;
  h.bucket_first_size = t->cfg.bucket_first_size;
  std::memcpy(&h.bucket_growth_bits, &t->cfg.bucket_growth, sizeof(double));
  if (t->cfg.bucket_first_size == 0) h.bucket_growth_bits = 0;  // lambda unused
  return h;
}

// Bytes of the device block a snapshot carries: everything but the scan partials
// (scratch between calls), i.e. [slots | meta | pending] and the value pool.
uint64_t pool_offset(const wc_table* t) {
  return t->d_pool ? static_cast<uint64_t>(static_cast<char*>(t->d_pool) - static_cast<char*>(t->d_block)) : 0;
}

}  // namespace

extern "C" {

wc_status wc_table_dump_slots(const wc_table* t, void* h_out, uint64_t bytes, void* stream) {
  if (t == nullptr || h_out == nullptr || bytes < t->table_bytes) return WC_ERR_INVALID_ARG;
  wc::DeviceGuard g(t->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(h_out, t->d_slots, t->table_bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return wc::cuda_status(e);
}

wc_status wc_table_dump_overflow_bits(const wc_table* t, uint32_t* h_out, uint64_t words, void* stream) {
  if (t == nullptr || h_out == nullptr) return WC_ERR_INVALID_ARG;
  if (t->d_ovf == nullptr) return WC_ERR_UNSUPPORTED;
  const uint64_t need = (t->windows + 3) / 4;
  if (words < need) return WC_ERR_INVALID_ARG;
  wc::DeviceGuard g(t->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(h_out, t->d_ovf, need * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return wc::cuda_status(e);
}

uint64_t wc_table_snapshot_bytes(const wc_table* t) {
  if (t == nullptr) return 0;
  const uint64_t pool_bytes = t->d_pool ? t->device_bytes - pool_offset(t) : 0;
  return sizeof(SnapHeader) + t->clear_bytes + pool_bytes;
}

wc_status wc_table_snapshot(const wc_table* t, void* h_out, uint64_t bytes, void* stream) {
  if (t == nullptr || h_out == nullptr || bytes < wc_table_snapshot_bytes(t)) return WC_ERR_INVALID_ARG;
  wc::DeviceGuard g(t->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const SnapHeader h = header_of(t);
  std::memcpy(h_out, &h, sizeof(h));
  char* dst = static_cast<char*>(h_out) + sizeof(h);
  cudaError_t e = cudaMemcpyAsync(dst, t->d_block, t->clear_bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && t->d_pool)
    e = cudaMemcpyAsync(dst + t->clear_bytes, t->d_pool, t->device_bytes - pool_offset(t), cudaMemcpyDeviceToHost,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return wc::cuda_status(e);
}

wc_status wc_table_restore(wc_table* t, const void* h_in, uint64_t bytes, void* stream) {
  if (t == nullptr || h_in == nullptr || bytes < sizeof(SnapHeader)) return WC_ERR_INVALID_ARG;
  SnapHeader h;
  std::memcpy(&h, h_in, sizeof(h));
  const SnapHeader want = header_of(t);
  if (h.magic != kMagic || h.kind != want.kind || h.key_bytes != want.key_bytes ||
      h.value_bytes != want.value_bytes || h.window_width != want.window_width || h.windows != want.windows ||
      h.pool_capacity != want.pool_capacity || h.seed != want.seed || h.device_bytes != want.device_bytes ||
      h.clear_bytes != want.clear_bytes || h.bucket_first_size != want.bucket_first_size ||
      h.bucket_growth_bits != want.bucket_growth_bits || bytes < wc_table_snapshot_bytes(t))
    return WC_ERR_INVALID_ARG;
  wc::DeviceGuard g(t->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const char* src = static_cast<const char*>(h_in) + sizeof(h);
  cudaError_t e = cudaMemcpyAsync(t->d_block, src, t->clear_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && t->d_pool)
    e = cudaMemcpyAsync(t->d_pool, src + t->clear_bytes, t->device_bytes - pool_offset(t), cudaMemcpyHostToDevice,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return wc::cuda_status(e);
}

wc_status wc_table_device_view(const wc_table* t, wc_device_view* h_out) {
  if (t == nullptr || h_out == nullptr) return WC_ERR_INVALID_ARG;
  const bool bl = t->cfg.kind == WC_MULTI_VALUE;
  if ((t->cfg.kind != WC_SINGLE_VALUE && t->cfg.kind != WC_MULTI_VALUE_OA && t->cfg.kind != WC_HASH_SET &&
       t->cfg.kind != WC_COUNTING && !bl) ||
      t->d_vals != nullptr)
    return WC_ERR_UNSUPPORTED;
  // per-element appends need buckets of known sizes (a growth strategy) and pool offsets
  // below bit 63 of the list handle, which marks a list whose next bucket is being made
  if (bl && (t->growth == wc::kGrowExact || t->pool_capacity >= (1ull << 34))) return WC_ERR_UNSUPPORTED;
  *h_out = wc_device_view{};
  h_out->slots = t->d_slots;
  h_out->status = t->d_status;
  h_out->size = t->d_size;
  h_out->overflow_bits = t->d_ovf;
  h_out->seed = t->cfg.seed;
  h_out->capacity = t->capacity;
  h_out->windows = static_cast<uint32_t>(t->windows);
  h_out->window_width = static_cast<uint32_t>(t->W);
  h_out->kind = t->cfg.kind;
  h_out->key_bytes = t->cfg.key_bytes;
  h_out->value_bytes = t->cfg.value_bytes;
  h_out->slot_bytes = static_cast<int32_t>(t->slot_bytes);
  if (bl) {
    h_out->pool = t->d_pool;
    h_out->pool_cursor = t->d_cursor;
    h_out->num_keys = t->d_nkeys;
    h_out->pool_capacity = t->pool_capacity;
    h_out->growth = t->growth;
    h_out->bucket_size = t->cfg.bucket_first_size;
    h_out->bucket_foot0 = t->grow_foot0;
    h_out->bucket_foot = t->grow_foot;
    h_out->bucket_count = t->nbuckets;
    h_out->bucket_cum_size = t->d_growth;
    h_out->bucket_cum_foot = t->d_growth ? t->d_growth + t->nbuckets : nullptr;
  }
  return WC_OK;
}

wc_status wc_check_status(wc_table* t, uint32_t* h_flags_or_null, void* stream) {
  uint32_t f = 0;
  wc_status st = wc_get_status(t, &f, 1, stream);
  if (st != WC_OK) return st;
  if (h_flags_or_null != nullptr) *h_flags_or_null = f;
  if (f & WC_FLAG_QUEUE_TIMEOUT) return WC_ERR_TIMEOUT;
  if (f & (WC_FLAG_PROBE_LIMIT | WC_FLAG_POOL_EXHAUSTED | WC_FLAG_COUNT_OVERFLOW)) return WC_ERR_FULL;
  return WC_OK;
}

}  // extern "C"
