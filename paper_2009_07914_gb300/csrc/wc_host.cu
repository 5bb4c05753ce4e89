// Bulk calls on host buffers (include/wc.h: wc_insert_host, wc_retrieve_host): the batch
// moves through a ring of device staging buffers in chunks, copies on the table's own copy
// streams overlapping the kernels of the neighbouring chunks on the caller's stream.
// Host code only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>

#include "wc.h"
#include "wc_internal.h"

namespace wc {

constexpr int kStages = 3;  // staging buffers: copies may run two chunks ahead of the kernels

// Per-table state of the host pipeline, created on first use.
struct HostPipe {
  int device = -1;
  cudaStream_t in = nullptr, out = nullptr;  // copy streams (host -> device, device -> host)
  cudaEvent_t ready[kStages] = {}, done[kStages] = {}, freed[kStages] = {}, tail = nullptr;
  void* stage = nullptr;                     // kStages staging buffers of `each` bytes
  uint64_t each = 0;
};

uint64_t host_pipe_bytes(const wc_table* t) {
  return t->host != nullptr && t->host->stage != nullptr ? kStages * t->host->each : 0;
}

void host_pipe_free(wc_table* t) {
  HostPipe* h = t->host;
  if (h == nullptr) return;
  if (h->in) cudaStreamSynchronize(h->in);
  if (h->out) cudaStreamSynchronize(h->out);
  for (int b = 0; b < kStages; ++b) {
    if (h->ready[b]) cudaEventDestroy(h->ready[b]);
    if (h->done[b]) cudaEventDestroy(h->done[b]);
    if (h->freed[b]) cudaEventDestroy(h->freed[b]);
  }
  if (h->tail) cudaEventDestroy(h->tail);
  if (h->in) cudaStreamDestroy(h->in);
  if (h->out) cudaStreamDestroy(h->out);
  if (h->stage) cudaFree(h->stage);
  delete h;
  t->host = nullptr;
}

namespace {

// Chunk sizes.  A large insert is split by table region and swept region by region, which
// pays off with large batches (2^27 pairs at load 0.9 into 1.2 GB: 4.8 ms in one call, 5.4
// in chunks of 2^25, 7.4 in chunks of 2^23), so inserts move in large chunks after a small
// first one that starts the kernels early.  Lookups are as fast in chunks of 2^23 as in one
// call, and small chunks keep the pipeline's fill and drain short.
constexpr uint64_t kInsertFirst = 1ull << 23;
constexpr uint64_t kInsertChunk = 1ull << 25;
constexpr uint64_t kRetrieveChunk = 1ull << 23;

// Size of insert chunk c when `left` pairs remain (chunk = the large size for this batch).
uint64_t insert_chunk(uint64_t c, uint64_t left, uint64_t chunk) {
  return std::min(left, c == 0 ? std::min(kInsertFirst, chunk) : chunk);
}

cudaError_t pipe_of(wc_table* t, uint64_t each, HostPipe** out) {
  HostPipe* h = t->host;
  if (h == nullptr) {
    h = new (std::nothrow) HostPipe();
    if (h == nullptr) return cudaErrorMemoryAllocation;
    t->host = h;
    h->device = t->device;
    cudaError_t e = cudaStreamCreateWithFlags(&h->in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->out, cudaStreamNonBlocking);
    for (int b = 0; b < kStages && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&h->ready[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->done[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->freed[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->tail, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      host_pipe_free(t);
      return e;
    }
  }
  if (h->each < each) {
    if (h->stage) {
      cudaStreamSynchronize(h->in);
      cudaStreamSynchronize(h->out);
      cudaDeviceSynchronize();  // kernels of earlier calls may still read the staging
      cudaFree(h->stage);
      h->stage = nullptr;
      h->each = 0;
    }
    cudaError_t e = cudaMalloc(&h->stage, kStages * each);
    if (e != cudaSuccess) {
      h->stage = nullptr;
      return e;
    }
    h->each = each;
  }
  *out = h;
  return cudaSuccess;
}

uint64_t align256(uint64_t x) { return (x + 255) / 256 * 256; }

bool is_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

}  // namespace
}  // namespace wc

using namespace wc;

extern "C" {

wc_status wc_insert_host(wc_table* t, const void* h_keys, const void* h_values, uint64_t n, void* stream) {
  TraceRange trace("wc_insert_host");
  if (t == nullptr) return WC_ERR_INVALID_ARG;
  if (n == 0) return WC_OK;
  const bool no_values = t->cfg.kind == WC_HASH_SET || t->cfg.kind == WC_BLOOM_FILTER ||
                         (t->cfg.kind == WC_COUNTING && h_values == nullptr);
  if (h_keys == nullptr || !is_host(h_keys) || (!no_values && (h_values == nullptr || !is_host(h_values))))
    return WC_ERR_INVALID_ARG;
  if (t->cfg.kind == WC_MULTI_VALUE && n >= (1ull << 31)) return WC_ERR_INVALID_ARG;
  DeviceGuard g(t->device);
  const uint64_t kb = static_cast<uint64_t>(t->cfg.key_bytes), vb = no_values ? 0 : t->cfg.value_bytes;
  const uint64_t chunk = std::min<uint64_t>(n, kInsertChunk);
  const uint64_t koff = 0, voff = align256(chunk * kb);
  HostPipe* h = nullptr;
  cudaError_t e = pipe_of(t, voff + align256(chunk * vb), &h);
  if (e != cudaSuccess) return cuda_status(e);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t base = 0;
  for (uint64_t c = 0; base < n; ++c) {
    const int b = static_cast<int>(c % kStages);
    const uint64_t cnt = insert_chunk(c, n - base, chunk);
    char* buf = static_cast<char*>(h->stage) + b * h->each;
    // the buffer is free once the insert that last read it has run
    if ((e = cudaStreamWaitEvent(h->in, h->freed[b], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(buf + koff, static_cast<const char*>(h_keys) + base * kb, cnt * kb,
                             cudaMemcpyHostToDevice, h->in)) != cudaSuccess)
      break;
    if (!no_values && (e = cudaMemcpyAsync(buf + voff, static_cast<const char*>(h_values) + base * vb, cnt * vb,
                                           cudaMemcpyHostToDevice, h->in)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(h->ready[b], h->in)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(s, h->ready[b], 0)) != cudaSuccess) break;
    const wc_status st = wc_insert(t, buf + koff, no_values ? nullptr : buf + voff, cnt, stream);
    if (st != WC_OK) return st;
    if ((e = cudaEventRecord(h->freed[b], s)) != cudaSuccess) break;
    base += cnt;
  }
  return cuda_status(e);
}

wc_status wc_retrieve_host(wc_table* t, const void* h_keys, uint64_t n, void* h_values_out, uint8_t* h_found_or_null,
                           void* stream) {
  TraceRange trace("wc_retrieve_host");
  if (t == nullptr) return WC_ERR_INVALID_ARG;
  if (t->cfg.kind != WC_SINGLE_VALUE && t->cfg.kind != WC_COUNTING) return WC_ERR_UNSUPPORTED;
  if (n == 0) return WC_OK;
  if (h_keys == nullptr || h_values_out == nullptr || !is_host(h_keys) || !is_host(h_values_out) ||
      (h_found_or_null != nullptr && !is_host(h_found_or_null)))
    return WC_ERR_INVALID_ARG;
  DeviceGuard g(t->device);
  const uint64_t kb = static_cast<uint64_t>(t->cfg.key_bytes), vb = static_cast<uint64_t>(t->cfg.value_bytes);
  const uint64_t chunk = std::min<uint64_t>(n, kRetrieveChunk);
  const uint64_t ooff = align256(chunk * kb), foff = ooff + align256(chunk * vb);
  HostPipe* h = nullptr;
  cudaError_t e = pipe_of(t, foff + align256(chunk), &h);
  if (e != cudaSuccess) return cuda_status(e);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t nchunks = (n + chunk - 1) / chunk;
  for (uint64_t c = 0; c < nchunks; ++c) {
    const int b = static_cast<int>(c % kStages);
    const uint64_t base = c * chunk, cnt = std::min(chunk, n - base);
    char* buf = static_cast<char*>(h->stage) + b * h->each;
    // the buffer is free once its previous results have been copied out
    if ((e = cudaStreamWaitEvent(h->in, h->freed[b], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(buf, static_cast<const char*>(h_keys) + base * kb, cnt * kb, cudaMemcpyHostToDevice,
                             h->in)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(h->ready[b], h->in)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(s, h->ready[b], 0)) != cudaSuccess) break;
    const wc_status st = wc_retrieve(t, buf, cnt, buf + ooff,
                                     h_found_or_null ? reinterpret_cast<uint8_t*>(buf + foff) : nullptr, stream);
    if (st != WC_OK) return st;
    if ((e = cudaEventRecord(h->done[b], s)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(h->out, h->done[b], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(static_cast<char*>(h_values_out) + base * vb, buf + ooff, cnt * vb,
                             cudaMemcpyDeviceToHost, h->out)) != cudaSuccess)
      break;
    if (h_found_or_null &&
        (e = cudaMemcpyAsync(h_found_or_null + base, buf + foff, cnt, cudaMemcpyDeviceToHost, h->out)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(h->freed[b], h->out)) != cudaSuccess) break;
  }
  // the caller's stream completes after the last copy out
  if (e == cudaSuccess) e = cudaEventRecord(h->tail, h->out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->tail, 0);
  return cuda_status(e);
}

}  // extern "C"
