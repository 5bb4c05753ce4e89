// Batched executor (include/wc_exec.h): one persistent kernel, replayed as a CUDA graph,
// serves a batch of bulk operations on many single-value tables from a device work list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "wc.h"
#include "wc_exec.h"
#include "wc_internal.h"
#include "wc_launch.cuh"
#include "wc_sv_kernels.cuh"

namespace wc {
namespace {

constexpr uint32_t kMaxExecItems = 4096;
constexpr uint32_t kMinTileKeys = 64;
constexpr int kExecThreads = 256;
constexpr int kTicketRing = 256;

struct ExecItem {
  TableDesc t;
  const void* keys;
  const void* vals;
  void* out;
  uint8_t* found;
  uint64_t n;
  uint64_t tile_begin;  // first tile of this item in the batch's tile sequence
  uint32_t op;
  int32_t dep;          // group this item waits for (-1: none)
  uint32_t group;       // group this item counts its finished tiles into
  uint32_t tile_keys;   // keys per tile of this item
};

struct ExecHeader {
  uint64_t total_tiles;
  uint32_t nitems;
  uint32_t ngroups;
  uint64_t ticket;  // this batch's ticket (completion flags hold ticket + 1)
};

// Device layout: [header 256 B | group tile counts max*8 | items max*sizeof(ExecItem)]
//                [next tile 8 | group done counters max*8 | item done counters max*8]
//                [status 4]
struct Layout {
  size_t hdr = 0, gtiles = 256, items = 0, next = 0, gdone = 0, idone = 0, status = 0, total = 0;
  explicit Layout(uint32_t max) {
    items = gtiles + static_cast<size_t>(max) * 8;
    next = (items + static_cast<size_t>(max) * sizeof(ExecItem) + 255) / 256 * 256;
    gdone = next + 8;
    idone = gdone + static_cast<size_t>(max) * 8;
    status = idone + static_cast<size_t>(max) * 8;
    total = (status + 4 + 255) / 256 * 256;
  }
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Lane 0 of a warp: wait until group g has finished all its tiles, at most timeout_ns.
__device__ bool wait_group(const unsigned long long* gtiles, const unsigned long long* gdone, int32_t g,
                           uint64_t timeout_ns) {
  const unsigned long long need = gtiles[g];
  const volatile unsigned long long* d = gdone + g;
  if (*d >= need) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (*d >= need) return true;
    if (global_ns() - t0 > timeout_ns) return false;
    __nanosleep(256);
  }
}

// Lanes per key per operation (packed 64-bit slots): GI for inserts, GR for lookups and
// erases; the kernel is instantiated for every valid pair of each window width.
template <int W, int GI, int GR>
__global__ void __launch_bounds__(kExecThreads, 3) k_exec(const ExecHeader* __restrict__ hdr,
                                                       const unsigned long long* __restrict__ gtiles,
                                                       const ExecItem* __restrict__ items,
                                                       unsigned long long* __restrict__ next_tile,
                                                       unsigned long long* __restrict__ gdone,
                                                       unsigned long long* __restrict__ idone,
                                                       unsigned long long* item_flags, uint32_t* xstatus,
                                                       uint64_t timeout_ns) {
  using L = LayoutP32;
  constexpr int SI = W / GI, SR = W / GR;
  __shared__ uint64_t s_tb[kMaxExecItems];
  const uint32_t nitems = hdr->nitems;
  const uint64_t total = hdr->total_tiles;
  for (uint32_t i = threadIdx.x; i < nitems; i += kExecThreads) s_tb[i] = items[i].tile_begin;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long tile = 0;
    if (lane == 0) tile = atomicAdd(next_tile, 1ull);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= total) break;
    uint32_t lo = 0, hi = nitems - 1;  // last item whose first tile <= tile
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (s_tb[mid] <= tile) lo = mid;
      else hi = mid - 1;
    }
    const ExecItem& it = items[lo];
    const TableDesc t = it.t;
    const uint32_t op = it.op;
    bool ok = true;
    if (it.dep >= 0) {
      if (lane == 0) ok = wait_group(gtiles, gdone, it.dep, timeout_ns);
      ok = __shfl_sync(kFull, ok, 0);
      __threadfence();
    }
    if (ok) {
      const uint64_t begin = (tile - it.tile_begin) * it.tile_keys;
      const uint64_t end = begin + it.tile_keys < it.n ? begin + it.tile_keys : it.n;
      RangeSrc src(begin, end);
      uint32_t flags = 0;
      long long delta = 0;
      if (op == WC_OP_INSERT) {
        sv_insert_range<L, GI, SI>(t, static_cast<const uint32_t*>(it.keys), static_cast<const uint32_t*>(it.vals),
                                   src, flags, delta);
      } else if (op == WC_OP_RETRIEVE) {
        EmitValue<L> emit{static_cast<uint32_t*>(it.out), it.found, nullptr};
        sv_retrieve_range<L, GR, SR>(t, static_cast<const uint32_t*>(it.keys), src, emit, flags);
      } else {
        NoOnErase none;
        long long removed = 0;
        sv_erase_range<L, GR, SR>(t, static_cast<const uint32_t*>(it.keys), src, flags, removed, none);
        delta = -removed;
      }
      flush_flags(t.status, flags);
      flush_delta(t.size, delta);
    } else if (lane == 0) {
      atomicOr(xstatus, kFlagQueueTimeout);
      atomicOr(t.status, kFlagQueueTimeout);
    }
    __syncwarp();
    __threadfence();
    if (lane == 0) {
      atomicAdd(gdone + it.group, 1ull);
      // the warp that finishes an item's last tile reports it to the host (mapped memory)
      const unsigned long long item_tiles = (it.n + it.tile_keys - 1) / it.tile_keys;
      if (atomicAdd(idone + lo, 1ull) + 1 == item_tiles) {
        __threadfence_system();
        const unsigned long long flag = hdr->ticket + 1;
        asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(item_flags + lo), "l"(flag) : "memory");
      }
    }
  }
}

}  // namespace
}  // namespace wc

using namespace wc;

struct wc_executor {
  wc_executor_config cfg;
  int sm_count = 1;
  Layout lay{1};
  char* d_buf = nullptr;
  char* h_stage[2] = {nullptr, nullptr};
  unsigned long long* h_flags[2] = {nullptr, nullptr};  // mapped: per item, ticket + 1 once done
  uint64_t slot_ticket[2] = {~0ull, ~0ull};
  std::vector<int32_t> item_map[2];  // caller's item index -> kernel item index (-1: n == 0)
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  cudaEvent_t ring[kTicketRing] = {};
  uint64_t next_ticket = 0;
  cudaStream_t last_stream = nullptr;
  // one graph per staging slot: [H2D copy of that slot's work list | reset of the tile and
  // group counters | kernel], all with fixed arguments, so a submit never updates a graph
  // that may still be running
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraphNode_t copy_node[2] = {nullptr, nullptr};  // the work-list copy of each graph
  void* kernel = nullptr;
  unsigned grid_blocks = 1;  // blocks of the persistent kernel
};

namespace {

void free_executor(wc_executor* ex) {
  for (int i = 0; i < 2; ++i) {
    if (ex->exec[i]) cudaGraphExecDestroy(ex->exec[i]);
    if (ex->graph[i]) cudaGraphDestroy(ex->graph[i]);
  }
  for (auto& e : ex->ring)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    if (ex->stage_ev[i]) cudaEventDestroy(ex->stage_ev[i]);
    if (ex->h_stage[i]) cudaFreeHost(ex->h_stage[i]);
    if (ex->h_flags[i]) cudaFreeHost(ex->h_flags[i]);
  }
  if (ex->d_buf) cudaFree(ex->d_buf);
  delete ex;
}

// The kernel of (W, GI, GR), or nullptr for a pair outside the instantiated sets.
void* kernel_for(int W, int GI, int GR) {
#define WC_EXEC_K(Wv, I, R) \
  if (W == (Wv) && GI == (I) && GR == (R)) return reinterpret_cast<void*>(k_exec<Wv, I, R>);
  WC_EXEC_K(4, 1, 1) WC_EXEC_K(4, 1, 2) WC_EXEC_K(4, 2, 1) WC_EXEC_K(4, 2, 2)
  WC_EXEC_K(8, 1, 1) WC_EXEC_K(8, 1, 2) WC_EXEC_K(8, 1, 4) WC_EXEC_K(8, 2, 1) WC_EXEC_K(8, 2, 2)
  WC_EXEC_K(8, 2, 4) WC_EXEC_K(8, 4, 1) WC_EXEC_K(8, 4, 2) WC_EXEC_K(8, 4, 4)
  WC_EXEC_K(16, 2, 2) WC_EXEC_K(16, 2, 4) WC_EXEC_K(16, 4, 2) WC_EXEC_K(16, 4, 4)
#undef WC_EXEC_K
  return nullptr;
}

}  // namespace

extern "C" {

wc_status wc_executor_create(wc_executor** out, const wc_executor_config* cfg) {
  if (out == nullptr || cfg == nullptr) return WC_ERR_INVALID_ARG;
  *out = nullptr;
  const int W = cfg->window_width;
  if (W != 4 && W != 8 && W != 16) return WC_ERR_INVALID_ARG;
  if (cfg->max_items == 0 || cfg->max_items > kMaxExecItems) return WC_ERR_INVALID_ARG;
  const uint32_t tk = cfg->tile_keys ? cfg->tile_keys : 4096;
  if (tk < kMinTileKeys || tk > 65536 || (tk & (tk - 1))) return WC_ERR_INVALID_ARG;
  wc_executor* ex = new (std::nothrow) wc_executor();
  if (ex == nullptr) return WC_ERR_OUT_OF_MEMORY;
  ex->cfg = *cfg;
  ex->cfg.tile_keys = tk;
  if (ex->cfg.timeout_ns == 0) ex->cfg.timeout_ns = 2000000000ull;
  DeviceGuard guard(cfg->device);
  ex->sm_count = sm_count_of(cfg->device);
  ex->lay = Layout(cfg->max_items);
  const int gi = cfg->group_insert ? cfg->group_insert : (W == 4 ? 1 : 2);
  const int gr = cfg->group_retrieve ? cfg->group_retrieve : (W == 16 ? 4 : 2);
  ex->kernel = kernel_for(W, gi, gr);
  if (ex->kernel == nullptr) {
    delete ex;
    return WC_ERR_INVALID_ARG;
  }
  bool ok = cudaMalloc(&ex->d_buf, ex->lay.total) == cudaSuccess &&
            cudaMemset(ex->d_buf, 0, ex->lay.total) == cudaSuccess;
  for (int i = 0; ok && i < 2; ++i) {
    ok = cudaHostAlloc(&ex->h_stage[i], ex->lay.next, cudaHostAllocDefault) == cudaSuccess &&
         cudaHostAlloc(reinterpret_cast<void**>(&ex->h_flags[i]), static_cast<size_t>(cfg->max_items) * 8,
                       cudaHostAllocMapped) == cudaSuccess &&
         cudaEventCreateWithFlags(&ex->stage_ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (ok) std::memset(ex->h_flags[i], 0, static_cast<size_t>(cfg->max_items) * 8);
  }
  for (int i = 0; ok && i < kTicketRing; ++i) ok = cudaEventCreateWithFlags(&ex->ring[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_executor(ex);
    return WC_ERR_OUT_OF_MEMORY;
  }
  // graphs: H2D copy of the work list -> reset of the tile/group counters -> kernel
  int bps = occupancy_cached(ex->kernel, kExecThreads, 0);
  const auto* hdr = reinterpret_cast<const ExecHeader*>(ex->d_buf + ex->lay.hdr);
  const auto* gt = reinterpret_cast<const unsigned long long*>(ex->d_buf + ex->lay.gtiles);
  const auto* items = reinterpret_cast<const ExecItem*>(ex->d_buf + ex->lay.items);
  auto* next = reinterpret_cast<unsigned long long*>(ex->d_buf + ex->lay.next);
  auto* gdone = reinterpret_cast<unsigned long long*>(ex->d_buf + ex->lay.gdone);
  auto* idone = reinterpret_cast<unsigned long long*>(ex->d_buf + ex->lay.idone);
  auto* xst = reinterpret_cast<uint32_t*>(ex->d_buf + ex->lay.status);
  uint64_t tmo = ex->cfg.timeout_ns;
  for (int g = 0; ok && g < 2; ++g) {
    unsigned long long* dflags = nullptr;
    ok = cudaHostGetDevicePointer(reinterpret_cast<void**>(&dflags), ex->h_flags[g], 0) == cudaSuccess;
    void* args[] = {&hdr, &gt, &items, &next, &gdone, &idone, &dflags, &xst, &tmo};
    cudaGraphNode_t n_copy = nullptr, n_set = nullptr, n_kernel = nullptr;
    ok = ok && cudaGraphCreate(&ex->graph[g], 0) == cudaSuccess;
    if (ok)
      ok = cudaGraphAddMemcpyNode1D(&n_copy, ex->graph[g], nullptr, 0, ex->d_buf, ex->h_stage[g], ex->lay.next,
                                    cudaMemcpyHostToDevice) == cudaSuccess;
    ex->copy_node[g] = n_copy;
    if (ok) {
      cudaMemsetParams mp = {};
      mp.dst = ex->d_buf + ex->lay.next;
      mp.value = 0;
      mp.elementSize = 1;
      mp.width = ex->lay.status - ex->lay.next;
      mp.height = 1;
      ok = cudaGraphAddMemsetNode(&n_set, ex->graph[g], &n_copy, 1, &mp) == cudaSuccess;
    }
    if (ok) {
      cudaKernelNodeParams kp = {};
      kp.func = ex->kernel;
      ex->grid_blocks = static_cast<unsigned>(bps * ex->sm_count);
      kp.gridDim = dim3(ex->grid_blocks);
      kp.blockDim = dim3(kExecThreads);
      kp.kernelParams = args;
      ok = cudaGraphAddKernelNode(&n_kernel, ex->graph[g], &n_set, 1, &kp) == cudaSuccess &&
           cudaGraphInstantiate(&ex->exec[g], ex->graph[g], 0) == cudaSuccess;
    }
  }
  if (!ok) {
    cudaGetLastError();
    free_executor(ex);
    return WC_ERR_CUDA;
  }
  *out = ex;
  return WC_OK;
}

wc_status wc_executor_destroy(wc_executor* ex) {
  if (ex == nullptr) return WC_ERR_INVALID_ARG;
  DeviceGuard guard(ex->cfg.device);
  cudaDeviceSynchronize();
  free_executor(ex);
  return WC_OK;
}

wc_status wc_executor_submit(wc_executor* ex, const wc_work* h_items, uint32_t count, void* stream,
                             uint64_t* h_ticket) {
  if (ex == nullptr || h_ticket == nullptr || (count > 0 && h_items == nullptr)) return WC_ERR_INVALID_ARG;
  if (count > ex->cfg.max_items) return WC_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < count; ++i) {
    const wc_work& w = h_items[i];
    const wc_table* t = w.table;
    if (t == nullptr || w.op < WC_OP_INSERT || w.op > WC_OP_ERASE) return WC_ERR_INVALID_ARG;
    if (t->cfg.kind != WC_SINGLE_VALUE || t->d_vals != nullptr || t->slot_bytes != 8 || static_cast<int>(t->W) != ex->cfg.window_width ||
        t->device != ex->cfg.device)
      return WC_ERR_UNSUPPORTED;
    if (w.n > 0 && (w.d_keys == nullptr || (w.op == WC_OP_INSERT && w.d_values == nullptr) ||
                    (w.op == WC_OP_RETRIEVE && w.d_values_out == nullptr)))
      return WC_ERR_INVALID_ARG;
    if (w.n >= (1ull << 40)) return WC_ERR_INVALID_ARG;
  }
  DeviceGuard guard(ex->cfg.device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t ticket = ex->next_ticket++;
  const int slot = static_cast<int>(ticket & 1);
  // the staging buffer of this slot was last read by the launch two tickets ago
  if (cudaEventSynchronize(ex->stage_ev[slot]) != cudaSuccess) return WC_ERR_CUDA;
  char* st = ex->h_stage[slot];
  auto* hdr = reinterpret_cast<ExecHeader*>(st + ex->lay.hdr);
  auto* gt = reinterpret_cast<unsigned long long*>(st + ex->lay.gtiles);
  auto* items = reinterpret_cast<ExecItem*>(st + ex->lay.items);
  // groups: consecutive retrieves on a table share one; every write is its own group
  std::unordered_map<const wc_table*, std::pair<int32_t, int32_t>> cur;  // table -> (group, op)
  uint32_t ni = 0, ng = 0;
  uint64_t tiles = 0;
  bool stalled = false;
  // Every item is cut into tiles small enough to spread it over all of the kernel's warps
  // (from kMinTileKeys up to the configured tile size): the warps take tiles in order, so
  // an item's keys are then probed by the whole GPU at once and a small request finishes
  // about as soon as it would as a call of its own.
  const uint64_t warps = static_cast<uint64_t>(ex->grid_blocks) * (kExecThreads / 32);
  const uint64_t tk_max = ex->cfg.tile_keys;
  ex->item_map[slot].assign(count, -1);
  for (uint32_t i = 0; i < count; ++i) {
    const wc_work& w = h_items[i];
    if (w.n == 0) continue;
    ex->item_map[slot][i] = static_cast<int32_t>(ni);
    ExecItem& it = items[ni++];
    it.t = desc_of(w.table);
    it.keys = w.d_keys;
    it.vals = w.d_values;
    it.out = w.d_values_out;
    it.found = w.d_found_out;
    it.n = w.n;
    it.tile_begin = tiles;
    it.op = static_cast<uint32_t>(w.op);
    uint64_t tk = (w.n + warps - 1) / warps;
    tk = std::min<uint64_t>(tk_max, std::max<uint64_t>(kMinTileKeys, (tk + kMinTileKeys - 1) / kMinTileKeys * kMinTileKeys));
    it.tile_keys = static_cast<uint32_t>(tk);
    const uint64_t nt = (w.n + tk - 1) / tk;
    tiles += nt;
    auto f = cur.find(w.table);
    if (f != cur.end() && w.op == WC_OP_RETRIEVE && f->second.second == WC_OP_RETRIEVE) {
      it.group = static_cast<uint32_t>(f->second.first);
      // joins the open retrieve group: waits for what that group waits for
      it.dep = -1;
      for (uint32_t k = ni - 1; k-- > 0;)
        if (items[k].group == it.group) {
          it.dep = items[k].dep;
          break;
        }
    } else {
      it.dep = f != cur.end() ? f->second.first : -1;
      it.group = ng;
      gt[ng++] = 0;
      cur[w.table] = {static_cast<int32_t>(it.group), w.op};
    }
    gt[it.group] += nt;
    if (ex->cfg.test_stall && !stalled && w.op != WC_OP_RETRIEVE) {
      gt[it.group] += 1;  // never reached: dependents of this group time out
      stalled = true;
    }
  }
  *h_ticket = ticket;
  ex->last_stream = s;
  ex->slot_ticket[slot] = ticket;
  if (ni == 0) return cudaEventRecord(ex->ring[ticket % kTicketRing], s) == cudaSuccess ? WC_OK : WC_ERR_CUDA;
  hdr->total_tiles = tiles;
  hdr->nitems = ni;
  hdr->ngroups = ng;
  hdr->ticket = ticket;
  // copy only the part of the work list this batch uses (header, group counts, its items):
  // a small batch then costs a few KB of copy instead of the whole list's capacity
  const size_t used = ex->lay.items + static_cast<size_t>(ni) * sizeof(ExecItem);
  cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(ex->exec[slot], ex->copy_node[slot], ex->d_buf,
                                                     ex->h_stage[slot], used, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex->exec[slot], s);
  if (e == cudaSuccess) e = cudaEventRecord(ex->stage_ev[slot], s);
  if (e == cudaSuccess) e = cudaEventRecord(ex->ring[ticket % kTicketRing], s);
  return e == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}

wc_status wc_executor_query(wc_executor* ex, uint64_t ticket, int32_t* h_done) {
  if (ex == nullptr || h_done == nullptr || ticket >= ex->next_ticket) return WC_ERR_INVALID_ARG;
  if (ticket + kTicketRing < ex->next_ticket) {
    *h_done = 1;  // older than the ring: finished before a later launch on the same stream
    return WC_OK;
  }
  DeviceGuard guard(ex->cfg.device);
  const cudaError_t e = cudaEventQuery(ex->ring[ticket % kTicketRing]);
  if (e == cudaSuccess) {
    *h_done = 1;
    return WC_OK;
  }
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    *h_done = 0;
    return WC_OK;
  }
  return WC_ERR_CUDA;
}

wc_status wc_executor_query_item(wc_executor* ex, uint64_t ticket, uint32_t index, int32_t* h_done) {
  if (ex == nullptr || h_done == nullptr || ticket >= ex->next_ticket) return WC_ERR_INVALID_ARG;
  const int slot = static_cast<int>(ticket & 1);
  if (ex->slot_ticket[slot] != ticket) {
    *h_done = 1;  // the slot was reused, which waits for this batch to finish
    return WC_OK;
  }
  if (index >= ex->item_map[slot].size()) return WC_ERR_INVALID_ARG;
  const int32_t k = ex->item_map[slot][index];
  if (k < 0) {
    *h_done = 1;
    return WC_OK;
  }
  const volatile unsigned long long* f = ex->h_flags[slot];
  *h_done = f[k] == ticket + 1 ? 1 : 0;
  return WC_OK;
}

wc_status wc_executor_wait(wc_executor* ex, uint64_t ticket) {
  if (ex == nullptr || ticket >= ex->next_ticket) return WC_ERR_INVALID_ARG;
  if (ticket + kTicketRing < ex->next_ticket) return WC_OK;
  DeviceGuard guard(ex->cfg.device);
  return cudaEventSynchronize(ex->ring[ticket % kTicketRing]) == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}

wc_status wc_executor_get_status(wc_executor* ex, uint32_t* h_flags, int32_t clear) {
  if (ex == nullptr || h_flags == nullptr) return WC_ERR_INVALID_ARG;
  DeviceGuard guard(ex->cfg.device);
  cudaStream_t s = ex->last_stream;
  uint32_t* d = reinterpret_cast<uint32_t*>(ex->d_buf + ex->lay.status);
  cudaError_t e = cudaMemcpyAsync(h_flags, d, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && clear) e = cudaMemsetAsync(d, 0, 4, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? WC_OK : WC_ERR_CUDA;
}

}  // extern "C"
