// Request-serving loop (include/wc_serve.h): admission by HBM budget, continuous batching
// into the batched executor, or per-call launches as the baseline.  Host code only.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <deque>
#include <thread>
#include <unordered_set>
#include <vector>

#include "wc.h"
#include "wc_exec.h"
#include "wc_internal.h"
#include "wc_serve.h"

namespace {

struct Launch {
  uint64_t ticket = 0;       // batched launch
  cudaEvent_t ev = nullptr;  // per-call launch
  std::vector<uint32_t> reqs;
  size_t left = 0;           // requests not finished yet
};

wc_status launch_one(const wc_work& w, void* stream) {
  switch (w.op) {
    case WC_OP_INSERT: return wc_insert(w.table, w.d_keys, w.d_values, w.n, stream);
    case WC_OP_RETRIEVE: return wc_retrieve(w.table, w.d_keys, w.n, w.d_values_out, w.d_found_out, stream);
    case WC_OP_ERASE: return wc_erase(w.table, w.d_keys, w.n, stream);
    default: return WC_ERR_INVALID_ARG;
  }
}

}  // namespace

extern "C" wc_status wc_serve_run(wc_executor* ex, const wc_request* reqs, uint32_t nreq, const wc_serve_config* cfg,
                                  void* stream, wc_request_timing* timing, wc_serve_stats* stats) {
  if (cfg == nullptr || timing == nullptr || stats == nullptr || (nreq > 0 && reqs == nullptr))
    return WC_ERR_INVALID_ARG;
  const bool batched = cfg->mode == WC_SERVE_BATCHED;
  if (!batched && cfg->mode != WC_SERVE_PER_CALL) return WC_ERR_INVALID_ARG;
  if (batched && ex == nullptr) return WC_ERR_INVALID_ARG;
  if (cfg->max_inflight == 0 || cfg->max_batch_items == 0) return WC_ERR_INVALID_ARG;
  for (uint32_t i = 1; i < nreq; ++i)
    if (reqs[i].arrival_ns < reqs[i - 1].arrival_ns) return WC_ERR_INVALID_ARG;
  // HBM the served tables hold for the whole run (slots, metadata, scratch they own): the
  // budget covers them first, and the admitted requests' buffers share what is left
  uint64_t resident = 0;
  {
    std::unordered_set<const wc_table*> seen;
    for (uint32_t i = 0; i < nreq; ++i) {
      const wc_table* t = reqs[i].work.table;
      if (t == nullptr) return WC_ERR_INVALID_ARG;
      if (seen.insert(t).second) resident += t->device_bytes + t->scratch_bytes + wc::host_pipe_bytes(t);
    }
  }
  if (resident > cfg->hbm_budget_bytes) return WC_ERR_OUT_OF_MEMORY;

  std::vector<cudaEvent_t> pool;
  {
    pool.resize(cfg->max_inflight);
    for (auto& e : pool)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        for (auto& f : pool)
          if (f) cudaEventDestroy(f);
        return WC_ERR_CUDA;
      }
  }
  const auto t0 = std::chrono::steady_clock::now();
  auto now_ns = [&]() {
    return static_cast<uint64_t>(
        std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count());
  };
  uint32_t next_arrival = 0, completed = 0;
  std::deque<uint32_t> waiting;  // arrived, not admitted
  std::deque<uint32_t> ready;    // admitted, not launched
  std::deque<Launch> inflight;   // launched, not seen finished (one stream: finish in order)
  uint64_t admitted_bytes = 0, peak = 0, launches = 0, keys = 0;
  uint32_t pool_next = 0;
  std::vector<wc_work> batch;
  batch.reserve(cfg->max_batch_items);
  std::vector<uint8_t> finished(nreq, 0);
  bool progress = false;
  auto finish = [&](uint32_t r, uint64_t t) {
    if (finished[r]) return;
    finished[r] = 1;
    timing[r].completed_ns = t;
    admitted_bytes -= reqs[r].io_bytes;
    ++completed;
    progress = true;
  };
  wc_status st = WC_OK;

  while (completed < nreq && st == WC_OK) {
    progress = false;
    uint64_t now = now_ns();
    while (next_arrival < nreq && reqs[next_arrival].arrival_ns <= now) waiting.push_back(next_arrival++);
    // admission in arrival order within the HBM budget
    while (!waiting.empty()) {
      const uint32_t r = waiting.front();
      const uint64_t b = reqs[r].io_bytes;
      if (resident + admitted_bytes + b > cfg->hbm_budget_bytes && admitted_bytes != 0) break;
      admitted_bytes += b;
      peak = std::max(peak, resident + admitted_bytes);
      timing[r].admitted_ns = now;
      ready.push_back(r);
      waiting.pop_front();
      progress = true;
    }
    // completions: a per-call launch finishes as a whole; a batched request finishes when
    // its own item does (reported by the executor through mapped memory)
    for (auto it = inflight.begin(); it != inflight.end() && st == WC_OK;) {
      Launch& f = *it;
      const uint64_t t = now_ns();
      if (f.ev != nullptr) {
        const cudaError_t e = cudaEventQuery(f.ev);
        if (e == cudaErrorNotReady) {
          cudaGetLastError();
          ++it;
          continue;
        }
        if (e != cudaSuccess) {
          st = WC_ERR_CUDA;
          break;
        }
        for (uint32_t r : f.reqs) finish(r, t);
        f.left = 0;
      } else {
        for (uint32_t j = 0; j < f.reqs.size(); ++j) {
          const uint32_t r = f.reqs[j];
          if (finished[r]) continue;
          int32_t done = 0;
          st = wc_executor_query_item(ex, f.ticket, j, &done);
          if (st != WC_OK) break;
          if (done) {
            finish(r, t);
            --f.left;
          }
        }
      }
      if (f.left == 0) {
        it = inflight.erase(it);
        progress = true;
      } else {
        ++it;
      }
    }
    // launches: while a slot is free, pack the admitted requests (continuous batching)
    while (st == WC_OK && !ready.empty() && inflight.size() < cfg->max_inflight) {
      Launch l;
      const uint64_t t = now_ns();
      // A lone request (nothing else admitted or waiting) runs at once as its own bulk
      // call: there is nothing to pack it with, and the plain launch has the shortest path
      // to the device.  Batches form from the requests that queue up while earlier work
      // is on the device.
      const bool lone = ready.size() == 1 && waiting.empty();
      const bool solo = !batched || lone ||
                        (cfg->solo_min_keys && reqs[ready.front()].work.n >= cfg->solo_min_keys);
      if (!solo) {
        batch.clear();
        uint64_t nk = 0;
        while (!ready.empty() && batch.size() < cfg->max_batch_items) {
          const uint32_t r = ready.front();
          if (!batch.empty() && nk + reqs[r].work.n > cfg->max_batch_keys) break;
          if (cfg->solo_min_keys && reqs[r].work.n >= cfg->solo_min_keys) break;  // keeps arrival order
          batch.push_back(reqs[r].work);
          nk += reqs[r].work.n;
          l.reqs.push_back(r);
          ready.pop_front();
        }
        st = wc_executor_submit(ex, batch.data(), static_cast<uint32_t>(batch.size()), stream, &l.ticket);
        keys += nk;
      } else {
        const uint32_t r = ready.front();
        ready.pop_front();
        l.reqs.push_back(r);
        st = launch_one(reqs[r].work, stream);
        l.ev = pool[pool_next++ % pool.size()];
        if (st == WC_OK && cudaEventRecord(l.ev, static_cast<cudaStream_t>(stream)) != cudaSuccess) st = WC_ERR_CUDA;
        keys += reqs[r].work.n;
      }
      for (uint32_t r : l.reqs) {
        timing[r].launched_ns = t;
        timing[r].batch = static_cast<uint32_t>(launches);
      }
      ++launches;
      l.left = l.reqs.size();
      inflight.push_back(std::move(l));
      progress = true;
    }
    if (!progress) std::this_thread::yield();
  }
  if (st == WC_OK && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) st = WC_ERR_CUDA;
  stats->wall_ns = now_ns();
  uint64_t last = 0;
  for (uint32_t i = 0; i < nreq; ++i) last = std::max(last, timing[i].completed_ns);
  if (nreq) stats->wall_ns = last;
  stats->launches = launches;
  stats->keys = keys;
  stats->peak_admitted_bytes = peak;
  stats->resident_bytes = resident;
  for (auto& e : pool) cudaEventDestroy(e);
  return st;
}
