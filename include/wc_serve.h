/*
 * wc_serve.h -- a request-serving loop over device-resident tables.
 *
 * The paper has no counterpart (it benchmarks bulk calls one at a time, Sec. V); this
 * loop serves a stream of insert / retrieve / erase requests as they arrive:
 *   - admission: a request is admitted when the HBM of the served tables (every device
 *     byte they own, counted once per table for the whole run) plus that held by admitted,
 *     unfinished requests (their `io_bytes`) plus its own stays within the budget;
 *     requests are admitted in arrival order (a request that does not fit waits, and so do
 *     the ones behind it);
 *   - continuous batching (WC_SERVE_BATCHED): admitted requests are packed into the next
 *     batched launch (wc_exec.h) while up to `max_inflight` earlier batches are still on
 *     the device, so requests arriving during a launch join the next one; a lone request
 *     (no other admitted or waiting) runs at once as its own bulk call (nothing to pack it
 *     with);
 *   - WC_SERVE_PER_CALL: every admitted request is launched at once as its own bulk call
 *     (the plain per-call API of wc.h) -- the baseline the batched mode is compared with.
 * Results are the same in both modes and equal to running the requests one by one in
 * arrival order: per-table program order is kept (wc_exec.h).
 *
 * The loop runs on the calling thread in real time: request i becomes visible when the
 * clock passes start + arrival_ns[i].  It returns when every request has completed.
 */
#ifndef WC_SERVE_H_
#define WC_SERVE_H_

#include <stdint.h>

#include "wc.h"
#include "wc_exec.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { WC_SERVE_BATCHED = 0, WC_SERVE_PER_CALL = 1 };

typedef struct {
  wc_work work;         /* what to run (table, op, device buffers, n) */
  uint64_t arrival_ns;  /* arrival time, relative to the start of the run */
  uint64_t io_bytes;    /* HBM the request holds while admitted (its buffers) */
} wc_request;

typedef struct {
  uint64_t hbm_budget_bytes;  /* cap on the io_bytes of admitted, unfinished requests */
  uint64_t max_batch_keys;    /* keys per batched launch (a larger request goes alone) */
  uint32_t max_batch_items;   /* requests per batched launch (<= the executor's max) */
  uint32_t max_inflight;      /* batches (or per-call launches) on the device at once */
  int32_t mode;               /* WC_SERVE_BATCHED or WC_SERVE_PER_CALL */
  int32_t reserved;
  uint64_t solo_min_keys;     /* WC_SERVE_BATCHED: a request of at least this many keys runs
                                 as its own bulk call (in order with the batches), since a
                                 large batch gains nothing from packing and the per-call
                                 path applies its own scheme (e.g. the region split);
                                 0 = batch everything */
} wc_serve_config;

typedef struct {
  uint64_t admitted_ns;   /* relative to the start of the run */
  uint64_t launched_ns;
  uint64_t completed_ns;  /* when the host saw the launch holding it finish */
  uint32_t batch;         /* index of the launch that ran it */
  uint32_t reserved;
} wc_request_timing;

typedef struct {
  uint64_t wall_ns;       /* start of the run to the last completion */
  uint64_t launches;      /* batched launches or per-call launches */
  uint64_t keys;          /* keys processed */
  uint64_t peak_admitted_bytes;  /* most HBM held at once: resident_bytes + admitted io_bytes */
  uint64_t resident_bytes;       /* device bytes of the served tables (counted against the budget) */
} wc_serve_stats;

/* Serve `nreq` requests (sorted by arrival_ns).  `ex` is required for WC_SERVE_BATCHED
 * and ignored otherwise.  h_timing receives one record per request; h_stats the totals.
 * All device work goes to `stream`.  A request larger than what the tables leave of the
 * budget is admitted alone when nothing else is in flight; tables that alone exceed the
 * budget return WC_ERR_OUT_OF_MEMORY before anything runs. */
wc_status wc_serve_run(wc_executor* ex, const wc_request* h_requests, uint32_t nreq, const wc_serve_config* cfg,
                       void* stream, wc_request_timing* h_timing, wc_serve_stats* h_stats);

#ifdef __cplusplus
}
#endif

#endif /* WC_SERVE_H_ */
