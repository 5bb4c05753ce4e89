/*
 * wc_exec.h -- batched execution of many bulk operations on many tables in ONE launch.
 *
 * The paper runs each bulk operation as its own kernel on a stream and leaves overlap to
 * CUDA streams (Sec. IV-D).  This executor instead packs a batch of work items -- bulk
 * insert / retrieve / erase calls on single-value tables of any capacity -- into one
 * persistent kernel: every warp pulls fixed-size tiles of keys from a device work queue,
 * so tables of uneven size and batches from a thousand to millions of keys share the
 * SMs without per-call launch overhead or tail effects.  The launch is a CUDA graph
 * (H2D copy of the work list, counter reset, kernel) replayed per batch.
 *
 * Ordering: items are applied as if in submission order per table.  Retrieves that
 * follow each other on one table run concurrently; every insert or erase waits for all
 * earlier items on its table and is waited for by all later ones (the overlap rules of
 * Sec. IV-D, made strict so results equal a sequential run).  Items on different tables
 * are independent.  Waits inside the kernel are bounded by a deadline on the device's
 * global timer; a wait that runs out skips its tile and raises WC_FLAG_QUEUE_TIMEOUT in
 * the executor's and the table's status word (the batch's results are then invalid).
 *
 * Conventions as in wc.h.  Supported tables: single-value, 4-byte keys and values,
 * window width equal to the executor's.
 */
#ifndef WC_EXEC_H_
#define WC_EXEC_H_

#include <stdint.h>

#include "wc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wc_executor wc_executor;

typedef struct {
  int32_t op;             /* WC_OP_INSERT, WC_OP_RETRIEVE or WC_OP_ERASE */
  int32_t reserved;
  wc_table* table;
  const void* d_keys;     /* n keys (device) */
  const void* d_values;   /* insert: n values (device) */
  void* d_values_out;     /* retrieve: n values out (device) */
  uint8_t* d_found_out;   /* retrieve: optional n-byte found mask (device) */
  uint64_t n;
} wc_work;

typedef struct {
  int32_t device;
  int32_t window_width;   /* window width of every table the executor serves (4, 8, 16) */
  uint32_t max_items;     /* work items per batch */
  uint32_t tile_keys;     /* most keys per tile (power of two, 64..65536; 0 = 4096): each
                             item is cut into tiles of a multiple of 64 keys, small enough to
                             spread it over every warp of the kernel, up to this size */
  uint64_t timeout_ns;    /* bound of every device-side wait (0 = 2 s) */
  int32_t test_stall;     /* testing: 1 = the first write item of every batch is never
                             reported complete, so items depending on it time out */
  int32_t reserved;
  int32_t group_insert;   /* lanes per key of inserts (0 = 2 for W 8 and 16, 1 for W 4);
                             W 4: 1 or 2, W 8: 1, 2 or 4, W 16: 2 or 4 -- e.g. the autotuner's
                             direct-insert choice for the tables' key width and load */
  int32_t group_retrieve; /* lanes per key of lookups and erases (0 = 2, 4 for W 16); same sets */
} wc_executor_config;

/* Create an executor: device work-list buffers, two pinned host staging buffers, the
 * captured graph.  Synchronous. */
wc_status wc_executor_create(wc_executor** out, const wc_executor_config* cfg);
wc_status wc_executor_destroy(wc_executor* ex);

/* Launch one batch of `count` items on `stream` (asynchronous).  All submits of one
 * executor must go to the same stream.  The host arrays are copied before the call
 * returns.  *h_ticket receives the batch's ticket for wc_executor_query/wait.
 * WC_ERR_UNSUPPORTED for an item whose table the executor cannot serve. */
wc_status wc_executor_submit(wc_executor* ex, const wc_work* h_items, uint32_t count, void* stream,
                             uint64_t* h_ticket);

/* Non-blocking: *h_done = 1 once the batch `ticket` has finished on the device. */
wc_status wc_executor_query(wc_executor* ex, uint64_t ticket, int32_t* h_done);

/* Non-blocking, no CUDA call: *h_done = 1 once item `index` (its position in the
 * wc_executor_submit array) of batch `ticket` has finished -- each item reports on its
 * own through mapped host memory when its last tile is done, so small items of a large
 * batch complete early.  Device-side results of a finished item are visible to work
 * ordered after it on the executor's stream. */
wc_status wc_executor_query_item(wc_executor* ex, uint64_t ticket, uint32_t index, int32_t* h_done);

/* Block until batch `ticket` has finished. */
wc_status wc_executor_wait(wc_executor* ex, uint64_t ticket);

/* Executor status word (WC_FLAG_QUEUE_TIMEOUT); with clear != 0 reset afterwards.
 * Synchronises the executor's last stream. */
wc_status wc_executor_get_status(wc_executor* ex, uint32_t* h_flags, int32_t clear);

#ifdef __cplusplus
}
#endif

#endif /* WC_EXEC_H_ */
