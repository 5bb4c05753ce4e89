/*
 * wc_roofline.h -- measurement support: the random-access roofline of the device.
 *
 * The paper has no counterpart; its hot path is bounded by random accesses to global
 * memory (one probing window per key and probe step, Sec. IV-B2), so the library ships
 * the probes that measure that bound on the device it runs on:
 *   - random reads of `access_bytes` contiguous, aligned bytes at uniformly random
 *     positions of a buffer (the window load of a probe), by one thread or by a group of
 *     adjacent threads (a probing group), with a chosen number in flight per thread, and
 *   - the same read followed by a 64-bit CAS on the first word (the slot claim of an
 *     insert), and
 *   - random stores of `access_bytes` (the scatter of per-query results back to their
 *     input positions).
 * Conventions as in wc.h (device pointers d_*, host pointers h_*, void* stream).
 */
#ifndef WC_ROOFLINE_H_
#define WC_ROOFLINE_H_

#include <stdint.h>

#include "wc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint64_t buffer_bytes;   /* bytes of d_buffer accessed (multiple of access_bytes) */
  uint64_t accesses;       /* number of random accesses */
  uint64_t seed;           /* positions are fmix64(seed ^ i) scaled to the buffer */
  uint32_t access_bytes;   /* 8, 16, 32, 64 or 128 (mode 2 also 4) */
  uint32_t mode;           /* 0 = read only, 1 = read then CAS (old -> old + 1), 2 = store */
  uint32_t block_threads;  /* 0 = 256 */
  uint32_t blocks_per_sm;  /* 0 = occupancy limit */
  uint32_t in_flight;      /* reads: independent accesses in flight per thread, 1/2/4/8/16 (0 = 4) */
  uint32_t lanes;          /* reads: adjacent threads sharing one access, each reading
                              access_bytes / lanes >= 8 bytes of it, 1/2/4 (0 = 1) */
} wc_rand_access_config;

/* Launch the probe on `stream` over d_buffer (device, buffer_bytes, 256-byte aligned).
 * d_sink (device, one uint64) receives an XOR of everything read, so the loads cannot be
 * elided (unused by mode 2, still required).  Mode 2 overwrites the buffer.
 * Asynchronous; time it with events on `stream`. */
wc_status wc_bench_random_access(void* d_buffer, const wc_rand_access_config* cfg, uint64_t* d_sink,
                                 void* stream);

/* Device-API probe (include/wc_device_api.cuh) on a single-value 4+4-byte table: one
 * kernel whose threads produce the keys k_i = (i * 2654435761 mod 2^32) xor key_seed
 * (i < n; distinct) and, per thread, mode 0 inserts (k_i, i), mode 1 looks k_i up and adds
 * the found values into d_sink (one uint64) -- a fused producer with no key batch in
 * memory.  Asynchronous on `stream`. */
wc_status wc_bench_device_api(wc_table* t, int32_t mode, uint64_t n, uint32_t key_seed, uint64_t* d_sink,
                              void* stream);

/* The same fused producer with the device API's group-cooperative operations: tiles of
 * `group` threads (1, 2 or 4; W 8 or 16) produce one key each and insert it (mode 0) or look
 * it up (mode 1) together -- one window read per tile, votes over the tile. */
wc_status wc_bench_device_api_group(wc_table* t, int32_t mode, int32_t group, uint64_t n, uint32_t key_seed,
                                    uint64_t* d_sink, void* stream);

/* Device-API probe of the bucket list (include/wc_device_api.cuh, wc_dev::append): one
 * thread per pair appends (d_keys[i], d_values[i]) -- device arrays of the table's key and
 * value widths -- to a bucket multi-value table created with a growth strategy, every pair
 * an independent concurrent append (Sec. IV-C).  Status conditions go to the table's
 * status word.  Asynchronous on `stream`; WC_ERR_UNSUPPORTED for other tables. */
wc_status wc_bench_mv_append(wc_table* t, const void* d_keys, const void* d_values, uint64_t n, void* stream);

/* The CUDA context's L2 fetch-granularity limit (cudaLimitMaxL2FetchGranularity, bytes;
 * a hint of how much the L2 fetches from DRAM on a miss).  Process-local: the setting
 * ends with the process. */
wc_status wc_set_l2_fetch_granularity(int32_t bytes);
wc_status wc_get_l2_fetch_granularity(int32_t* h_bytes);

#ifdef __cplusplus
}
#endif

#endif /* WC_ROOFLINE_H_ */
