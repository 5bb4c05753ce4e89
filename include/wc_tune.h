/*
 * wc_tune.h -- the library's autotuner: picks the probing window width W and the launch
 * shape of each bulk operation (lanes per key, keys in flight) by timing the library's own
 * kernels on a synthetic sample.
 *
 * The paper fixes the window (32 slots, one warp) and lets the user pick the cooperative
 * group size by hand (Sec. IV-B2, "fixed window with variable CG size"); it reports that
 * the best size depends on the key width and the load (Sec. V-A).  Here the choice is
 * measured on the GPU at hand: for every window width allowed for the table's slot width
 * (or the one the caller fixes), a table of the caller's kind, widths and options is
 * filled to the given load with `sample_keys` distinct keys, and every valid group size
 * of insert, retrieve (and keys in flight 1 or 2 where the lookup kernel supports it) and
 * erase is timed with CUDA events (best of three calls).  A lookup is timed on two query
 * streams: uniform keys, half of them absent (bound by HBM), and queries over a hot 1/64 of
 * the keys (bound by L2, as a skewed stream's hot keys are); a shape has to serve both.
 * W is the one with the smallest insert + retrieve time.  A shape or width replaces the
 * library's default only when it is more than 10 % faster: the sample stands for tables of
 * other sizes and query streams, and only clear wins on it carry over to them.
 *
 * wc_table_create uses it for window_width = 0 (wc.h): single-value, counting and
 * hash-set tables in packed slots are created with the tuned W and shapes for load 0.9,
 * on a sample of 2^20 keys for tables of up to 32 MiB of slots (they live in L2) and on a
 * table of 256 MiB of slots otherwise (twice the L2), cached per process, so the first such
 * create of a process takes a fraction of a second longer.  The environment variable
 * WC_AUTOTUNE=0 turns that off (the fixed defaults are used).
 *
 * Conventions as in wc.h.
 */
#ifndef WC_TUNE_H_
#define WC_TUNE_H_

#include <stdint.h>

#include "wc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t window_width;    /* the chosen W */
  int32_t candidates;      /* launch shapes timed (all window widths) */
  int32_t from_cache;      /* 1: answered from the process-wide cache, nothing was timed */
  int32_t reserved;
  wc_launch launch[3];     /* the chosen shapes of WC_OP_INSERT, WC_OP_RETRIEVE, WC_OP_ERASE */
  double ms[3];            /* their best time on the sample: insert of sample_keys pairs,
                              lookup of sample_keys uniform queries (half of them absent)
                              plus sample_keys hot ones, erase of the sample_keys keys */
  uint64_t sample_keys;
  double load;
} wc_tuning;

/* Tune for tables configured as *cfg (kind WC_SINGLE_VALUE, WC_COUNTING or WC_HASH_SET,
 * packed slots; cfg->window_width 0 = tune W too, else keep it; min_capacity is ignored:
 * the sample sets the size) at load factor `load` (0.05 .. 0.99) with `sample_keys` keys
 * (2^10 .. 2^26).  use_cache != 0: a result for the same device, kind, widths, options,
 * window width, load (to 0.01) and sample size is returned from the process-wide cache
 * when there is one, and a new result is stored there.  Synchronous: creates its own
 * tables, buffers and stream on cfg->device and frees them.  Errors: WC_ERR_INVALID_ARG
 * (arguments), WC_ERR_UNSUPPORTED (other kinds, struct-of-arrays tables),
 * WC_ERR_OUT_OF_MEMORY (the sample does not fit), WC_ERR_CUDA. */
wc_status wc_autotune(const wc_table_config* cfg, double load, uint64_t sample_keys, int32_t use_cache,
                      wc_tuning* h_out);

/* The sample size wc_table_create tunes on for window_width = 0 and this configuration
 * (its load is 0.9): 2^20 keys when min_capacity slots take at most 32 MiB, else the keys
 * of a 256 MiB table at load 0.9.  A later wc_autotune(cfg, 0.9, this, 1, ...) returns
 * that tuning from the cache.  Host only; 0 for a NULL cfg. */
uint64_t wc_autotune_sample_keys(const wc_table_config* cfg);

/* Set a table's insert, retrieve and erase launch shapes from a tuning (wc_table_set_launch
 * for each).  WC_ERR_INVALID_ARG when the table's window width differs from the tuning's
 * or a shape is not valid for the table.  Host only. */
wc_status wc_table_apply_tuning(wc_table* t, const wc_tuning* tuning);

#ifdef __cplusplus
}
#endif

#endif /* WC_TUNE_H_ */
