/*
 * wc.h -- C ABI of a GB300-native (sm_103a) library of bulk open-addressing GPU hash
 * tables, after WarpCore (Juenger et al., "WarpCore: A Library for fast Hash Tables on
 * GPUs", 2020).
 *
 * Conventions for every call below
 *   - Pointers named d_* must be device-accessible: global memory of the table's device,
 *     or host memory mapped into the device's address space (pinned with cudaHostAlloc /
 *     cudaMallocHost), which the kernels then read and write over NVLink-C2C themselves;
 *     any other pointer is refused with WC_ERR_INVALID_ARG before anything is launched.
 *     Pointers named h_* are host pointers (the *_host calls stage them through the
 *     device, which is faster than device access to host memory for scattered outputs).  The caller owns every key, value, output
 *     and offset buffer; the library owns a table's slot array, value pool and the few
 *     device words (status, counters) it allocates at create time.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Bulk operations are asynchronous with respect to the host; only calls that hand a
 *     value back to the host (wc_size, wc_load_factor, wc_get_status, wc_count_values with
 *     h_total != NULL) synchronise `stream` (Sec. IV-D of the paper).
 *   - Keys and values are unsigned integers of `key_bytes` / `value_bytes` width, packed
 *     densely (element i at byte offset i * width).  Input arrays must be aligned to
 *     their element width.
 *   - Sentinels: key 0 marks an empty slot and the all-ones key marks a tombstone
 *     (Sec. IV-B1 and IV-B5).  They cannot be stored: an input holding one is skipped
 *     and raises WC_FLAG_INVALID_KEY in the device status word.
 *   - Errors the host can see (bad arguments, allocation failure, an op the table kind
 *     does not support, a CUDA launch error) are returned at once as wc_status.
 *     Conditions found on the device accumulate as bits of the table's status word
 *     (WC_FLAG_*), read with wc_get_status.
 *   - A table is not thread-safe across host threads.  Operations of the same kind may
 *     overlap on different streams; a write (insert, erase) must not overlap any other
 *     kind of operation on the same table (Sec. IV-D).
 */
#ifndef WC_H_
#define WC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wc_table wc_table;

typedef enum {
  WC_OK = 0,
  WC_ERR_INVALID_ARG = 1,   /* null pointer, bad width, n too large, misaligned buffer */
  WC_ERR_OUT_OF_MEMORY = 2, /* cudaMalloc failed at create time */
  WC_ERR_FULL = 3,          /* reported by wc_get_status when PROBE_LIMIT was raised */
  WC_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  WC_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out (queue path) */
  WC_ERR_UNSUPPORTED = 6    /* the operation does not exist for this table kind */
} wc_status;

/* Bits of the device status word (see wc_get_status). */
enum {
  WC_FLAG_DUPLICATE_KEY = 1,  /* single-value insert met a key already stored (Sec. IV-B3);
                                 the stored value was overwritten */
  WC_FLAG_INVALID_KEY = 2,    /* an input key was a sentinel (0 or all ones) */
  WC_FLAG_PROBE_LIMIT = 4,    /* an insert visited every window without a free slot */
  WC_FLAG_POOL_EXHAUSTED = 8, /* multi-value insert ran out of value-pool space */
  WC_FLAG_COUNT_OVERFLOW = 16,/* a multi-value key would exceed 2^28 - 1 values */
  WC_FLAG_QUEUE_TIMEOUT = 32  /* the batched executor gave up waiting (bounded wait) */
};

/* Table kinds.
 *   WC_SINGLE_VALUE     one value per key (Sec. IV-B3).
 *   WC_MULTI_VALUE      many values per key: keys stored once in a key store, values in
 *                       per-key buckets of a value pool (Sec. IV-C, the bucket-list table).
 *   WC_MULTI_VALUE_OA   many values per key, open addressing: every pair takes its own
 *                       slot of the single-value slot layouts along the key's probing
 *                       sequence (Sec. IV and Sec. V-C, the multi-value hash table).  Insert
 *                       appends; count_values / retrieve_multi walk the sequence up to the
 *                       first window holding an empty slot and count or copy every match;
 *                       erase tombstones every copy.  wc_retrieve is not available.
 *   WC_HASH_SET         a set of keys (Sec. IV: HashSet), one 4- or 8-byte key per slot
 *                       (value_bytes 0): insert, wc_contains, erase.
 *   WC_COUNTING         occurrence counts per key (Sec. IV: CountingHashTable), the
 *                       single-value slot layouts: an insert of a stored key adds its weight
 *                       (wc_insert's values; NULL = 1 each) to the stored count, wrapping at
 *                       the value width; wc_retrieve returns counts; erase removes keys.
 *   WC_BLOOM_FILTER     set membership with false positives (Sec. IV: BloomFilter): a
 *                       blocked filter -- each key sets k bits inside one 256-bit block
 *                       (one 32-byte sector) picked by its hash.  min_capacity = bits
 *                       (rounded up to whole blocks), window_width = k (1..16, 0 = 8),
 *                       value_bytes 0; insert and wc_contains only (no erase); wc_size
 *                       counts inserted keys.  False-positive rate for n keys in m bits:
 *                       about the average over blocks of (1 - exp(-k x / 256))^k, x the
 *                       block's key count (Poisson with mean 256 n / m). */
enum { WC_SINGLE_VALUE = 0, WC_MULTI_VALUE = 1, WC_MULTI_VALUE_OA = 2, WC_HASH_SET = 3, WC_COUNTING = 4,
       WC_BLOOM_FILTER = 5 };

/* Table configuration.
 *   kind                 WC_SINGLE_VALUE, WC_MULTI_VALUE or WC_MULTI_VALUE_OA.
 *   key_bytes/value_bytes  single-value and open-addressing multi-value: 4/4 (key and
 *                        value packed in one 64-bit slot word, claimed by one 64-bit CAS,
 *                        Sec. IV-B1) or 8/8 (one 16-byte slot claimed by one 128-bit CAS).
 *                        bucket multi-value: key 4 or 8,
 *                        value 4 or 8 (keys are stored once in a 16-byte key-store slot
 *                        next to a handle to their values, Sec. IV-C).
 *   window_width         slots per probing window W (the inner linear-probing window of
 *                        the cooperative probing scheme, Sec. IV-B2).  Windows are
 *                        aligned to W slots.  0 = autotuned: single-value, counting and
 *                        hash-set tables in packed slots take the window width and launch
 *                        shapes the library's autotuner measures fastest for their kind,
 *                        widths and options at load 0.9 (wc_tune.h; once per process and
 *                        size class, synchronous); other tables, or with the environment
 *                        variable WC_AUTOTUNE=0, 64-byte windows (W = 64 / slot bytes).
 *                        Allowed: 8, 16, 32 (4-byte slots); 4, 8, 16, 32 (8-byte slots);
 *                        2, 4, 8, 16 (16-byte slots); 2, 4, 8 (bucket multi-value key store).
 *   min_capacity         requested slots (key-store slots for multi-value).  The table
 *                        holds capacity = p * W slots with p the smallest prime
 *                        >= ceil(min_capacity / W), so the outer double-hashing sequence
 *                        over the p windows visits every window once (Sec. IV-B2).
 *                        p must stay below 2^32.
 *   value_pool_capacity  bucket multi-value only: value elements in the pool (headers of
 *                        repeat-insert segments included); at most 2^35.  Ignored otherwise.
 *   seed                 seeds the two hash functions of the outer probing scheme.
 *   device               CUDA device ordinal the table lives on.
 *   l2_persist           1 = launch this table's kernels with an L2 access-policy window
 *                        marking the slot array persisting (useful when it fits in L2).
 *   options              WC_OPT_* bits (0 = none).
 *   bucket_first_size    bucket multi-value only: 0 (default) = every insert call appends
 *                        one bucket of exactly its count per key (the bucket list with
 *                        lambda = 1, s0 = count, Sec. V-C); s0 >= 1 = the growth strategy
 *                        of Sec. IV-C: a key's buckets have sizes s0, s1 = ceil(lambda * s0),
 *                        ..., s_i = ceil(lambda * s_{i-1}), each filled before the next is
 *                        allocated, so calls append into the key's last bucket first.
 *   bucket_growth        lambda >= 1 for the growth strategy (ignored when
 *                        bucket_first_size = 0).  lambda > 1 must reach 2^28 values within
 *                        1024 buckets (e.g. lambda = 1.1, s0 = 1 needs 161); lambda = 1 gives
 *                        buckets of s0 values each.
 */
typedef struct {
  int32_t kind;
  int32_t key_bytes;
  int32_t value_bytes;
  int32_t window_width;
  int32_t device;
  int32_t l2_persist;
  int32_t options;
  int32_t reserved;       /* 0 */
  uint64_t min_capacity;
  uint64_t value_pool_capacity;
  uint64_t seed;
  uint64_t bucket_first_size;
  double bucket_growth;
} wc_table_config;

/* WC_OPT_OVERFLOW_BITS (single-value, counting and hash-set tables; no counterpart in the
 * paper): keep eight overflow bits per window (one byte).  Each key has a 3-bit tag g, the
 * low three bits of h = fmix64(key ^ seed) (wc_device_api.cuh: probe_init); an insert that
 * walks past a window because it holds no empty slot sets bit g of that window's byte.
 * Lookups and erases then stop at a window without the key, without an empty slot and with
 * bit g clear -- a key of tag g stored further on would have set it -- instead of walking
 * on to a window with an empty slot.  Shortens the walks of absent keys at high load (W = 8,
 * load 0.9: 2.9 windows per absent key without the bits, 1.2 with them); costs present keys
 * outside their first window one dependent read of the byte per window (skewed queries of
 * present keys: slower), and inserts one atomic OR per window walked past.  The bits cost
 * one byte per window. */
enum { WC_OPT_OVERFLOW_BITS = 1 };

/* WC_OPT_SOA (single-value tables): struct-of-arrays layout (Sec. IV-A) -- the keys in one
 * array (4- or 8-byte slots, probed like a hash set's), the values in a second array of
 * the same length.  An insert claims the key slot with one CAS and then writes the value
 * with a plain store (complete when the call is; the paper's relaxed value writes); a hit
 * reads the value at the key's index.  Windows are of W keys (4-byte keys: 8, 16, 32,
 * default 16; 8-byte keys: 4, 8, 16, 32, default 8).  Not served by the batched executor,
 * wc_insert_noalloc or the device API. */
enum { WC_OPT_SOA = 2 };

/* Sizes of a created table (host copy; no device access). */
typedef struct {
  uint64_t capacity;        /* slots (key-store slots for multi-value) = windows * W */
  uint64_t windows;         /* p, prime */
  uint64_t slot_bytes;      /* 8 or 16 */
  uint64_t table_bytes;     /* bytes of the slot array */
  uint64_t pool_capacity;   /* multi-value value-pool elements (0 for single-value) */
  uint64_t device_bytes;    /* every device byte the table owns */
  int32_t window_width;     /* W */
  int32_t kind;
  int32_t options;          /* WC_OPT_* bits the table was created with */
  int32_t reserved;
  uint64_t work_bytes;      /* device scratch and staging the table holds at the moment
                               (grown on demand by region-split calls and host-buffer calls,
                               kept until wc_table_destroy); not in device_bytes */
} wc_table_info;

/* Launch shape of one operation class.  group_size = lanes that probe one key together
 * (the cooperative group of Sec. IV-B2; W / group_size slots per lane, walked
 * consecutively by each lane, Sec. IV-B2 "fixed window with variable CG size");
 * block_threads = CUDA block size, 32..256 in steps of 32 (the bucket multi-value table's
 * insert: 256 or 512, the block of its aggregation passes, default 256, with tiles of four
 * keys per thread); blocks_per_sm = resident blocks per SM the grid is
 * sized for (0 = the occupancy limit); scheme = how a bulk call visits the table
 * (WC_SCHEME_*); region_mib = table MiB per region of the blocked scheme (0 = 32; a region
 * holds a power of two of windows, the most that fit in region_mib MiB);
 * keys_in_flight = keys each group probes at once (1 or 2; 0 = 1): with 2, every trip of
 * a group loads the windows of two keys, so twice as many random window reads are in
 * flight per warp (single-value retrieves of up to 32 bytes of window per lane; elsewhere
 * it is taken as 1).  Default 2 for lookups of 4+4-byte single-value tables, else 1. */
typedef struct {
  int32_t group_size;
  int32_t block_threads;
  int32_t blocks_per_sm;
  int32_t scheme;
  int32_t region_mib;
  int32_t keys_in_flight;
} wc_launch;

/* WC_SCHEME_DIRECT: every key probes the table where its hash points, in input order.
 * WC_SCHEME_BLOCKED: the batch is first split by table region (the multi-split of
 * Sec. IV-E applied to regions of one table) and then probed region by region, so the
 * active part of the table stays in L2; needs scratch of n * (key + value) bytes, which
 * the table allocates on first use (stream-ordered) and keeps.  Inserts of single-value,
 * counting, hash-set and open-addressing multi-value tables; retrieves of single-value and
 * counting tables (the results are split back into input order).  WC_SCHEME_AUTO picks
 * BLOCKED for those inserts when the batch holds at least 2^18 pairs and the table is
 * larger than 64 MiB, DIRECT otherwise.
 * WC_SCHEME_DEDUP (lookups of single-value, counting and hash-set tables: wc_retrieve,
 * wc_contains): direct probing, but equal keys among each 32 consecutive queries of a
 * warp are found with one warp vote (__match_any_sync) and probed once, the result written
 * to each of their positions.  For skewed query streams, where the hot keys repeat inside
 * a warp's queries; on distinct queries it only adds the vote. */
enum { WC_SCHEME_AUTO = 0, WC_SCHEME_DIRECT = 1, WC_SCHEME_BLOCKED = 2, WC_SCHEME_DEDUP = 3 };

enum { WC_OP_INSERT = 0, WC_OP_RETRIEVE = 1, WC_OP_ERASE = 2, WC_OP_COUNT = 3, WC_OP__N = 4 };

/* ---- lifecycle ------------------------------------------------------------------ */

/* Plan a table's geometry without a device: p = smallest prime >= ceil(min_capacity/W),
 * capacity = p * W (Sec. IV-B2, c = p * 32 generalised to c = p * W).  Host only.
 * Returns WC_ERR_INVALID_ARG for W outside 1..64 or p >= 2^32. */
wc_status wc_plan_capacity(uint64_t min_capacity, int32_t window_width, uint64_t* h_windows,
                           uint64_t* h_capacity);

/* Create a table on cfg->device: allocates and clears (every slot = empty key) its slot
 * array, value pool and status/counter words.  Synchronous.  *out is owned by the caller
 * and released with wc_table_destroy. */
wc_status wc_table_create(wc_table** out, const wc_table_config* cfg);

/* Free everything the table owns.  The caller must make sure no work on it is pending. */
wc_status wc_table_destroy(wc_table* t);

/* Reset to empty on `stream`: every slot back to the empty key, counters, status word
 * and value-pool cursor to zero (Sec. IV-B1: slots start as k_e). */
wc_status wc_table_clear(wc_table* t, void* stream);

wc_status wc_table_get_info(const wc_table* t, wc_table_info* h_out);

/* Override the launch shape of one operation class (see wc_launch); the autotuners
 * (wc_tune.h and the Python package's) call this.  group_size must divide W and give 8..64 bytes per lane
 * (or be 1..32 with W / group_size slots per lane <= 8).  Host only. */
wc_status wc_table_set_launch(wc_table* t, int32_t op, const wc_launch* launch);
wc_status wc_table_get_launch(const wc_table* t, int32_t op, wc_launch* h_out);

/* ---- bulk operations (Sec. IV-B3 .. IV-B5) ----------------------------------------- */

/* Insert n pairs (d_keys[i], d_values[i]).  Open-addressing multi-value: every pair
 * claims the earliest free or tombstoned slot of its key's probing sequence, with no
 * duplicate check (a table at capacity raises WC_FLAG_PROBE_LIMIT for the pairs that find
 * no slot).  Single-value: a new key claims the earliest
 * free or tombstoned slot of its probing sequence with one CAS of the packed pair
 * (Sec. IV-B2 steps 1-7); a key already present gets its value overwritten and raises
 * WC_FLAG_DUPLICATE_KEY (Sec. IV-B3).  If the same key occurs several times in one
 * batch, the stored value is one of that batch's values for it.  Multi-value: every
 * pair is appended (Sec. IV-B4); values of one call are stored contiguously per key in
 * the value pool (a bucket of exactly that call's count, linked to the key's earlier
 * buckets, Sec. IV-C with lambda = 1, s0 = count).  A multi-value insert keeps per-tile
 * records of its counting pass in the table's scratch (12 bytes per pair, plus the region
 * split's key + value bytes per pair for batches of 2^20 or more into key stores over
 * 64 MiB), grown on demand and held until wc_table_destroy.  n < 2^32. */
wc_status wc_insert(wc_table* t, const void* d_keys, const void* d_values, uint64_t n,
                    void* stream);

/* Insert without allocating: the same result as wc_insert on a single-value table (the
 * paper has no counterpart -- this is a deployment variant of the region-split insert).
 * For callers that cannot allocate device memory during the call (memory reserved up
 * front, another allocator owning the device, code that must not grow a caching
 * allocator): the batch is split by table region inside a static device buffer of
 * WC_NOALLOC_SCRATCH_BYTES that the library holds in every context that loads it, until
 * the process exits.  n may be at most WC_NOALLOC_SCRATCH_BYTES / (key_bytes +
 * value_bytes) minus a few elements (2,097,088 pairs of 4+4 bytes; 1,048,544 of 8+8);
 * larger n returns WC_ERR_INVALID_ARG -- split the batch.  Keys and values must be memory
 * the table's device can reach, as for wc_insert (pageable host memory or another GPU's
 * memory: WC_ERR_INVALID_ARG).  The first call on a device (and the first after that
 * device's context was reset) looks up the buffer's device address with that device
 * current; under lazy module loading that lookup is also what places the buffer on the
 * device, so it can fail with WC_ERR_OUT_OF_MEMORY when the device is full: make that first
 * call early, and before capturing any stream.  All calls on a device share the buffer,
 * which keeps what the last call left in it: calls whose GPU work may overlap (different
 * streams with no ordering) race and must be ordered by the caller.  Multi-value and
 * struct-of-arrays tables return WC_ERR_UNSUPPORTED. */
#define WC_NOALLOC_SCRATCH_BYTES (16ull << 20)
wc_status wc_insert_noalloc(wc_table* t, const void* d_keys, const void* d_values, uint64_t n,
                            void* stream);

/* wc_insert (Sec. IV-B2, IV-B3) from HOST buffers: h_keys[i], h_values[i] as d_keys and
 * d_values, in host memory (pinned for full speed; pageable memory works, with copies
 * synchronous to the host).  The batch moves to the device in chunks of up to 2^25 pairs
 * (the first of up to 2^23) through three device staging buffers the table keeps
 * (allocated on first use, freed by wc_table_destroy), each chunk's copy on the table's own
 * copy stream overlapping the inserts of the chunks before it on `stream`.  Asynchronous:
 * the host buffers stay owned by the caller and must stay valid and unchanged until
 * `stream` has passed this call.  Values may be NULL where wc_insert allows it.  Errors:
 * WC_ERR_INVALID_ARG for a NULL table or buffer or a buffer the runtime reports as device
 * or managed memory, WC_ERR_OUT_OF_MEMORY when the staging buffers cannot be allocated,
 * WC_ERR_CUDA for a failed copy; otherwise as wc_insert, chunk by chunk (chunks before a
 * failing one stay inserted). */
wc_status wc_insert_host(wc_table* t, const void* h_keys, const void* h_values, uint64_t n, void* stream);

/* Single-value retrieve (Sec. IV-B4; counting tables: the counts): d_values_out[i] = value
 * of d_keys[i], or all ones
 * (NOT_FOUND) when absent; d_found_or_null[i] = 1/0 when the mask is given (a stored value
 * may itself be all ones).  Probing stops at the key or at the first window holding an
 * empty slot; in tables with WC_OPT_OVERFLOW_BITS also at the first window without the
 * key whose overflow bit for the key's tag is clear (no key of that tag was ever placed
 * beyond it).  Multi-value tables return WC_ERR_UNSUPPORTED. */
wc_status wc_retrieve(wc_table* t, const void* d_keys, uint64_t n, void* d_values_out,
                      uint8_t* d_found_or_null, void* stream);

/* wc_retrieve (Sec. IV-B4) from and into HOST buffers: h_keys[i] in, h_values_out[i] and
 * (if given) h_found_or_null[i] out, layouts as wc_retrieve's, all owned by the caller.
 * Chunks of up to 2^23 queries are copied in on one copy stream, looked up on `stream` and
 * the results copied out on another, so the copies of neighbouring chunks overlap the
 * lookups; `stream` completes after the last copy out, and the outputs may be read only
 * then.  Single-value and counting tables (others: WC_ERR_UNSUPPORTED).  Asynchronous and
 * with the errors of wc_insert_host. */
wc_status wc_retrieve_host(wc_table* t, const void* h_keys, uint64_t n, void* h_values_out,
                           uint8_t* h_found_or_null, void* stream);

/* Membership (Sec. IV-B4 without values): d_found[i] = 1 if d_keys[i] is stored, else 0
 * (Bloom filters: 1 if all the key's bits are set -- possibly a false positive, never a
 * false negative).  Single-value, counting, hash-set and Bloom-filter tables. */
wc_status wc_contains(wc_table* t, const void* d_keys, uint64_t n, uint8_t* d_found, void* stream);

/* Erase (Sec. IV-B5): the key's slot becomes a tombstone; absent keys are a no-op.
 * Multi-value: removes every value of the key (bucket table: its pool space is not
 * reused; open-addressing table: every copy's slot becomes a tombstone). */
wc_status wc_erase(wc_table* t, const void* d_keys, uint64_t n, void* stream);

/* Multi-value counting pass (Sec. IV-B4, both multi-value kinds): d_offsets[0..n]
 * (n+1 uint64, caller-allocated)
 * receives the exclusive prefix sum of the per-query value counts, so query i's values
 * go to [d_offsets[i], d_offsets[i+1]) and d_offsets[n] is the total.  If h_total_or_null
 * is given the call synchronises `stream` and stores the total there.  Sentinel
 * queries count 0.  Single-value tables return WC_ERR_UNSUPPORTED. */
wc_status wc_count_values(wc_table* t, const void* d_keys, uint64_t n, uint64_t* d_offsets,
                          uint64_t* h_total_or_null, void* stream);

/* Multi-value retrieve into CSR form (Sec. IV-B4): writes the values of query i to
 * d_values_out[d_offsets[i] .. d_offsets[i+1]), with d_offsets from wc_count_values on
 * the same keys and an unchanged table.  The order of values inside a segment is
 * unspecified.  d_values_out holds d_offsets[n] elements of value_bytes and must not be
 * NULL when n > 0. */
wc_status wc_retrieve_multi(wc_table* t, const void* d_keys, uint64_t n,
                            const uint64_t* d_offsets, void* d_values_out, void* stream);

/* ---- metrics (blocking) ---------------------------------------------------------- */

/* Single-value: live keys.  Multi-value (both kinds): stored key-value pairs.
 * Synchronises stream. */
wc_status wc_size(wc_table* t, uint64_t* h_out, void* stream);

/* Multi-value: distinct live keys (open-addressing kind: counted on the device by a pass
 * over the slots, which finds each key's first copy along its probing sequence).
 * Single-value: same as wc_size.  Synchronises stream. */
wc_status wc_num_keys(wc_table* t, uint64_t* h_out, void* stream);

/* Bucket multi-value: value-pool elements allocated so far (bucket values, their headers
 * and alignment padding; the storage-density denominator of Sec. IV-C).  Other kinds: 0.
 * Synchronises stream. */
wc_status wc_value_pool_used(wc_table* t, uint64_t* h_out, void* stream);

/* Load factor alpha = live keys / capacity (key-store load for the bucket multi-value
 * table, Sec. II; occupied slots = stored pairs / capacity for the open-addressing one).
 * Single-value tables have storage density rho = alpha (Sec. IV-C). */
wc_status wc_load_factor(wc_table* t, double* h_out, void* stream);

/* Read the device status word (WC_FLAG_* bits accumulated since the last clear); with
 * clear != 0 it is reset to 0 afterwards.  Synchronises stream. */
wc_status wc_get_status(wc_table* t, uint32_t* h_flags, int32_t clear, void* stream);

/* wc_get_status with clear, folded into a status code: WC_ERR_TIMEOUT if QUEUE_TIMEOUT
 * was raised, WC_ERR_FULL if PROBE_LIMIT, POOL_EXHAUSTED or COUNT_OVERFLOW was (pairs
 * were not stored), else WC_OK (DUPLICATE_KEY and INVALID_KEY are warnings).  The raw
 * bits go to *h_flags_or_null.  Synchronises stream. */
wc_status wc_check_status(wc_table* t, uint32_t* h_flags_or_null, void* stream);

/* Static description of a status code. */
const char* wc_status_string(wc_status s);

/* ---- device-side access (include/wc_device_api.cuh) ------------------------------- */

/* Everything a user kernel needs to operate on a table with the device API of
 * wc_device_api.cuh: device pointers and geometry, passed to kernels by value.  The
 * pointers stay valid until wc_table_destroy. */
typedef struct {
  void* slots;                 /* capacity slots, layout of wc_table_config */
  uint32_t* status;            /* the table's status word (WC_FLAG_* bits) */
  unsigned long long* size;    /* stored pairs */
  uint32_t* overflow_bits;     /* WC_OPT_OVERFLOW_BITS tables (byte w = window w), else NULL */
  uint64_t seed;
  uint64_t capacity;           /* windows * window_width */
  uint32_t windows;            /* p */
  uint32_t window_width;       /* W */
  int32_t kind;
  int32_t key_bytes;
  int32_t value_bytes;
  int32_t slot_bytes;
  /* bucket multi-value tables with a growth strategy (per-element appends); else zero */
  void* pool;                          /* value pool, value_bytes per element */
  unsigned long long* pool_cursor;     /* next free pool element */
  unsigned long long* num_keys;        /* distinct live keys */
  const uint64_t* bucket_cum_size;     /* lambda > 1: values in buckets 0..i, i < bucket_count */
  const uint64_t* bucket_cum_foot;     /* lambda > 1: pool elements of buckets 0..i */
  uint64_t pool_capacity;              /* pool elements */
  uint64_t bucket_size;                /* lambda = 1: values per bucket (s0) */
  uint64_t bucket_foot0, bucket_foot;  /* lambda = 1: pool elements of bucket 0 / of a later one */
  uint32_t bucket_count;               /* lambda > 1: entries of the two tables */
  int32_t growth;                      /* 1: lambda = 1, 2: lambda > 1 (the tables) */
  uint64_t wait_ns;                    /* bound of an append's wait for a blocked list (0: 1 s) */
} wc_device_view;

/* Fill *h_out for a single-value table (per-element insert / retrieve / erase, for_each,
 * for_all), a hash set (set_insert / set_contains / set_erase), a counting table
 * (count_add / count_get), an open-addressing multi-value table (for_all only) or a bucket
 * multi-value table created with a growth strategy (bucket_first_size > 0; per-element
 * appends, whose pool must hold fewer than 2^34 elements).  Host only.
 * WC_ERR_UNSUPPORTED for struct-of-arrays tables, Bloom filters and other bucket
 * multi-value tables (their buckets are sized per bulk call). */
wc_status wc_table_device_view(const wc_table* t, wc_device_view* h_out);

/* ---- host copies: inspection, checkpoint and resume (no counterpart in the paper) -- */

/* Copy the slot array (wc_table_info.table_bytes bytes, slot i at byte i * slot_bytes,
 * layout as in wc_table_config) to host memory h_out of `bytes` >= table_bytes.
 * Synchronises stream.  Used by the slot-dump invariant checks of the tests. */
wc_status wc_table_dump_slots(const wc_table* t, void* h_out, uint64_t bytes, void* stream);

/* Copy a table's overflow bits (WC_OPT_OVERFLOW_BITS): ceil(windows / 4) uint32 words, byte
 * w % 4 (little-endian) of word w / 4 = window w's eight bits, to h_out (`words` >= that).  WC_ERR_UNSUPPORTED for a
 * table without them.  Synchronises stream. */
wc_status wc_table_dump_overflow_bits(const wc_table* t, uint32_t* h_out, uint64_t words, void* stream);

/* Bytes of a whole-table snapshot: a header with the table's geometry, then its slots,
 * counters, status word and (multi-value) pending array and value pool. */
uint64_t wc_table_snapshot_bytes(const wc_table* t);

/* Write a snapshot to host memory h_out (`bytes` >= wc_table_snapshot_bytes).  No
 * operation on the table may be in flight on another stream.  Synchronises stream. */
wc_status wc_table_snapshot(const wc_table* t, void* h_out, uint64_t bytes, void* stream);

/* Replace the table's contents with a snapshot taken from a table of the same kind,
 * widths, window width, window count, pool capacity and seed (WC_ERR_INVALID_ARG
 * otherwise, table unchanged).  Synchronises stream. */
wc_status wc_table_restore(wc_table* t, const void* h_in, uint64_t bytes, void* stream);

/* ---- testing hook --------------------------------------------------------------- */

/* The next `count` device allocations of the library (wc_table_create, the scratch of
 * the region-split insert) fail as if the device were out of memory; 0 turns it off.
 * Process-wide.  For tests of the out-of-memory paths. */
wc_status wc_debug_fail_allocations(uint32_t count);

#ifdef __cplusplus
}
#endif

#endif /* WC_H_ */
