/*
 * cafs.h -- C ABI of the GB300 (sm_103a) count-and-emit frequency sort.
 *
 * The operation is the one the CAFS paper ("CAFS: A Cache-Aware Frequency
 * Sort for Low-Cardinality Integer Data on x86-64") defines:
 *
 *   Sec. 3.1   sort N integer keys ascending; equal keys are
 *              indistinguishable, so only the values are produced;
 *   Sec. 4.1   count every distinct key, then emit (key, count) pairs in
 *              increasing key order;
 *   Alg. 2     estimate the number of distinct keys K from 1024 strided
 *              samples with the smoothed Chao1 estimator (Eq. 5);
 *   Alg. 3     dispatch: already sorted -> bypass, N < 2048 -> direct sort,
 *              K_hat <= 8 and u <= 8 -> tiny count, 2*K_hat > N -> radix
 *              fallback, otherwise the hash-count main path;
 *   Eq. 6      size the hash table M = bit_ceil(8*K_hat/cap), 8 <= M <=
 *              bit_ceil(N/cap), C = M*cap slots;
 *   Alg. 4     a guard reroutes to the fallback when the table overflows;
 *              here the guard fires when the number of distinct keys exceeds
 *              L = C/2 (an order-independent restatement of the paper's
 *              insertion-order-dependent spill test).
 *
 * Keys are signed two's-complement int32 or int64 sorted ascending (the
 * paper's Sec. 5 types); unsigned and IEEE-float keys are accepted too (see
 * cafs_dtype).  Beyond the paper: a stable argsort (Sec. 3.1's permutation),
 * a batched form, a request server and per-call hash seeds.
 *
 * Conventions shared by every entry point:
 *   - Device pointers are caller-owned CUDA device (or managed) memory of n
 *     elements, naturally aligned for the element type.  `keys` is read-only
 *     unless out == keys (in-place sorting is allowed); any other overlap of
 *     the two ranges is rejected with CAFS_ERR_ALIAS.
 *   - n == 0 is a no-op returning CAFS_OK (NULL pointers allowed then).
 *   - n must be <= 2^32 - 1 (counts are 32-bit, like the paper's bucket
 *     counters, Sec. 4.2); larger n returns CAFS_ERR_TOO_LARGE.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) on the current device.  Argument errors are returned
 *     synchronously and nothing is enqueued.  Device-side failures (a bounded
 *     wait that ran out) are reported through cafs_report.device_status.
 *   - The library owns a workspace per (device, stream), allocated on first
 *     use and grown on demand (growing synchronises the device).  Calls on the
 *     same stream are serialised by the stream; calls on different streams use
 *     different workspaces and may overlap.
 *   - All entry points are thread-safe.
 */
#ifndef CAFS_H
#define CAFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Key types.  Signed integers sort in their natural order (the paper ships
 * int32/int64, Sec. 5).  Unsigned integers sort in their natural order and
 * IEEE-754 floats in the standard's totalOrder (negative NaNs, -inf, negative
 * numbers, -0, +0, positive numbers, +inf, positive NaNs; equal keys are
 * equal bit patterns): the library maps them onto signed integers of the same
 * width by an order-preserving bijection (unsigned: flip the sign bit; float:
 * flip the magnitude bits of negative values), sorts those, and maps the
 * output back, one extra elementwise read and write of the column each way.
 * cafs_sort, cafs_sort_ex, cafs_sort_host, cafs_estimate_k, cafs_argsort,
 * the batched form (per column: keys mapped into out before the launch,
 * sorted there, mapped back after it) and the request server accept every
 * type; the allocation-free entry point takes CAFS_INT32 and CAFS_INT64 only
 * (else CAFS_ERR_UNSUPPORTED_DTYPE). */
typedef enum {
  CAFS_INT32 = 0,
  CAFS_INT64 = 1,
  CAFS_UINT32 = 2,
  CAFS_UINT64 = 3,
  CAFS_FLOAT32 = 4,
  CAFS_FLOAT64 = 5
} cafs_dtype;

typedef enum {
  CAFS_OK = 0,
  CAFS_ERR_INVALID_ARGUMENT = 1,
  CAFS_ERR_UNSUPPORTED_DTYPE = 2,
  CAFS_ERR_TOO_LARGE = 3,
  CAFS_ERR_ALIAS = 4,
  CAFS_ERR_OUT_OF_MEMORY = 5,
  CAFS_ERR_CUDA = 6,
  CAFS_ERR_TIMEOUT = 7,
  CAFS_ERR_INTERNAL = 8,
  CAFS_ERR_BUSY = 9
} cafs_status;

/* The branch that produced (or, for the dispatcher, was selected for) the
 * output.  Table 2 / Algorithm 3 give EMPTY..MAIN; the *_RADIX and
 * TINY_MISS_* values name what happens after the tiny-count check (Sec. 4.4)
 * and the overflow guard (Alg. 4). */
typedef enum {
  CAFS_PATH_EMPTY = 0,
  CAFS_PATH_BYPASS_SORTED = 1,
  CAFS_PATH_SMALL_N = 2,
  CAFS_PATH_TINY = 3,
  CAFS_PATH_MAIN = 4,
  CAFS_PATH_HIGH_ENTROPY_RADIX = 5,
  CAFS_PATH_MAIN_OVERFLOW_RADIX = 6,
  CAFS_PATH_TINY_MISS_MAIN = 7,
  CAFS_PATH_TINY_MISS_MAIN_OVERFLOW_RADIX = 8
} cafs_path;

/* Sampler, Chao1 and sizing results (Alg. 2, Eq. 5, Eq. 6). */
typedef struct {
  uint64_t n;          /* number of keys                                    */
  uint64_t stride;     /* max(1, floor(n / 1024))                           */
  uint32_t n_samples;  /* min(n, 1024)                                      */
  uint32_t u;          /* distinct sample values                            */
  uint32_t f1;         /* sample values seen exactly once                   */
  uint32_t f2;         /* sample values seen exactly twice                  */
  uint64_t k_hat;      /* u + floor(f1^2 / (2 (f2 + 1))), or n if u == 1024 */
  int32_t saturated;   /* 1 when u == 1024                                  */
  int32_t sample_nondecreasing; /* the samples, in position order, ascend   */
  uint64_t M;          /* buckets, Eq. 6 with clamps                        */
  uint64_t C;          /* slots = M * cap (cap 4 for int64, 8 for int32)    */
  uint64_t L;          /* overflow limit on distinct keys = C / 2           */
  cafs_path dispatch;  /* Alg. 3 decision: EMPTY, BYPASS_SORTED, SMALL_N,
                          TINY, HIGH_ENTROPY_RADIX or MAIN                  */
} cafs_estimate;

/* What a finished sort did. */
typedef struct {
  cafs_estimate est;   /* the estimate the dispatcher used               */
  cafs_path path;      /* branch that produced the output                */
  uint64_t k_distinct; /* distinct keys counted (TINY, MAIN, TINY_MISS_MAIN
                          paths); 0 when the branch does not count        */
  cafs_status device_status; /* CAFS_OK or CAFS_ERR_TIMEOUT               */
  /* Device timestamps (ns, GPU global timer) at the pipeline's phase
   * boundaries: [0] start, [1] sampled, [2] monotone scan done, [3] counted,
   * [4] pairs sorted and scanned, [5] last CTA finished; 0 where a phase did
   * not run (N < 2048 columns report none). */
  uint64_t timeline_ns[6];
} cafs_report;

/* Sort n keys from `keys` into `out` (ascending, signed), asynchronously on
 * `stream`.  Implements Sec. 3.1 via Algorithms 2-4.  Returns after
 * enqueueing.  `keys` and `out` are device pointers (see conventions). */
cafs_status cafs_sort(const void* keys, size_t n, cafs_dtype dtype, void* out,
                      void* stream);

/* As cafs_sort; when `report` (host memory) is non-NULL the call waits for
 * the stream and fills *report with the estimate, the branch taken, the
 * number of distinct keys counted and the device status.  With report == NULL
 * it behaves exactly like cafs_sort. */
cafs_status cafs_sort_ex(const void* keys, size_t n, cafs_dtype dtype, void* out,
                         cafs_report* report, void* stream);

/* Stable argsort: the permutation pi of Sec. 3.1's problem statement,
 * x[pi[0]] <= x[pi[1]] <= ... <= x[pi[n-1]], with equal keys in input order.
 * keys: device pointer, n elements of dtype (not written).
 * out: device pointer, n elements: receives the sorted keys (the same result
 *   as cafs_sort).  perm: device pointer, n uint32_t: receives pi.
 * keys, out and perm must not overlap at all (CAFS_ERR_ALIAS); n <= 2^32-1.
 * The column takes the path cafs_sort would take (Alg. 3); on the count
 * paths each key's rank among the K' distinct keys is then sorted stably
 * with its input position (one LSD radix pass per byte of K'-1), on the
 * radix paths the (key, position) pairs are; a sorted column gives the
 * identity.  Asynchronous on `stream` unless `report` is non-NULL (then
 * blocking, as cafs_sort_ex).  The library keeps 16 bytes per key of extra
 * scratch for this call in the stream's workspace. */
cafs_status cafs_argsort(const void* keys, size_t n, cafs_dtype dtype, void* out, uint32_t* perm,
                         cafs_report* report, void* stream);

/* Sampler + Chao1 + dispatcher only (Alg. 2 and Alg. 3, Eq. 5-6): fills *est
 * (host memory).  Blocking: waits for `stream`.  The IsMonotone test of
 * Alg. 3 is a full scan on the device, run only when the samples ascend. */
cafs_status cafs_estimate_k(const void* keys, size_t n, cafs_dtype dtype,
                            cafs_estimate* est, void* stream);

/* End-to-end form for host buffers: copies n keys from host memory
 * `host_keys` to a library-owned device buffer, sorts them on the device and
 * copies the result to host memory `host_out` (which may equal host_keys).
 * Blocking.  Pinned host memory gives the fastest copies; pageable memory
 * works.  `report` may be NULL. */
cafs_status cafs_sort_host(const void* host_keys, size_t n, cafs_dtype dtype,
                           void* host_out, cafs_report* report, void* stream);

/* Allocation-free variant of cafs_sort (the paper has no counterpart).  For
 * callers that cannot allocate device memory: engines that hand out only
 * pre-reserved memory pools and forbid any other allocation, processes that
 * run under a fixed device-memory budget, and latency-critical loops where
 * the implicit device synchronisation of cudaMalloc/cudaFree is not
 * acceptable.  This call performs no cudaMalloc/cudaFree and calls no
 * allocating library routine.  Its scratch is one file-scope device array of
 * about 25 MiB that every GPU loading the library holds until the process
 * exits.  n must be <= 2^19 (524288) keys, else CAFS_ERR_TOO_LARGE; other
 * arguments as for cafs_sort.  The first call on a device resolves the
 * array's device address and sets kernel attributes, so make that first call
 * before any stream capture.  All calls share the array (it keeps the
 * previous call's contents; the control block and the hash table's used
 * slots are cleared by every call): calls whose work overlaps on the GPU --
 * other streams, other host threads -- race and must be serialised by the
 * caller.  No report: a device-side failure (a bounded wait that ran out)
 * is not reported by this call, and the output is then undefined. */
cafs_status cafs_sort_noalloc(const void* keys, size_t n, cafs_dtype dtype, void* out,
                              void* stream);

/* ---- Batched form (no counterpart in the paper) -----------------------------
 * Many columns sorted by one persistent cooperative launch per key type
 * present (int32 columns, then int64 columns), one CTA per SM.
 * Each column gets exactly the result, path and report that cafs_sort_ex
 * gives it alone.  Columns with n >= grid_min_n are sorted one after another
 * by all CTAs together; the others form a work queue, longest first, from
 * which each CTA takes whole columns and sorts each alone; radix-fallback
 * columns of the queue with n >= defer_min_n are set aside and sorted by all
 * CTAs at the end.  Columns are independent: no two columns of a batch may
 * overlap in memory (keys == out within one column is allowed). */
typedef struct {
  const void* keys;    /* device pointer, n elements                        */
  void* out;           /* device pointer, n elements; may equal keys        */
  size_t n;
  cafs_dtype dtype;    /* any key type; unsigned and float keys are mapped
                          into out before the launch and back after it      */
  int32_t reserved;    /* must be 0                                          */
} cafs_column;

/* Scheduling knobs of the batched kernel.  They change the speed, never a
 * result.  0 in any field selects the default (cafs_batch_tuning_default). */
typedef struct {
  uint64_t grid_min_n;      /* all-CTA columns: n >= this (>= 2048; 0: per
                               batch, max(2^16, 2 * total keys / CTAs))    */
  uint64_t defer_min_n;     /* set-aside radix columns: n >= this (0: per
                               batch, max(2^15, queue keys / (2 * CTAs)))   */
  uint64_t cta_table_slots; /* hash table of each per-CTA slot, slots: power
                               of two >= 64; a queue column whose Eq. 6
                               table is larger is set aside after sampling
                               and sorted by all CTAs (0: large enough for
                               the longest queue column, never sets aside) */
  uint32_t local_slots_max; /* per-CTA shared hash table cap, slots: power
                               of two in [256, 8192] (8192)                */
  uint32_t replicas_max;    /* counter replicas per shared slot: power of
                               two in [1, 32] (32)                         */
  uint32_t emit_tile_vec;   /* emit tile in 16-byte vectors: multiple of
                               1024, <= 8192 (4096)                        */
  uint32_t ctas;            /* CTAs of the launch (0: one per SM)           */
  uint32_t reserved;        /* must be 0                                    */
  uint32_t reserved2;
} cafs_batch_tuning;

cafs_status cafs_batch_tuning_default(cafs_batch_tuning* tuning);

/* Sorts ncols columns (host array `cols`) with one batched launch on
 * `stream`.  The library keeps a batch workspace per (device, stream), grown
 * on demand: per SM one slot (a 16-byte-per-slot hash table, its pair
 * arrays and a radix buffer for columns shorter than defer_min_n; about
 * 37 MB for a longest queue column of 2^20 keys, less with
 * cta_table_slots), plus one all-CTA slot sized like cafs_sort's workspace
 * for the longest column.  When `reports`
 * (host, ncols entries) is non-NULL the call waits and fills one report per
 * column; otherwise it returns after enqueueing.  Argument errors in any
 * column are returned before anything is enqueued. */
cafs_status cafs_sort_batch(const cafs_column* cols, size_t ncols, cafs_report* reports,
                            void* stream);
/* As cafs_sort_batch with explicit knobs (NULL = defaults). */
cafs_status cafs_sort_batch_tuned(const cafs_column* cols, size_t ncols,
                                  const cafs_batch_tuning* tuning, cafs_report* reports,
                                  void* stream);

/* A batch plan: the columns, a workspace of its own and a CUDA graph holding
 * the launch (and the memsets that zero its control words), recorded once on
 * the current device.  Every cafs_batch_plan_launch replays the graph on
 * `stream`, sorting the same column buffers again (refill them in place
 * between launches).  Launches of one plan must not overlap on the GPU.
 * cafs_batch_plan_reports waits for `stream` and fills ncols reports (host)
 * for the last launch. */
typedef struct cafs_batch_plan cafs_batch_plan;
cafs_status cafs_batch_plan_create(const cafs_column* cols, size_t ncols,
                                   const cafs_batch_tuning* tuning, cafs_batch_plan** plan);
cafs_status cafs_batch_plan_launch(cafs_batch_plan* plan, void* stream);
cafs_status cafs_batch_plan_reports(cafs_batch_plan* plan, cafs_report* reports, void* stream);
size_t cafs_batch_plan_columns(const cafs_batch_plan* plan);
void cafs_batch_plan_destroy(cafs_batch_plan* plan);

/* Autotuner measurement step: for each of the ncand knob settings, records a
 * plan over `cols`, launches it once to warm up and `reps` more times on
 * `stream` (CUDA events around each launch), and stores the median launch
 * time in ms[c]; *best = the index of the fastest.  The columns are sorted
 * (1 + reps) * ncand times; results never depend on the knobs.  Blocking. */
cafs_status cafs_batch_autotune(const cafs_column* cols, size_t ncols,
                                const cafs_batch_tuning* candidates, size_t ncand, int reps,
                                double* ms, size_t* best, void* stream);

/* ---- Served form (no counterpart in the paper) ------------------------------
 * A request server on the current device.  At creation it reserves its
 * whole device-memory budget once: the batched kernel's workspace for
 * max_batch_columns requests of up to max_request_keys keys, and an arena
 * for request buffers (the rest of the budget).  Requests (host buffers) are
 * admitted first come first served whenever their keys fit in the arena;
 * everything admitted while the previous launch runs is sorted by the next
 * batched launch (continuous batching).  A request's keys stay in one arena
 * buffer from the copy in to the copy out; the buffer is released when the
 * sorted keys are in host_out.  Server threads do the copies and launches;
 * all entry points are thread-safe. */
typedef struct {
  uint32_t max_batch_columns;  /* requests per batched launch (1024)        */
  uint32_t max_inflight;       /* batched launches in flight (3)            */
  uint64_t max_request_keys;   /* longest request accepted (2^22)           */
  cafs_batch_tuning tuning;    /* knobs of the batched kernel               */
  uint32_t reserved;           /* must be 0                                  */
  uint32_t reserved2;
} cafs_server_config;

typedef struct {
  uint64_t launches, completed, keys_done, pending;
  uint64_t arena_bytes, arena_peak_bytes, workspace_bytes;
} cafs_server_stats_t;

typedef struct cafs_server cafs_server;

cafs_status cafs_server_config_default(cafs_server_config* cfg);
/* cfg may be NULL (defaults).  CAFS_ERR_OUT_OF_MEMORY when the budget does
 * not cover the workspace plus a non-empty arena, or cannot be reserved. */
cafs_status cafs_server_create(size_t mem_budget_bytes, const cafs_server_config* cfg,
                               cafs_server** server);
/* Enqueues a request: n keys of `dtype` at host_keys, sorted keys to
 * host_out (may equal host_keys); both must stay valid until the matching
 * cafs_server_wait returns.  Pinned host memory gives the fastest copies.
 * n > max_request_keys (or larger than the arena): CAFS_ERR_TOO_LARGE. */
cafs_status cafs_server_submit(cafs_server* server, const void* host_keys, size_t n, cafs_dtype dtype,
                               void* host_out, uint64_t* ticket);
/* Blocks until the request is done; fills the report (may be NULL) and the
 * latency from submission to the result being in host_out (may be NULL). */
cafs_status cafs_server_wait(cafs_server* server, uint64_t ticket, cafs_report* report,
                             double* latency_us);
cafs_status cafs_server_stats(cafs_server* server, cafs_server_stats_t* stats);
void cafs_server_destroy(cafs_server* server);

/* One request of a replayed trace. */
typedef struct {
  const void* host_keys;
  void* host_out;
  size_t n;
  cafs_dtype dtype;
  int32_t reserved;            /* must be 0                                  */
} cafs_request;

/* Open-loop replay of a request trace against a server: request i is
 * submitted arrival_s[i] seconds (non-decreasing) after the call starts,
 * from a native thread that waits for each arrival time; latency_us[i] is
 * the time from that arrival time to the result being in host_out.
 * *elapsed_s (may be NULL) = first arrival to last completion.  reports may
 * be NULL. */
cafs_status cafs_server_run_trace(cafs_server* server, const cafs_request* reqs, size_t nreq,
                                  const double* arrival_s, double* latency_us, cafs_report* reports,
                                  double* elapsed_s);
/* The same trace served one request at a time with cafs_sort_host on
 * `stream` (the serial baseline of the served form). */
cafs_status cafs_serial_run_trace(const cafs_request* reqs, size_t nreq, const double* arrival_s,
                                  double* latency_us, cafs_report* reports, double* elapsed_s,
                                  void* stream);

/* Hash seed (randomised multipliers against adversarial keys; Eq. 4 fixes the golden-ratio
 * multiplier).  seed == 0 (the default): every table hash uses the
 * golden-ratio constants.  seed != 0: every later call (each sort, argsort,
 * batch launch or plan, server launch) draws its own odd 64-bit Eq. 4
 * multiplier and odd 32-bit shared-table multiplier from the seed and a
 * process-wide call counter (SplitMix64), so that no fixed key set collides
 * in every call.  Which slot a key lands in never changes a count, a result,
 * a path or a report field; only the speed of adversarial inputs changes.
 * Setting a seed restarts the call counter. */
void cafs_set_hash_seed(uint64_t seed);

/* Testing hooks (no counterpart in the paper).  `flags` bit 0 makes CTA 0 of
 * the next pipeline launches skip the first grid barrier, so that the other
 * CTAs' bounded wait runs out and the launch reports CAFS_ERR_TIMEOUT in
 * cafs_report.device_status; no GPU fault is involved.  `wait_timeout_ns`
 * bounds every device-side wait (0 restores the default of one second).
 * Pass flags = 0 to return to normal operation. */
void cafs_set_test_hooks(uint32_t flags, uint64_t wait_timeout_ns);

/* Number of kernels the library launched on the calling process so far
 * (all entry points, all devices).  Diagnostic counter. */
uint64_t cafs_kernel_launch_count(void);

/* Human-readable names; never NULL. */
const char* cafs_status_string(cafs_status s);
const char* cafs_path_string(cafs_path p);

#ifdef __cplusplus
}
#endif

#endif /* CAFS_H */
