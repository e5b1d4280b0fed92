/*
 * lcs.h — C ABI of the GB300 (sm_103a) LCS library (liblcs.so).
 *
 * The library fills the dynamic-programming table of the longest common subsequence (LCS) of two byte strings and
 * traces one LCS back, as defined in Dash & Nayak, "Parallel Algorithm for Longest Common Subsequence in a String":
 *
 *   c[i,0] = c[0,j] = 0;  c[i,j] = c[i-1,j-1] + 1 if x_i = y_j, else max(c[i-1,j], c[i,j-1])   (§I.B, §I.C)
 *
 * X = x_1..x_m indexes the rows and Y = y_1..y_n the columns; the LCS length is c[m,n] (§I.C, LCS-length). The
 * traced string is the one Print-LCS (§I.D) emits from b[m,n] when b takes the paper's tie-break: DIAG on every
 * match, otherwise UP when c[i-1,j] >= c[i,j-1] and LEFT when not. Symbols are bytes (0..255) compared for
 * equality; DNA over {A,C,G,T} (§I) is one case of that.
 *
 * Conventions for every call:
 *   - Return value: LCS_OK (0) or a negative LCS_ERR_* code; lcs_serve_poll may also return LCS_PENDING. No C++
 *     exception crosses this boundary.
 *   - Sizes are element counts (bytes for strings). A pointer may be NULL only when its size is 0.
 *   - Host pointers are ordinary (pageable or pinned) host memory. "_dev" calls take device pointers (for instance
 *     the data_ptr() of CUDA tensors) and a cudaStream_t passed as void* (NULL = the context's own stream); they
 *     return after enqueueing the work, which then runs in stream order.
 *   - The caller owns every buffer it passes; the library never keeps a caller pointer past the call (serving
 *     copies its inputs at submit).
 *   - A context serialises its own calls with an internal lock; use one context per host thread for concurrency.
 */
#ifndef LCS_H_
#define LCS_H_

#include <stdint.h>

#if defined(__GNUC__)
#define LCS_API __attribute__((visibility("default")))
#else
#define LCS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------------------------- */
#define LCS_OK 0
#define LCS_PENDING 1          /* lcs_serve_poll: the request is admitted or queued but not finished yet */
#define LCS_ERR_INVALID -1     /* bad argument: NULL with a nonzero size, m*n overflow, unknown ticket, ... */
#define LCS_ERR_NOMEM -2       /* device memory for the request could not be allocated (or can never fit) */
#define LCS_ERR_CAPACITY -3    /* output buffer too small; *out_len holds the required size */
#define LCS_ERR_BUSY -4        /* serving queue full (back-pressure); retry later */
#define LCS_ERR_TIMEOUT -5     /* a bounded device-side wait expired (the kernel returned instead of hanging) */
#define LCS_ERR_CUDA -6        /* a CUDA runtime call failed */
#define LCS_ERR_INTERNAL -7    /* an internal consistency check failed */

/* Human-readable text for a status code (static storage; never NULL). */
LCS_API const char* lcs_strerror(int status);

/* ---- context ------------------------------------------------------------------------------------------------ */
typedef struct lcs_ctx lcs_ctx;

/* Creates a context on CUDA device `device`: its own non-blocking stream and grow-only device scratch buffers.
 * *out receives the handle. Errors: LCS_ERR_INVALID (out NULL or no such device), LCS_ERR_CUDA. */
LCS_API int lcs_ctx_create(int device, lcs_ctx** out);

/* Waits for all work of the context and frees everything it owns. NULL is ignored. */
LCS_API void lcs_ctx_destroy(lcs_ctx* ctx);

/* Waits for the context's streams and returns (and clears) any error latched by an earlier "_dev" call's kernels
 * (LCS_ERR_TIMEOUT, LCS_ERR_INTERNAL) or LCS_OK. */
LCS_API int lcs_ctx_sync(lcs_ctx* ctx);

/* ---- stage timing ----------------------------------------------------------------------------------------------
 * The paper times its method with omp_get_wtime around the whole computation (§II.A, steps 6 and 21, EXEC_TIME).
 * Here every stage of the last length/traceback call is timed with CUDA events recorded on the call's stream. */
typedef struct lcs_profile {
  double prep_ms;        /* alphabet, match masks and per-row symbol offsets (per pair for lcs_batch) */
  double fill_ms;        /* the table fill kernel (all rows; both tables when the reversed strings run too);
                            for lcs_batch, the persistent batch kernel */
  double trace_ms;       /* corridors, segment walks, chain and output assembly (0 for length-only calls) */
  double total_ms;       /* first stage start to last stage end */
  uint64_t fill_blocks;  /* thread blocks of the fill launch */
  uint64_t cells;        /* m * n of the call */
} lcs_profile;

/* enable != 0 makes later calls record stage events (a few microseconds of overhead per call). */
LCS_API int lcs_ctx_set_profiling(lcs_ctx* ctx, int enable);

/* Waits for the last profiled call's events and fills *out. LCS_ERR_INVALID when profiling is off or no call was
 * profiled yet. */
LCS_API int lcs_ctx_last_profile(lcs_ctx* ctx, lcs_profile* out);

/* ---- fill configuration (no counterpart in the paper: how the table fill of §I.C is laid out on the GPU) -------- */

/* rows_per_step: rows of the table one systolic step of the fill covers (8 or 16); vg_select: 0 = the default
 * hand-off validation group of the fill's warps, 1 = the alternative (32 steps at 8 rows, 16 at 16 rows). Every
 * configuration gives the same results; only the time differs. mode 0 = length-only calls, 1 = traceback calls
 * (lcs_traceback*, lcs_tables*). */
typedef struct lcs_fill_config {
  uint32_t rows_per_step;
  uint32_t vg_select;
} lcs_fill_config;

LCS_API int lcs_ctx_get_fill_config(lcs_ctx* ctx, uint32_t mode, lcs_fill_config* out);
LCS_API int lcs_ctx_set_fill_config(lcs_ctx* ctx, uint32_t mode, const lcs_fill_config* cfg);

/* Autotuner: times every configuration on the device pair (d_x, m, d_y, n) in the given mode (one untimed and
 * three timed calls each, events on `stream`), keeps the fastest in the context for that mode and returns it in
 * *best with its median time in *best_ms (either may be NULL). Blocking. The caller may store the result and set
 * it on later contexts with lcs_ctx_set_fill_config. */
LCS_API int lcs_ctx_autotune_dev(lcs_ctx* ctx, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                                 uint32_t mode, void* stream, lcs_fill_config* best, double* best_ms);

/* ---- measurement probes (no counterpart in the paper: the ceilings the table fill is measured against) --------- */

/* INT32 throughput of the whole device for one instruction sequence, every SM full of independent chains.
 * mix 0: the row update of one 32-column word of the §I.C recurrence in bit-parallel form (U = V & P; the carry-in
 *        shift, S = V + U + carry and the carry collection; V' = S | (V & ~P)): 5 instructions;
 * mix 1: the same plus the traceback's direction word T = S ^ V ^ U: 6 instructions;
 * mix 2: one three-input logic operation.
 * iters: loop iterations per thread (each runs 4 chains); 200000 takes some tens of milliseconds. */
typedef struct lcs_int_rate {
  double ops_per_s;        /* instructions of the mix per second over the device (CUDA-event timed launch) */
  double ops_per_clk_sm;   /* per SM and SM clock cycle (cycles from clock64 in every block, the longest) */
  double sm_clock_mhz;     /* SM clock during the launch: cycles / event time */
  double kernel_ms;        /* event time of the timed launch */
  int32_t sms;             /* multiprocessors of the device (cudaDevAttrMultiProcessorCount) */
  int32_t blocks_per_sm;   /* resident blocks of 256 threads per SM */
  uint32_t ops_per_chain;  /* instructions per chain and iteration of the mix (5, 6 or 1) */
  uint32_t threads;        /* threads of the launch */
} lcs_int_rate;

/* Runs two launches on `device` (a warm-up, then the timed one) with buffers it allocates and frees. Blocking.
 * Errors: LCS_ERR_INVALID (out NULL, mix > 2, iters 0, no such device), LCS_ERR_CUDA. */
LCS_API int lcs_probe_int_rate(int device, uint32_t mix, uint32_t iters, lcs_int_rate* out);

/* The dependency floor of one systolic step of the table fill: clock cycles per step of rows_per_step (8 or 16)
 * rows when one warp per SM sub-partition runs only the fill's row arithmetic and its two carry shuffles per step
 * (match masks in registers; in traceback mode (traceback != 0) also the fill's two 16-byte bitmap stores per lane).
 * steps (1 .. 2^24) are timed with clock64 after 64 untimed ones; *cycles_per_step is the median of the 4 warps.
 * Multiplied by the fill's chain of steps (row-blocks + one step per 32-column word of the row) it bounds the time
 * of one pair's fill from below. Blocking. Errors: LCS_ERR_INVALID, LCS_ERR_CUDA. */
LCS_API int lcs_probe_step_floor(int device, uint32_t rows_per_step, int traceback, uint32_t steps,
                                 double* cycles_per_step);

/* The same 8-row traceback step with its match masks supplied four ways (alphabet of 4 symbols, so Y's codes have
 * two bit planes), to weigh the fill's shared-memory table against masks formed in registers:
 * source 0: the masks in registers (= lcs_probe_step_floor(device, 8, 1, ...));
 * source 1: the fill's way: each row's mask read from a shared table of every symbol's mask at the lane's word, at
 *           the row's symbol offset (offsets from a shared ring two steps ahead, masks one step ahead);
 * source 2: P = ~((pl0 ^ s0) | (pl1 ^ s1)) from the lane's two bit planes pl0, pl1 of Y's codes, s0 / s1 all ones
 *           where the row's code bit is set, each made by one byte permute from codes stored as byte sign bits (one
 *           16-byte shared load per step);
 * source 3: the same formula with s0 / s1 of every row stored expanded (four 16-byte shared loads per step).
 * steps (1 .. 2^24); *cycles_per_step is the median of the 4 warps. Blocking.
 * Errors: LCS_ERR_INVALID (source > 3, steps out of range, NULL output, no such device), LCS_ERR_CUDA. */
LCS_API int lcs_probe_step_masks(int device, uint32_t source, uint32_t steps, double* cycles_per_step);

/* ---- length (paper §I.C, LCS-length; returns c[m,n]) --------------------------------------------------------- */

/* Repeated calls (lcs_length*, lcs_traceback*): a call that repeats the previous call on the context with the same
 * arguments (the same buffers, sizes and outputs; host-buffer calls of one shape stage into the context's own
 * buffers, so they repeat too) is captured once as a CUDA graph, on its second occurrence, and replayed with one
 * launch from then on, instead of eight launches. The graph reads the buffers' contents when it runs. The capture
 * costs one extra host step once per new set of arguments; LCS_NO_PAIR_GRAPH=1 in the environment at context
 * creation turns it off. Pairs of the one-launch small path (see lcs_traceback) are never captured. With stage
 * timing on (lcs_ctx_set_profiling), the graph records the stage events too, so replayed calls are profiled. */

/* Host buffers x[0..m), y[0..n); writes c[m,n] to *out_len. Blocking. m = 0 or n = 0 gives 0. Errors:
 * LCS_ERR_INVALID (NULL with nonzero size, out_len NULL), LCS_ERR_NOMEM, LCS_ERR_CUDA, LCS_ERR_TIMEOUT. */
LCS_API int lcs_length(lcs_ctx* ctx, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint64_t* out_len);

/* Device buffers; writes c[m,n] to the device word *d_out_len in stream order. Asynchronous; kernel-side errors
 * are latched and reported by lcs_ctx_sync. */
LCS_API int lcs_length_dev(lcs_ctx* ctx, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                   uint64_t* d_out_len, void* stream);

/* LCS length of two device strings without allocating any device memory. This entry point is an addition of the
 * library; the paper has no counterpart. It is meant for callers that must not allocate device memory: code that
 * runs inside a framework owning the whole device-memory pool or a fixed memory budget (an allocation there would
 * fragment the pool or exceed the budget), and latency-critical loops, where cudaMalloc/cudaFree would synchronise
 * the device and stall work on other streams.
 *   - Limit: m, n <= 65536; larger sizes are rejected with LCS_ERR_INVALID.
 *   - Scratch: a 6.5 MiB array that the library reserves statically in device memory. Every GPU that loads the
 *     library holds it until the process exits. The first call on a device, made with that device current, looks up
 *     the array's device address (a runtime query).
 *   - The array is shared by all calls on a device and keeps the last call's contents (each call clears what must
 *     start at zero). Calls that overlapped on the GPU would race on it; this entry point therefore serialises its
 *     calls per device and waits for each one.
 *   - d_x, d_y and d_out_len are device pointers owned by the caller. The work is enqueued on `stream` (NULL = the
 *     default stream); the call returns after the stream has finished it, with c[m,n] in *d_out_len on LCS_OK. It
 *     also waits for its own work when it fails part way, so a failed call leaves nothing running on the array.
 *   - The call never falls back to allocating: the per-call buffers are fixed parts of the array, and a request that
 *     did not fit one of them fails with LCS_ERR_INTERNAL.
 *   - Errors: LCS_ERR_INVALID, LCS_ERR_CUDA, LCS_ERR_TIMEOUT, LCS_ERR_INTERNAL. */
LCS_API int lcs_length_noalloc(const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n, uint64_t* d_out_len,
                               void* stream);

/* ---- traceback (paper §I.C LCS-length with table b, then §I.D Print-LCS) -------------------------------------- */

/* Host buffers. Writes the LCS (forward order) to out[0..len) and len to *out_len. out_cap >= min(m, n) is always
 * enough; a smaller out_cap that cannot hold the result gives LCS_ERR_CAPACITY with *out_len = the LCS length.
 * Device memory of about m*n/8 bytes (a 1-bit-per-cell direction bitmap) is needed: LCS_ERR_NOMEM when it
 * cannot be allocated. Blocking. (Pairs with m <= 1024 and n <= 992, for lcs_length* as well, run as one launch
 * with the bitmap in on-chip memory; the results are the same.) */
LCS_API int lcs_traceback(lcs_ctx* ctx, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint8_t* out,
                  uint64_t out_cap, uint64_t* out_len);

/* Device buffers: d_out (capacity out_cap >= min(m, n), else LCS_ERR_CAPACITY at the call) receives the LCS and
 * the device word *d_out_len its length. Asynchronous in `stream`. */
LCS_API int lcs_traceback_dev(lcs_ctx* ctx, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                      uint8_t* d_out, uint64_t out_cap, uint64_t* d_out_len, void* stream);

/* ---- full tables (paper §I.C: LCS-length returns the tables c and b) ------------------------------------------ */

/* c[i][j] = length of an LCS of X[1..i] and Y[1..j] for 0 <= i <= m, 0 <= j <= n, written row-major to
 * c[i * (n + 1) + j] ((m + 1) * (n + 1) uint32 values). b[i-1][j-1] for 1 <= i <= m, 1 <= j <= n is the paper's
 * arrow, written row-major to b[(i - 1) * n + (j - 1)] (m * n bytes): 1 = diagonal (x_i = y_j), 2 = up
 * (c[i-1][j] >= c[i][j-1]), 3 = left. b may be NULL when m * n = 0. Meant for inspection of small and medium
 * problems: the device holds both tables plus an m*n/8-byte direction bitmap (LCS_ERR_NOMEM when that does not
 * fit). Host buffers, blocking. */
LCS_API int lcs_tables(lcs_ctx* ctx, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint32_t* c,
                       uint8_t* b);

/* The same into device buffers d_c and d_b, asynchronous in `stream` (NULL: the context's stream). */
LCS_API int lcs_tables_dev(lcs_ctx* ctx, const uint8_t* d_x, uint64_t m, const uint8_t* d_y, uint64_t n,
                           uint32_t* d_c, uint8_t* d_b, void* stream);

/* ---- batch: many independent pairs, lengths only (c[m_k, n_k] for every pair k) ------------------------------- */

/* Pair k is x = xs[x_off[k] .. x_off[k+1]) and y = ys[y_off[k] .. y_off[k+1]) (count+1 offsets each, non-
 * decreasing, host memory). out_lens[k] receives its LCS length. Blocking. When both string ranges are page-locked
 * host memory mapped for the device (cudaMallocHost / cudaHostAlloc / cudaHostRegister), the kernels read them in
 * place over the host link and nothing is copied into device buffers first; pageable strings are copied (small
 * batches through a page-locked staging area of the context). Errors: LCS_ERR_INVALID (bad offsets),
 * LCS_ERR_NOMEM, LCS_ERR_CUDA, LCS_ERR_TIMEOUT. */
LCS_API int lcs_batch(lcs_ctx* ctx, const uint8_t* xs, const uint64_t* x_off, const uint8_t* ys, const uint64_t* y_off,
              uint64_t count, uint64_t* out_lens);

/* The same with device buffers (offsets too); asynchronous in `stream`. The batch is planned on the host, so the
 * call copies the offsets back and waits for `stream` to reach that copy before it enqueues the batch. */
LCS_API int lcs_batch_dev(lcs_ctx* ctx, const uint8_t* d_xs, const uint64_t* d_x_off, const uint8_t* d_ys,
                  const uint64_t* d_y_off, uint64_t count, uint64_t* d_out_lens, void* stream);

/* The same with the strings and lengths in device memory and the offsets x_off / y_off (count+1 each) in host
 * memory, as a caller that assembled the batch holds them: no copy back and no wait; the call returns once the
 * batch is enqueued in `stream` (the offsets are read before it returns). Errors as lcs_batch, except that a
 * device-side timeout is latched and reported by lcs_ctx_sync, as for the other asynchronous calls. */
LCS_API int lcs_batch_dev_hoff(lcs_ctx* ctx, const uint8_t* d_xs, const uint64_t* x_off, const uint8_t* d_ys,
                               const uint64_t* y_off, uint64_t count, uint64_t* d_out_lens, void* stream);

/* Batch configuration (no counterpart in the paper: how the batched fill of §I.C is laid out on the GPU). The rows
 * of a pair are worked by a group of lanes of one warp, each lane holding consecutive 32-column words of the row.
 *   words_per_lane: 2, 4 or 8 words per lane (a pair whose row does not fit 32 lanes at that width uses the next
 *                   larger; pairs with more than 4096 columns go through the single-pair path). Default 4.
 *   split_pct:      job height. A pair whose rows exceed split_pct % of the average rows per resident warp (and at
 *                   least 256) runs as two half-height jobs, the bottom half on the reversed strings, joined at the
 *                   middle row. 0 = never split. Default 100.
 *   blocks_per_sm:  resident blocks (8 warps each) of the persistent kernel per SM, 1 or 2; capped by shared memory
 *                   (a batch with 8 words per lane runs one). Default 1.
 *   reserved:       0.
 * Every configuration gives the same lengths; only the time differs. A new configuration takes effect at the next
 * lcs_batch* call (the cached plan of the last batch is dropped). */
typedef struct lcs_batch_config {
  uint32_t words_per_lane;
  uint32_t split_pct;
  uint32_t blocks_per_sm;
  uint32_t reserved;
} lcs_batch_config;

LCS_API int lcs_ctx_get_batch_config(lcs_ctx* ctx, lcs_batch_config* out);
/* LCS_ERR_INVALID when a field is out of range (words_per_lane not 2/4/8, split_pct > 1000, blocks_per_sm not 1/2,
 * reserved not 0). */
LCS_API int lcs_ctx_set_batch_config(lcs_ctx* ctx, const lcs_batch_config* cfg);

/* Batch autotuner: runs the batch given as for lcs_batch_dev (device buffers and offsets, d_out_lens receives the
 * lengths) under every configuration (words per lane 2/4/8 x split_pct 50/100/200/never x blocks per SM 1/2): a
 * planning call and a graph-capturing call, then three timed replays each (events on `stream`); keeps the
 * configuration with the fastest median in the context and returns it
 * in *best with its median time in *best_ms (either may be NULL). Blocking. Every configuration's lengths are
 * compared with the first one's; a difference returns LCS_ERR_INTERNAL and keeps the previous configuration. */
LCS_API int lcs_ctx_autotune_batch_dev(lcs_ctx* ctx, const uint8_t* d_xs, const uint64_t* d_x_off, const uint8_t* d_ys,
                                       const uint64_t* d_y_off, uint64_t count, uint64_t* d_out_lens, void* stream,
                                       lcs_batch_config* best, double* best_ms);

/* ---- serving: continuous batching of requests that arrive over time ------------------------------------------- */
typedef struct lcs_server lcs_server;

#define LCS_TRACEBACK 1u /* submit flag: also return the LCS string (else length only) */

typedef struct lcs_serve_cfg {
  uint32_t max_queue;          /* requests waiting or in flight before submit returns LCS_ERR_BUSY (0 = 65536) */
  uint32_t max_batch;          /* short pairs packed into one batched launch (0 = 4096); a wave also holds at most
                                  8 MiB of X and 2 MiB of Y symbols */
  uint64_t hbm_budget_bytes;   /* device bytes of the arena that holds the direction bitmaps of the tracebacks in
                                  flight, allocated at creation (0 = one 65536 x 65536 bitmap per pair worker, at
                                  most 60% of free memory). A traceback waits until its bitmap fits the arena */
  uint32_t long_pair_cells_log2; /* length-only pairs with m*n >= 2^this, or whose shorter side exceeds 4096 or
                                    longer side 16384, run on the single-pair path (0 = 2^24) */
  uint32_t pair_workers;       /* single-pair workers, each with its own stream and buffers (0 = 16, at most 32) */
} lcs_serve_cfg;

typedef struct lcs_result {
  int32_t status;              /* LCS_OK or the request's error code */
  uint32_t flags;              /* the submit flags */
  uint64_t length;             /* c[m,n] */
  const uint8_t* lcs;          /* traceback string (server-owned until lcs_result_release), NULL if none */
  uint64_t lcs_len;            /* bytes at lcs */
  double submit_to_done_s;     /* latency measured by the server: submit() to result ready */
} lcs_result;

/* Creates a server on ctx (the server then owns the context's streams until lcs_serve_destroy; do not call other
 * functions on ctx meanwhile). cfg may be NULL for defaults. Every device buffer the server uses is allocated here
 * (the workers' buffers for pairs of up to 65536 x 65536 and the bitmap arena), so that serving requests of those
 * sizes allocates no device memory. The workers (2 batch workers plus pair_workers) each run their own stream: give
 * the process at least that many hardware work queues by setting the environment variable
 * CUDA_DEVICE_MAX_CONNECTIONS (e.g. to 32) before its first CUDA call; with the runtime's default of 8, workers
 * share queues and wait on each other's kernels. Errors: LCS_ERR_NOMEM, LCS_ERR_CUDA, LCS_ERR_INVALID. */
LCS_API int lcs_serve_create(lcs_ctx* ctx, const lcs_serve_cfg* cfg, lcs_server** out);

/* Copies x and y and queues the request; *ticket identifies it. Errors: LCS_ERR_BUSY (queue full),
 * LCS_ERR_NOMEM (a traceback whose bitmap can never fit the budget), LCS_ERR_INVALID. */
LCS_API int lcs_serve_submit(lcs_server* srv, const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint32_t flags,
                     uint64_t* ticket);

/* Non-blocking: LCS_OK and *out filled when the request is done, LCS_PENDING while it is not, LCS_ERR_INVALID for
 * an unknown or released ticket. */
LCS_API int lcs_serve_poll(lcs_server* srv, uint64_t ticket, lcs_result* out);

/* Blocking variant of lcs_serve_poll with a timeout in seconds (< 0 waits forever); LCS_PENDING on timeout. */
LCS_API int lcs_serve_wait(lcs_server* srv, uint64_t ticket, double timeout_s, lcs_result* out);

/* Frees a finished request's result (its lcs string pointer becomes invalid). */
LCS_API void lcs_result_release(lcs_server* srv, uint64_t ticket);

/* Finishes in-flight work, frees all results and stops the scheduler thread. NULL is ignored. */
LCS_API void lcs_serve_destroy(lcs_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* LCS_H_ */
