/* rtg.h - C ABI of the GB300 library for all-pairs r-nearest-neighbour reporting with
 * randomly transformed grids (RTG).
 *
 * Method (Kleinbort, Salzman, Halperin, arXiv:1409.8112):
 *   Problem (Sec. I): given n points P in R^d and a radius r, report every pair {p, q} of P
 *   at Euclidean distance at most r.
 *   Alg. 1 (Sec. III): repeat m times: place a grid of cell side c under a random shift
 *   (and, in the second algorithm of Sec. III, a random rotation), associate every point
 *   with the cell it lies in, and report the pairs inside each non-empty cell that are at
 *   distance at most r.  Pairs found by several grids are reported once (Sec. III-B).
 *
 * Exact arithmetic contract (what makes the output a unique integer set):
 *   grid t is the row-major d x d matrix R_t followed by the shift s_t (m*(d*d+d) doubles);
 *   rotated coordinate  y_k = fma-chain: acc = s_k; acc = fma(R_t[k][l], p_l, acc), l=0..d-1
 *   cell coordinate     q_k = floor(y_k / c)          (IEEE double division)
 *   squared distance    s = 0; e = p_a[l] - p_b[l]; s = fma(e, e, s), l = 0..d-1, on the
 *                       original (unrotated) coordinates; FP32 input is widened exactly
 *   reported            s <= fl(r * r)
 * The library reaches this FP64 result bit for bit while doing its bulk arithmetic in
 * FP32: every decision whose FP32 value lies within a proven error bound of the boundary
 * is recomputed in FP64 with the sequence above.
 *
 * Output: the upper-triangular CSR of the reported set: row i lists every j > i with
 * {i, j} reported, ascending.  With RTG_FLAG_SYMMETRIC both (i, j) and (j, i) are stored
 * (the "store each pair twice" extension of Sec. III-B for multiple r-NN queries).
 *
 * Errors: every entry point returns an rtg_status; nothing is thrown across the ABI.
 * rtg_last_error() gives a text for the last failure on a context.  One context serialises
 * its synchronous calls on its own stream; distinct contexts are independent.
 *
 * Environment, read when a context is created (none changes a result):
 *   RTG_TUNE_CACHE=path       JSON file that keeps the autotuner's sort choices per device
 *   RTG_AUTOTUNE=0            take the default sort variant and enumeration knobs
 *   RTG_SORT_VARIANT=b,i,m    force a sort variant: digit bits, keys per thread, strategy
 *                             (0 look-back, 1 reduce-then-scan, 2 one cooperative launch)
 *   RTG_TUNE_PAIRS_MAX_CAND=x in-cell candidates above which the enumeration keeps its
 *                             default knobs (4e9)
 *   RTG_GRAPHS=0              launch every kernel directly instead of replaying CUDA graphs
 *   RTG_CELL_MAJOR=0          keep the grid in every sort key (no cell-major sort)
 *   RTG_SERVE_LANES=k         concurrent server lanes (1 to 8, default 2)
 *   RTG_SERVE_LOG=1           one line per served batch on stderr
 */
#ifndef RTG_H
#define RTG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RTG_OK = 0,
  RTG_E_INVALID = 1,        /* bad argument (sizes, non-finite values, null pointers) */
  RTG_E_NOMEM = 2,          /* device allocation failed */
  RTG_E_BUDGET = 3,         /* the request does not fit the context's memory budget */
  RTG_E_KEY_OVERFLOW = 4,   /* a grid's cell index range needs more than 64 key bits */
  RTG_E_CUDA = 5,           /* a CUDA call failed; see rtg_last_error */
  RTG_E_TIMEOUT = 6,        /* a bounded device or host wait ran out */
  RTG_PENDING = 7,          /* rtg_poll: the build is not finished yet */
  RTG_E_UNKNOWN_TICKET = 8, /* rtg_poll/rtg_wait: no such ticket */
  RTG_E_INTERNAL = 9        /* a device-side consistency check failed */
} rtg_status;

/* Flags. */
#define RTG_FLAG_SHIFT_ONLY 1u /* rtg_transforms_generate: R = identity (Alg. 1 as printed) */
#define RTG_FLAG_SYMMETRIC 2u  /* rtg_all_pairs: store (i,j) and (j,i) */
#define RTG_FLAG_TIMING 4u     /* rtg_all_pairs: fill rtg_stats.phase_us (adds events) */
#define RTG_FLAG_TWO_PASS 8u   /* enumerate twice (count, then write in place) instead of
                                  holding a pair buffer: less memory, more time */
#define RTG_FLAG_TC_FP16 16u   /* rtg_brute_force: distances from FP16 tensor-core tiles;
                                  rtg_all_pairs / rtg_batch_all_pairs: cells of more than 256
                                  points are filtered by FP16 tensor-core tiles (pairs the tile
                                  proves beyond r are dropped, every other pair is decided as
                                  without the flag: the same set) */
#define RTG_FLAG_TC_BF16 32u   /* as RTG_FLAG_TC_FP16 with BF16 tiles */
#define RTG_FLAG_BITSET 64u    /* small instances (n <= 16384 each): dedupe through an n x n
                                  bit matrix per instance (the flattened bit array of
                                  Sec. III-B) instead of the first-grid rule; same output */

/* Point coordinate types. */
#define RTG_DTYPE_F64 0
#define RTG_DTYPE_F32 1

#define RTG_MAX_DIM 16   /* d in [1, RTG_MAX_DIM] */
#define RTG_MAX_GRIDS 64 /* m in [1, RTG_MAX_GRIDS] */

typedef struct rtg_ctx rtg_ctx;

typedef struct {
  int device;                /* CUDA device ordinal */
  uint64_t mem_budget_bytes; /* cap on device memory the context may hold; 0 = no cap */
  void* stream;              /* cudaStream_t to run on, or NULL for a private stream */
  uint32_t flags;            /* reserved, pass 0 */
} rtg_config;

/* Per-build counters (all exact integers unless noted). */
typedef struct {
  int64_t candidates[RTG_MAX_GRIDS]; /* grid t: sum over non-empty cells of C(size, 2) */
  int64_t total_candidates;          /* sum of the above */
  int64_t owned_candidates;          /* candidates not beyond r by the FP32 test whose pair
                                        first shares a cell in their grid t */
  int64_t near_wall;     /* (point, grid) pairs with a coordinate within 1e-12 of a wall */
  int64_t near_r;        /* distinct co-located pairs with |dist - r| <= 1e-12 r */
  int64_t key_rechecks;  /* coordinates whose cell index was recomputed in FP64 */
  int64_t dist_rechecks; /* pairs whose distance test was recomputed in FP64 */
  int64_t large_cells;   /* cells handled by the tiled large-cell path */
  int64_t max_cell;      /* largest cell population over all grids */
  int64_t pairs;         /* unique reported pairs (= upper-triangular nnz) */
  int32_t key_bits;      /* bits of the (grid, cell) sort key */
  int32_t sort_passes;   /* radix passes run */
  int32_t launches;      /* kernels this build launched */
  int32_t attempts;      /* 1, or more when a launch assumption had to be corrected */
  int32_t sort_digit_bits; /* radix digit width used (8, 9, 10 or 11; autotuned per shape) */
  int32_t sort_tile_keys;  /* keys per sort tile (2048, 3072 or 4096; autotuned) */
  int32_t sort_lookback;   /* 1: single-kernel look-back passes, 0: reduce-then-scan,
                              2: every pass in one cooperative launch */
  int32_t sort_tuned;      /* 1 when the sort variant was measured on this device */
  double phase_us[8];    /* with RTG_FLAG_TIMING: prep+plan, keys, sort, pairs, scan,
                            scatter (or write), rowsort, total (microseconds, device events) */
  double max_abs_err_d2; /* tensor-core brute force: max |tile d^2 - FP64 d^2| over the pairs
                            the tiles did not reject */
  double band;           /* tensor-core brute force: half-width of the FP64 band around r^2 */
  int64_t phase_bytes[8]; /* device-memory bytes each phase must read and write by its design
                             (the phases of phase_us; [7] is their sum): the points, FP32 rows,
                             key rows, every sort pass's keys and indices, the gathered rows,
                             the emitted pairs, row counts and the CSR.  Cache hits and
                             re-reads are not counted */
  int64_t bytes_moved;    /* = phase_bytes[7] */
  int32_t pairs_spans_per_warp; /* in-cell enumeration: sorted-position spans per resident
                                   warp (autotuned per shape) */
  int32_t dense_cell_min;       /* cells of more points than this take the tiled kernels
                                   (autotuned per shape: 64, 128 or 256) */
  int32_t pairs_tuned;          /* 1 when the two above were measured on this device */
  int64_t mem_estimate;         /* served results: the admission estimate of their batch */
  int64_t mem_peak;             /* served results: device bytes their batch needed (the
                                   workspace its build asked for and its block CSR) */
  int32_t sort_cell_major;      /* 1 when the sort key was the cell index alone (one
                                   instance, where that saves a radix pass): the sort then
                                   orders (cell, grid, point) instead of (grid, cell, point);
                                   the reported pairs are the same */
  int32_t sort_key_bits;        /* bits the sort ordered: key_bits, or the cell index's when
                                   sort_cell_major is 1 */
} rtg_stats;

typedef struct {
  int64_t n;         /* number of points (rows) */
  int64_t nnz;       /* stored entries: pairs, or 2 * pairs when symmetric */
  int64_t* row_ptr;  /* device pointer, n + 1 entries */
  int32_t* col;      /* device pointer, nnz entries, ascending within each row */
  int32_t symmetric; /* 1 if both (i,j) and (j,i) are stored */
  uint64_t handle;   /* library bookkeeping; 0 = empty */
  rtg_stats stats;
} rtg_csr;

/* One roadmap of a batch. */
typedef struct {
  const void* points;        /* n x d row-major (host or device, as the call says) */
  int64_t n;
  int d;                     /* in [1, 16] */
  double r;                  /* reporting radius */
  double cell_side;          /* grid cell side c */
  const double* transforms;  /* host, m*(d*d+d) doubles (R_t row-major, then s_t) */
} rtg_instance;

/* One roadmap build request for the server (rtg_submit). */
typedef struct {
  const void* points;        /* host, n x d row-major; copied by rtg_submit */
  int dtype;                 /* RTG_DTYPE_F64 or RTG_DTYPE_F32 */
  int64_t n;
  int d;                     /* in [1, 16] */
  double r;
  double cell_side;
  const double* transforms;  /* host, m*(d*d+d) doubles; copied by rtg_submit */
  int m;                     /* in [1, 64] */
  uint32_t flags;            /* RTG_FLAG_SYMMETRIC */
} rtg_request;

/* Create a context on cfg->device.  *out receives the context or NULL on failure. */
rtg_status rtg_create(const rtg_config* cfg, rtg_ctx** out);

/* Destroy a context; releases every CSR it still owns.  NULL is allowed. */
void rtg_destroy(rtg_ctx* ctx);

/* Text for the last failure on ctx (or for context-less calls if ctx is NULL).  Valid until
 * the next call on that context. */
const char* rtg_last_error(const rtg_ctx* ctx);

/* The CUDA stream (cudaStream_t) every device operation of ctx is ordered on: the one given
 * in rtg_config, or the context's own.  Callers whose device inputs are produced on another
 * stream make this stream wait for it (an event) instead of synchronising the host.  NULL for
 * a NULL ctx. */
void* rtg_get_stream(const rtg_ctx* ctx);

/* Name of a status code. */
const char* rtg_status_string(rtg_status s);

/* Draw m grid transforms for Alg. 1 / its rotated variant (Sec. III): R_t Haar-distributed
 * on O(d) (QR of a seeded standard Gaussian matrix with diag(R) made positive; identity
 * with RTG_FLAG_SHIFT_ONLY) and s_t uniform in [0, cell_side)^d.  out (host) receives
 * m*(d*d+d) doubles, R_t row-major then s_t.  Deterministic in (seed, d, m, cell_side,
 * flags).  RTG_E_INVALID for d outside [1,16], m < 1, cell_side <= 0 or out == NULL. */
rtg_status rtg_transforms_generate(uint64_t seed, int d, int m, double cell_side,
                                   uint32_t flags, double* out);

/* Alg. 1 (Sec. III) over all m grids, with the pairs merged and deduplicated into a CSR
 * (Sec. III-B).  Synchronous: returns when the CSR is complete on the device.
 *   points     n x d row-major, dtype RTG_DTYPE_F64 or RTG_DTYPE_F32; a device pointer if
 *              points_on_device, else a host pointer (copied in).  Caller-owned, read-only.
 *   r          reporting radius (> 0, finite)
 *   transforms host pointer, m*(d*d+d) doubles as produced by rtg_transforms_generate
 *   cell_side  grid cell side c (> 0, finite); the paper takes c = c~ r with c~ > 1
 *   flags      RTG_FLAG_SYMMETRIC, RTG_FLAG_TIMING, RTG_FLAG_TWO_PASS, RTG_FLAG_BITSET,
 *              RTG_FLAG_TC_FP16 or RTG_FLAG_TC_BF16 (dense cells on tensor-core tiles)
 *   out        receives a library-owned device CSR; free it with rtg_release
 * Errors: RTG_E_INVALID (n < 0 or n >= 2^31, n * m >= 2^31, d outside [1,16], m outside
 * [1,64], r or c not positive and finite, a non-finite coordinate or transform entry),
 * RTG_E_KEY_OVERFLOW, RTG_E_BUDGET, RTG_E_NOMEM, RTG_E_CUDA, RTG_E_TIMEOUT.  n in {0, 1}
 * gives an empty CSR.
 * Limits beyond the paper's problem statement: n * m < 2^31, because every (point, grid)
 * element of the sort has a 32-bit position; and the composite sort key spends, besides the
 * mixed-radix cell key of each grid, log2 of the number of (instance, grid) blocks on a base
 * that keeps the grids (and instances of a batch) apart, so RTG_E_KEY_OVERFLOW comes when the
 * sum over grids of the cell-key ranges exceeds 2^64, not when one grid's range does.
 * FP64 coordinates beyond the FP32 range are accepted: the FP32 filters cannot bound them,
 * so the cell indices and distances whose error bounds they enter are decided in FP64
 * (slower, same set). */
rtg_status rtg_all_pairs(rtg_ctx* ctx, const void* points, int dtype, int points_on_device,
                         int64_t n, int d, double r, const double* transforms, int m,
                         double cell_side, uint32_t flags, rtg_csr* out);

/* Alg. 1 (Sec. III) for a batch of independent roadmaps in one build (one sequence of kernel
 * launches for all of them): every instance has its own points, n, d, r, cell side and m
 * transforms (m, dtype and points_on_device are common).  out receives the block-diagonal
 * CSR over the concatenated points: instance b owns rows and columns
 * [row_offsets[b], row_offsets[b+1]), and its block is exactly what rtg_all_pairs returns
 * for it alone, shifted by row_offsets[b].  row_offsets (host, count + 1 entries) may be
 * NULL.  Errors as rtg_all_pairs; RTG_E_INVALID also for count outside [1, 65535] or
 * sum(n) * m >= 2^31. */
rtg_status rtg_batch_all_pairs(rtg_ctx* ctx, const rtg_instance* items, int count, int m,
                               int dtype, int points_on_device, uint32_t flags, rtg_csr* out,
                               int64_t* row_offsets);

/* The exact all-pairs r-NN set of Sec. I (every pair {i, j} with s <= fl(r * r), s as in
 * the arithmetic contract above) by checking all n(n-1)/2 pairs on the device in tiles; the
 * recall denominator for Alg. 1 and an exact reference.  Same argument conventions and
 * errors as rtg_all_pairs (no transforms).  With count_only != 0 only out->nnz and
 * out->stats.pairs are set (no device memory is returned beyond the row pointers).
 * With RTG_FLAG_TC_FP16 or RTG_FLAG_TC_BF16 the distances come from tensor-core tiles
 * (|x|^2 + |y|^2 - 2 x.y, x.y as hi.hi + hi.lo + lo.hi of a half-precision split of the
 * centred coordinates, FP32 accumulation); a pair is rejected on the tile only when its d^2
 * exceeds r^2 + band, band = max(1e-3 r^2, proven error bound), and every other pair is
 * decided with the FP64 sequence, so the set is unchanged.  stats.band and
 * stats.max_abs_err_d2 report the band and the largest observed tile error. */
rtg_status rtg_brute_force(rtg_ctx* ctx, const void* points, int dtype, int points_on_device,
                           int64_t n, int d, double r, uint32_t flags, int count_only,
                           rtg_csr* out);

/* Exact pair count without any device allocation.  The paper has no counterpart: this is for
 * callers that cannot allocate device memory, such as a planner's control loop that runs
 * under a fixed memory plan or a latency budget, or a plug-in inside a host application that
 * owns every device allocation (rtg_create itself allocates, so such callers have no
 * context).  It counts the pairs {i, j} with s <= fl(r * r) (the same set and arithmetic as
 * rtg_brute_force) and writes the count to *count (host).
 *   points  device pointer, n x d row-major, dtype RTG_DTYPE_F64 or RTG_DTYPE_F32, n <= 65536
 *   stream  cudaStream_t to run on (NULL = legacy default stream); the call synchronises it
 * Scratch: one file-scope device array of about 4.4 MiB (status counters, plan, FP32 rows of
 * up to 65536 points with d <= 16, row counts), held by every GPU that loads the library
 * until the process exits.  The first call on a device, with that device current, looks up
 * the array's device address; that first call must come before any stream capture.  Every
 * call synchronises `stream` and copies the count back to host memory before it returns, so
 * no call can be made inside a stream capture (RTG_E_INVALID when `stream` is capturing).
 * Every call on a device shares the array and leaves its contents behind: calls that overlap
 * on the GPU (from different streams or threads) race and give undefined counts.  Nothing
 * here calls cudaMalloc, cudaFree or an allocating library routine.
 * Errors: RTG_E_INVALID (n > 65536, d outside [1,16], r not positive and finite, NULL
 * pointers, a non-finite coordinate, a capturing stream), RTG_E_CUDA, RTG_E_TIMEOUT; text via
 * rtg_last_error(NULL). */
rtg_status rtg_brute_count_noalloc(const void* points, int dtype, int64_t n, int d, double r,
                                   void* stream, uint64_t* count);

/* Serving: continuous batching of builds (Alg. 1 per request).  rtg_submit copies the
 * request's points and transforms and returns at once with a ticket; a server owned by the
 * context (started by the first submit) forms batches of waiting requests that share m,
 * dtype and flags, runs them on several streams concurrently, and hands each request its own
 * device CSR, bit-identical to what rtg_all_pairs returns for it alone.  Admission follows the
 * context's mem_budget_bytes: a batch starts only when its estimated footprint fits next to
 * the memory already held (results not yet released included); the oldest request goes first;
 * a request that cannot fit even alone fails with RTG_E_BUDGET.  Thread safe: submit, poll and
 * wait may be called from any thread.  The number of concurrent lanes is 2 (environment
 * variable RTG_SERVE_LANES, 1 to 8).
 * The result's stats describe the batch it ran in, except phase_us[0] (microseconds queued)
 * and phase_us[7] (microseconds from submit to completion).
 * Errors of rtg_submit: as rtg_all_pairs for invalid requests. */
rtg_status rtg_submit(rtg_ctx* ctx, const rtg_request* req, uint64_t* ticket);

/* RTG_PENDING while the request runs; otherwise its final status, and on RTG_OK *out holds its
 * CSR (free it with rtg_release).  A ticket is forgotten once a final status is returned;
 * RTG_E_UNKNOWN_TICKET for tickets never issued or already taken. */
rtg_status rtg_poll(rtg_ctx* ctx, uint64_t ticket, rtg_csr* out);

/* As rtg_poll, but waits up to timeout_us microseconds (negative: no limit) for a final
 * status; RTG_E_TIMEOUT if the request is still running then (the ticket stays valid). */
rtg_status rtg_wait(rtg_ctx* ctx, uint64_t ticket, int64_t timeout_us, rtg_csr* out);

/* Multiple r-nearest-neighbour queries (Sec. II): the neighbours of a subset of the points,
 * read from a stored pair set that holds every pair twice (Sec. III-B).
 *   graph   : a symmetric CSR returned by this context (RTG_FLAG_SYMMETRIC), not released
 *   queries : nq point indices in [0, graph->n), host or device (queries_on_device);
 *             repeats allowed
 *   out     : library-owned device CSR with nq rows; row k is the neighbour list of
 *             queries[k], ascending (out->symmetric = 0).  Free with rtg_release.
 * Synchronous.  Errors: RTG_E_INVALID (graph not symmetric, nq out of range, an index
 * outside the graph), RTG_E_BUDGET, RTG_E_NOMEM, RTG_E_CUDA. */
rtg_status rtg_query_neighbors(rtg_ctx* ctx, const rtg_csr* graph, const int32_t* queries,
                               int64_t nq, int queries_on_device, rtg_csr* out);

/* r-NN queries of new points from the stored grids (Sec. V: keep all m grids; for a query,
 * examine the m cells that contain it).  An index holds, on the device, what a build of
 * Alg. 1 makes for one point set: the m grids' sorted cell keys with their point indices,
 * a hash table per grid from cell key to its run, the per-point key rows, the FP32 rows, a
 * copy of the points and the plan (error bounds, key ranges, distance band).  It is charged to the context's budget until destroyed. */
typedef struct rtg_index rtg_index;

/* Builds the index of points (arguments as rtg_all_pairs; n may be 0).  *out receives a
 * handle owned by the caller, usable with this context only, until rtg_index_destroy (call it
 * before rtg_destroy of the context).  Synchronous.  Errors as rtg_all_pairs. */
rtg_status rtg_index_create(rtg_ctx* ctx, const void* points, int dtype, int points_on_device,
                            int64_t n, int d, double r, const double* transforms, int m,
                            double cell_side, rtg_index** out);

/* Answers nq queries: queries is nq x d row-major in the index's dtype, a device pointer if
 * queries_on_device, else a host pointer (copied in).  Row k of out lists, ascending, every
 * indexed point j that shares a cell with query k in at least one grid and lies within r of
 * it: squared distance on the original coordinates <= fl(r * r), the same FP64 sequence and
 * the same FP32 filter with FP64 recheck as the build.  out is a library-owned device CSR
 * with nq rows (out->symmetric = 0); free it with rtg_release.  Synchronous.
 * Errors: RTG_E_INVALID (NULL arguments, an index of another context, nq < 0 or
 * nq >= 2^31, a query coordinate not finite or beyond the FP32 range), RTG_E_BUDGET,
 * RTG_E_NOMEM, RTG_E_CUDA, RTG_E_TIMEOUT. */
rtg_status rtg_index_query(rtg_ctx* ctx, const rtg_index* index, const void* queries,
                           int queries_on_device, int64_t nq, rtg_csr* out);

/* Frees the index's device memory (stream ordered) and the handle.  NULL, or an index of
 * another context, is ignored. */
void rtg_index_destroy(rtg_ctx* ctx, rtg_index* index);

/* Grid parameters chosen by rtg_tune_params. */
typedef struct {
  int m;                /* number of grids */
  double cell_side;     /* c = c_factor * r */
  double c_factor;      /* c / r */
  double recall;        /* measured on the sample (reported pairs / exact pairs) */
  double build_us;      /* device time of a full-size build with (m, c) */
  int64_t sample_n;     /* points in the recall sample (a prefix of the input) */
  int64_t sample_exact; /* exact pairs of the sample */
  int candidates;       /* count-only builds measured */
} rtg_param_choice;

/* Choose c and m for a target recall (the parameter tuning of Sec. III-A): for each c/r in
 * {1.0, 1.1, 1.2, 1.3, 1.4, 1.5, 1.75, 2.0}, the smallest m <= 64 whose grids report at least
 * target_recall of the exact pairs of a prefix sample (at most 32768 points), then the
 * (c, m) with the least full-size build time.  The grids are the first m of
 * rtg_transforms_generate(seed, d, 64, c, flags & RTG_FLAG_SHIFT_ONLY), which equal
 * rtg_transforms_generate(seed, d, m, c, ...).  Builds on ctx; synchronous.  Errors as
 * rtg_all_pairs, and RTG_E_INVALID when no setting reaches the target. */
rtg_status rtg_tune_params(rtg_ctx* ctx, const void* points, int dtype, int points_on_device,
                           int64_t n, int d, double r, double target_recall, uint64_t seed,
                           uint32_t flags, rtg_param_choice* out);

/* Failure-path testing (the paper has no counterpart).  Every device wait of the library
 * (look-back chains of the sort and of the CSR row scan, the tensor-core kernel's wait for
 * its MMAs) is bounded: after wait_limit iterations (0 = the default, 2^22; the tensor-core
 * wait takes 16 times that) it gives up, flags the build and lets its kernel return, the call
 * returns RTG_E_TIMEOUT and the context stays usable.  inject makes chosen waits wait for
 * something that never happens, so that this path runs on demand:
 *   RTG_INJECT_SORT_WAIT  look-back sort passes wait for an epoch no tile publishes
 *   RTG_INJECT_SCAN_WAIT  the CSR row scan waits for predecessors that never publish
 *   RTG_INJECT_TC_WAIT    the tensor-core brute force waits on a barrier nothing arrives on
 * fail_alloc_after > 0 makes the fail_alloc_after-th device allocation of ctx from now on
 * fail once with RTG_E_NOMEM.  inject = 0 and fail_alloc_after = 0 restore normal operation.
 * Nothing here faults a GPU: each hook only makes a bounded wait or an allocation give up.
 * Errors: RTG_E_INVALID (NULL ctx, unknown bits, wait_limit >= 2^31). */
#define RTG_INJECT_SORT_WAIT 1u
#define RTG_INJECT_SCAN_WAIT 2u
#define RTG_INJECT_TC_WAIT 4u
rtg_status rtg_set_test_hooks(rtg_ctx* ctx, uint32_t inject, uint32_t wait_limit,
                              int64_t fail_alloc_after);

/* Free the device memory of a CSR returned by this context and zero *csr. */
rtg_status rtg_release(rtg_ctx* ctx, rtg_csr* csr);

/* Copy a CSR to host arrays (row_ptr: n + 1 entries, col: nnz entries).  Synchronous. */
rtg_status rtg_csr_download(rtg_ctx* ctx, const rtg_csr* csr, int64_t* row_ptr, int32_t* col);

#ifdef __cplusplus
}
#endif
#endif /* RTG_H */
