/*
 * spgemm_predict.h - C ABI of a GB300 (sm_103a) library that predicts the output
 * structure of a sparse matrix product C = A * B with the sampled compression
 * ratio of Du et al., "Predicting the Output Structure of Sparse Matrix
 * Multiplication with Sampled Compression Ratio" (arXiv 2207.13848).
 *
 * What the library computes (notation of Table I / Sec. II-A: A is M x K, B is
 * K x N):
 *   flop_i  number of intermediate products of output row i (Algorithm 1, Sec. V-A)
 *   F       FLOP(C) = sum of flop_i
 *   S       a seed-determined sample of A's rows (Sec. IV-A)
 *   f*, z*  FLOP and exact NNZ of the sampled output rows (Sec. IV-B, IV-D;
 *           sample_flop and sample_nnz of Algorithm 2, Sec. V-B)
 *   r*      f* / z*, the sampled compression ratio (Eq. 4)
 *   pred_i  ceil(flop_i / r*) = ceil(flop_i * z* / f*): the predicted nnz of row i
 *           (Eq. 4: the FLOP per output row divided by the predicted ratio)
 *   offsets exclusive prefix sum of pred (M + 1 entries): allocation offsets of C
 *
 * Conventions for every entry point:
 *   - Matrices, outputs, the result record and the workspace live in DEVICE
 *     memory owned by the caller.  The library allocates nothing and never
 *     synchronises the device; all work is queued on `stream` (a cudaStream_t
 *     passed as void*, NULL = the legacy default stream) and is complete when the
 *     stream reaches that point.
 *   - The return value reports errors found on the host before anything is
 *     queued (negative SPGEMM_ERR_* codes; nothing was launched).  Outcomes found
 *     on the device are written to res->status as SPGEMM_STATUS_* bits.
 *   - All counts are exact integers; results do not depend on launch shape,
 *     thread scheduling or the GPU model.
 *   - The workspace must be zero-filled before its first use and is left
 *     reusable by every call that ends with a status free of SPGEMM_STATUS_ERR_*
 *     bits, for any later call whose operands it is large enough for (the
 *     regions that must start from zero sit at fixed offsets); after such an
 *     error, zero it again.  Calls that share one workspace must not overlap in
 *     time (queue them on one stream).  A batch workspace (spgemm_batch_*) is
 *     a different layout and is not interchangeable with this one.
 */
#ifndef SPGEMM_PREDICT_H
#define SPGEMM_PREDICT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- host return codes ------------------------------------------------------ */
#define SPGEMM_OK 0
#define SPGEMM_ERR_INVALID_ARG (-1)  /* null pointer, negative size, bad mode or threshold */
#define SPGEMM_ERR_DIM_MISMATCH (-2) /* A.cols != B.rows */
#define SPGEMM_ERR_WORKSPACE (-3)    /* ws_bytes < spgemm_workspace_size(A, B) */
#define SPGEMM_ERR_CUDA (-4)         /* a CUDA launch or query failed */
#define SPGEMM_ERR_TOO_LARGE (-5)    /* a size does not fit the int32 index range */
#define SPGEMM_ERR_STATIC_CAPACITY (-6) /* spgemm_predict_structure_static: A.rows, A.cols or
                                           B.cols exceeds SPGEMM_STATIC_MAX_ROWS */

/* ---- device status bits (res->status) ------------------------------------------ */
#define SPGEMM_STATUS_OK 0
/* f* = 0 (empty sample, or only product-free rows sampled): the compression
 * ratio is undefined, so pred_i = flop_i (the upper-bound method of Sec. I).  For
 * the reference design: |S| = 0, same fallback. */
#define SPGEMM_STATUS_WARN_EMPTY_SAMPLE 0x1
/* reference design only: some pred_i exceeded 2^31 - 1 and was saturated. */
#define SPGEMM_STATUS_WARN_SATURATED 0x2
/* a column id or row offset outside its valid range was met; the offending terms
 * were counted as zero (no out-of-bounds access is made).  Results are invalid. */
#define SPGEMM_STATUS_ERR_BAD_INPUT 0x100
/* a bounded wait between thread blocks gave up (about one second); results are
 * invalid and the workspace must be zeroed again. */
#define SPGEMM_STATUS_ERR_TIMEOUT 0x200
/* validation only: some row is not strictly increasing (unsorted or repeated
 * column ids).  The predictor needs unique ids per row; order is free. */
#define SPGEMM_STATUS_WARN_UNSORTED 0x4

/* ---- types -------------------------------------------------------------------- */

/* CSR matrix (Sec. II-B): row offsets rpt[rows + 1] and column ids col[nnz],
 * int32, device memory, caller-owned.  Requirements: rpt[0] = 0, rpt
 * non-decreasing, rpt[rows] = nnz, 0 <= col < cols, ids unique within a row.
 * Values are never read: the method counts structural products and nonzeros. */
typedef struct spgemm_csr {
  int64_t rows;
  int64_t cols;
  int64_t nnz;
  const int32_t* rpt;
  const int32_t* col;
} spgemm_csr_t;

/* Row sampling (Sec. IV-A).  h32(seed, x) is the high 32 bits of output x + 1 of
 * SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) started at state `seed`. */
#define SPGEMM_SAMPLE_BERNOULLI 0  /* row i is in S iff h32(seed, i) < threshold */
#define SPGEMM_SAMPLE_PAPER_DRAW 1 /* Algorithm 2: draw r = 0..sample_num-1 picks row
                                      (h32(seed, r) * M) >> 32, with replacement;
                                      repeats count with multiplicity */

typedef struct spgemm_config {
  int32_t mode;        /* SPGEMM_SAMPLE_* */
  int32_t reserved0;   /* must be 0 */
  uint64_t threshold;  /* BERNOULLI: in [0, 2^32]; sampling ratio = threshold / 2^32;
                          2^32 samples every row */
  int64_t sample_num;  /* PAPER_DRAW: number of draws; 0 selects the paper's rule
                          min(floor(0.003 M), 300), at least 1 (Algorithm 2) */
  uint64_t seed;
} spgemm_config_t;

/* Scalars of one call, written to device memory at the end of the call. */
typedef struct spgemm_result {
  int64_t flop_total; /* F (0 where the call does not compute it) */
  int64_t flop_s;     /* f* */
  int64_t nnz_s;      /* z* */
  int64_t n_sampled;  /* |S| */
  int64_t pred_total; /* offsets[M] */
  int32_t status;     /* SPGEMM_STATUS_* bits */
  int32_t reserved;
} spgemm_result_t;

/* ---- entry points ----------------------------------------------------------------- */

/* Bytes of device workspace every entry point below needs for these operands:
 * about 8 * A.rows + A.cols + 8 * B.cols bytes plus a fixed 264 KB (the B.cols
 * part holds the bitmaps of sampled rows split over several thread blocks).  B
 * may be NULL, in which case B.cols is taken to be A.cols (C = A * A). */
size_t spgemm_workspace_size(const spgemm_csr_t* A, const spgemm_csr_t* B);

/* Algorithm 1 (Sec. V-A): flop_row[i] = sum over j in row i of A of
 * (B.rpt[A.col[j] + 1] - B.rpt[A.col[j]]), int32[A.rows]; res->flop_total = F.
 * flop_i < 2^31 always holds for valid inputs (flop_i <= nnz(B)). */
int spgemm_flop_per_row(const spgemm_csr_t* A, const spgemm_csr_t* B, int32_t* flop_row,
                        spgemm_result_t* res, void* ws, size_t ws_bytes, void* stream);

/* Steps a1-a4: draw the sample S, compute f* and z* (exact nnz of each sampled row
 * by deduplicating its products, Algorithm 2's hash loop), |S|.  r* = f* / z* is
 * the predicted compression ratio (Eq. 4).  res->flop_total is not computed (0). */
int spgemm_predict_cr(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_config_t* cfg,
                      spgemm_result_t* res, void* ws, size_t ws_bytes, void* stream);

/* The proposed method end to end (Eq. 4, Algorithm 2): f*, z* as in
 * spgemm_predict_cr, then pred_row[i] = ceil(flop_i * z* / f*) (int32[A.rows]) and
 * offsets = exclusive scan of pred_row (int64[A.rows + 1]).  flop_row
 * (int32[A.rows]) receives flop_i when not NULL.  res: F, f*, z*, |S|,
 * pred_total = offsets[M]; Z2* = F * z* / f*. */
int spgemm_predict_structure(const spgemm_csr_t* A, const spgemm_csr_t* B,
                             const spgemm_config_t* cfg, int32_t* pred_row, int64_t* offsets,
                             int32_t* flop_row, spgemm_result_t* res, void* ws, size_t ws_bytes,
                             void* stream);

/* The reference design of the prior sampling method (Sec. IV-C, Eq. 2): on the
 * same sample, Z1* = z* / p with p = |S| / M, CR1 = F / Z1*, and
 * pred_row[i] = ceil(flop_i * z* * M / (F * |S|)), saturated at 2^31 - 1;
 * offsets and flop_row as above. */
int spgemm_predict_reference(const spgemm_csr_t* A, const spgemm_csr_t* B,
                             const spgemm_config_t* cfg, int32_t* pred_row, int64_t* offsets,
                             int32_t* flop_row, spgemm_result_t* res, void* ws, size_t ws_bytes,
                             void* stream);

/* The precise method (symbolic phase, Sec. I), used as ground truth and as the
 * timed comparison: nnz_row[i] = exact nnz of output row i (int32[A.rows]),
 * offsets = exclusive scan (int64[A.rows + 1]); res->flop_total = F,
 * res->pred_total = NNZ(C). */
int spgemm_symbolic_exact(const spgemm_csr_t* A, const spgemm_csr_t* B, int32_t* nnz_row,
                          int64_t* offsets, spgemm_result_t* res, void* ws, size_t ws_bytes,
                          void* stream);

/* The sample S alone (Sec. IV-A): ids[0..|S|) in ascending row order (BERNOULLI)
 * or draw order (PAPER_DRAW); entries past |S| are untouched.  `capacity` is the
 * length of ids; |S| > capacity is a host error when it can be known on the host
 * (PAPER_DRAW) and is otherwise clipped, with res->n_sampled still the full |S|. */
int spgemm_sample_rows(int64_t rows, const spgemm_config_t* cfg, int32_t* ids, int64_t capacity,
                       spgemm_result_t* res, void* ws, size_t ws_bytes, void* stream);

/* Device-side check of the CSR requirements above.  res->status receives
 * SPGEMM_STATUS_ERR_BAD_INPUT (offsets or ids out of range) and/or
 * SPGEMM_STATUS_WARN_UNSORTED (a row not strictly increasing). */
int spgemm_validate_csr(const spgemm_csr_t* A, spgemm_result_t* res, void* ws, size_t ws_bytes,
                        void* stream);

/* Profiling hook (a library utility; the paper has no counterpart).  When
 * `before` and `after` are non-NULL cudaEvent_t handles (passed as void*), every
 * later call of spgemm_predict_structure, spgemm_predict_reference,
 * spgemm_flop_per_row and spgemm_symbolic_exact records `before` on its stream
 * just before the launch of its main kernel (the fused FLOP/prediction/scan
 * kernel; for the symbolic phase, the deduplication of all rows) and `after`
 * just after it, so cudaEventElapsedTime gives that kernel's duration.  Passing
 * NULL, NULL turns the hook off.  The setting is process-wide; it is meant for
 * benchmarks, not for concurrent use from several threads.  Returns SPGEMM_OK. */
int spgemm_set_profile_events(void* before, void* after);

/* Roofline calibration (a library utility; the paper has no counterpart).  The
 * FLOP pass of Algorithm 1 reads A's column ids in order and, for each, one
 * byte of a table of B's row lengths at a scattered position; on this GPU the
 * rate of those scattered lookups, not HBM bandwidth, bounds it.  This call
 * runs that access pattern alone: it streams col[0..n) (int32, device memory,
 * 16-byte aligned) and reads table[col[j]] (uint8, device memory, table_bytes
 * long; ids outside [0, table_bytes) count as zero) for every j, and writes
 * the sum of the bytes read to *out (uint64, device memory) on `stream`.
 * Timed by the caller, n / time is the device's lookup ceiling for that id
 * stream.  Returns SPGEMM_ERR_INVALID_ARG for a negative size, a null pointer
 * or an unaligned col, before anything is queued. */
int spgemm_lookup_probe(const int32_t* col, int64_t n, const uint8_t* table, int64_t table_bytes,
                        uint64_t* out, void* stream);

/* spgemm_predict_structure without a caller-supplied workspace.  The paper has
 * no counterpart: this is a library utility for callers that cannot allocate
 * device memory themselves, for example a host program whose device memory is
 * owned by another allocator it cannot reach (a framework's caching allocator
 * hands it only finished tensors), or a latency-critical loop that must not call
 * cudaMalloc because that call can synchronise the whole device.
 *
 * The scratch space is a fixed array of device memory compiled into the library,
 * sized for A.rows, A.cols and B.cols <= SPGEMM_STATIC_MAX_ROWS (about 35 MB).
 * Every GPU that loads the library holds it until the process exits.  Larger
 * problems are rejected with SPGEMM_ERR_STATIC_CAPACITY.  Every host check
 * (the arguments and codes of spgemm_predict_structure, then the capacity)
 * runs before anything is queued, so a call that returns a negative code has
 * queued no work.  The call allocates
 * nothing (no cudaMalloc/cudaFree, no allocating library routine): the caller
 * still passes the inputs, outputs and result record, as for
 * spgemm_predict_structure, and gets the same results.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the one array and clears its bookkeeping parts
 * (the 262 KB header and block slots, 4 * A.rows bytes of row queue and the
 * split-row slots; cudaMemsetAsync on `stream`) before use, so calls that
 * overlap on the GPU (on different streams, or from several threads) race and
 * must not be issued. */
#define SPGEMM_STATIC_MAX_ROWS (1ll << 21)
int spgemm_predict_structure_static(const spgemm_csr_t* A, const spgemm_csr_t* B,
                                    const spgemm_config_t* cfg, int32_t* pred_row,
                                    int64_t* offsets, int32_t* flop_row, spgemm_result_t* res,
                                    void* stream);

/* ---- batched prediction ---------------------------------------------------------------
 * Many independent predictions ("cases") of uneven sizes computed together: the
 * paper's method (Eq. 4, Algorithm 2) for every case, exactly as
 * spgemm_predict_structure computes it, but as one persistent launch (or, by
 * tuning, four: one per phase) that spans the whole batch, so small cases share
 * the GPU instead of each paying the latency of its own launches.  The paper predicts one product
 * at a time; batching is a library feature for callers with many products.
 * Per case, every output (pred_row, offsets, flop_row, the result record) is
 * bit-identical to spgemm_predict_structure with the same arguments, whatever
 * the batch composition and the tuning.
 *
 * Use: spgemm_batch_workspace_size -> allocate and zero-fill the workspace ->
 * spgemm_batch_prepare (writes the plan into the workspace) ->
 * spgemm_predict_batch as often as wanted (inputs may change between runs, their
 * shapes and addresses may not; graph-capturable).  A new batch needs a new
 * spgemm_batch_prepare on the same workspace. */

/* One case: operands, sampling configuration and outputs, with the meaning and
 * layout of spgemm_predict_structure's arguments (device memory, caller-owned).
 * cfg.mode is SPGEMM_SAMPLE_BERNOULLI or SPGEMM_SAMPLE_PAPER_DRAW. */
typedef struct spgemm_batch_item {
  spgemm_csr_t A;
  spgemm_csr_t B;
  spgemm_config_t cfg;
  int32_t* pred_row;        /* int32[A.rows] */
  int64_t* offsets;         /* int64[A.rows + 1] */
  int32_t* flop_row;        /* int32[A.rows], or NULL */
  spgemm_result_t* res;     /* one record per case */
} spgemm_batch_item_t;

/* Many single predictions queued by one call (a library utility; the paper has
 * no counterpart): for i = 0 .. n-1 in order, the spgemm_predict_structure call
 * of items[i] (its operands, configuration and outputs) with the workspace
 * ws[i] of ws_bytes[i] bytes, all on `stream`.  For a host that issues many
 * predictions (a serving loop), this replaces n calls across a language
 * boundary with one; each prediction is still its own launch, with results
 * bit-identical to spgemm_predict_structure.  Returns SPGEMM_OK, or the code of
 * the first call whose host checks fail, with *bad_item = its index (when
 * bad_item is not NULL): the calls before it were queued, none after it. */
int spgemm_predict_many(const spgemm_batch_item_t* items, int32_t n, void* const* ws, const size_t* ws_bytes,
                        int32_t* bad_item, void* stream);

/* Launch parameters of the batch; they change speed, never results.  0 selects
 * the default.  spgemm_batch_autotune measures candidates and picks one. */
typedef struct spgemm_batch_tuning {
  int32_t tile_items;         /* rows + nonzeros of A per FLOP tile, in [4096, 2^24]; default 16384 */
  int32_t warp_table;         /* hash slots per warp of the sampled-row pass: 512, 1024 or 2048;
                                 default 1024 */
  int32_t heavy_threshold;    /* products of a sampled row above which it is counted by a whole
                                 thread block instead of a warp, in [32, warp_table / 2];
                                 default warp_table / 2 */
  int32_t sample_chunk;       /* candidates per unit of work of the sampled-row pass, a
                                 multiple of 256 in [4096, 2^24]; default 32768 */
  int32_t flop_blocks_per_sm; /* resident blocks per SM of the FLOP pass, 1 .. what fits;
                                 default what fits (used by launches = 4) */
  int32_t launches;           /* 1: the whole batch as one persistent launch (one block per SM,
                                 grid barriers between the phases); 4: one persistent launch per
                                 phase (tables, sampled rows, heavy rows, FLOP and offsets), each
                                 with its own shared-memory size and block shape; default 4, the
                                 faster at scale (625 family cases: 33.3 against 42.0 ms) */
  int32_t reserved[2];        /* must be 0 */
} spgemm_batch_tuning_t;

/* What spgemm_batch_prepare planned; pass it to spgemm_predict_batch. */
typedef struct spgemm_batch_plan {
  int32_t n_cases;
  int32_t reserved0;
  int64_t total_rows;         /* sum of A.rows */
  int64_t total_candidates;   /* sum of the sample candidates (rows or draws) */
  int64_t total_tiles;        /* FLOP tiles */
  int64_t total_chunks;       /* work units of the sampled-row pass */
  int64_t total_table_blocks; /* blocks of the B row-length table pass */
  uint64_t ws_bytes;          /* workspace bytes the plan uses */
  spgemm_batch_tuning_t tuning; /* the tuning in force, defaults filled in */
} spgemm_batch_plan_t;

#define SPGEMM_BATCH_MAX_CASES (1 << 20)

/* Device workspace bytes for this batch under any tuning (0 for invalid
 * arguments).  About 4 bytes per row and 1 byte per column of A, 64 bytes
 * per 4096 rows + nonzeros of A, and 450 bytes per case. */
size_t spgemm_batch_workspace_size(const spgemm_batch_item_t* items, int32_t n);

/* Host bytes of the staging buffer spgemm_batch_prepare copies the plan from,
 * under any tuning. */
size_t spgemm_batch_staging_size(const spgemm_batch_item_t* items, int32_t n);

/* Checks every case as spgemm_predict_structure would (on the first failure,
 * returns its code and writes the case index to *bad_item when bad_item is not
 * NULL; nothing is queued), plans the batch under `tuning` (NULL = defaults)
 * into *plan, and queues on `stream` the copy of the plan into the workspace.
 * host_staging: page-locked host memory of at least spgemm_batch_staging_size
 * bytes that must stay untouched until the copy has completed on `stream`; or
 * NULL, in which case the call builds the plan in its own host memory and
 * returns only once the copy has completed.  The workspace must have been
 * zero-filled once before its first use; spgemm_batch_prepare may be called on
 * it again for another batch. */
int spgemm_batch_prepare(const spgemm_batch_item_t* items, int32_t n,
                         const spgemm_batch_tuning_t* tuning, spgemm_batch_plan_t* plan,
                         void* ws, size_t ws_bytes, void* host_staging, size_t staging_bytes,
                         int32_t* bad_item, void* stream);

/* Runs the prepared batch on `stream`: one 64-byte memset and one cooperative
 * kernel launch (tuning.launches = 1) or four launches (4), no host
 * synchronisation, capturable in a CUDA graph.  Every case's
 * outputs and result record are written as by spgemm_predict_structure;
 * result status bits are per case. */
int spgemm_predict_batch(const spgemm_batch_plan_t* plan, void* ws, size_t ws_bytes, void* stream);

/* Picks a tuning for this batch by measurement: prepares and runs the batch
 * under each candidate (hash-table size and heavy-row threshold, chunk size,
 * tile size, blocks per SM), `reps` timed runs each after one untimed run, and
 * writes the fastest (by the median of the runs) to *best and its time in
 * milliseconds to *best_ms (when not NULL).  Synchronous: blocks the host until
 * the measurements are done.  The phases are tuned in the four-launch form;
 * the pick is then timed end to end in both forms and the faster kept.
 * Leaves the workspace prepared with *best (as
 * spgemm_batch_prepare with *best and no staging buffer would) and the plan in
 * *plan.  Outputs are overwritten with the batch's (identical) results. */
int spgemm_batch_autotune(const spgemm_batch_item_t* items, int32_t n, void* ws, size_t ws_bytes,
                          int32_t reps, spgemm_batch_tuning_t* best, float* best_ms,
                          spgemm_batch_plan_t* plan, void* stream);

/* ---- the consumer: numeric product into the predicted allocation -----------------------
 * The prediction exists to size C before the numeric phase of C = A*B (Sec. I:
 * it replaces the symbolic phase of a two-phase SpGEMM).  These two calls are
 * that numeric phase.  spgemm_numeric_into computes every row of C into an
 * allocation sized by the prediction, in one of two ways:
 *   - per-row shares (alloc_offsets given, normally the offsets of
 *     spgemm_predict_structure): row i goes to c_col/c_val[alloc_offsets[i] ..]
 *     when its exact nnz is at most alloc_offsets[i+1] - alloc_offsets[i];
 *   - one pool (alloc_offsets NULL) of c_capacity entries, normally the
 *     predicted total pred_total = offsets[M] (Z2*, Eq. 4) plus any slack:
 *     each row takes exactly its nnz from the pool, at a position of the
 *     library's choosing, while the pool has room.
 * It writes each row's exact nnz (nnz_row) and start (row_start; -1 when the
 * row did not fit: an overflow, counted in res).  spgemm_numeric_compact then
 * builds the exact CSR of C: rows that were written are moved, rows that
 * overflowed are computed again straight into their exact place.  A caller
 * that can use (row_start, nnz_row) as is may skip the compaction when no row
 * overflowed.
 *
 * Values are single precision: a_val[nnz(A)], b_val[nnz(B)] in CSR order;
 * c_val = sum_k a_ik * b_kc, summed in single precision in no fixed order
 * (the structure is exact; a value differs from the exact sum by at most
 * (terms + 1) * 2^-24 * sum_k |a_ik * b_kc|).  Column ids within a row come
 * out in no particular order.  Structural entries are kept even when their sum
 * cancels to zero. */

/* Scalars of a numeric call (device memory, caller-owned). */
typedef struct spgemm_numeric_result {
  int64_t nnz_total;     /* NNZ(C) (spgemm_numeric_into) */
  int64_t overflow_rows; /* rows that did not fit the allocation */
  int64_t overflow_nnz;  /* the nnz of those rows */
  int64_t alloc_total;   /* alloc_offsets[A.rows] (shares) or c_capacity (pool) */
  int32_t status;        /* SPGEMM_STATUS_* bits (ERR_BAD_INPUT: an id or offset out of range) */
  int32_t reserved;
} spgemm_numeric_result_t;

/* alloc_offsets (int64[A.rows + 1], non-decreasing) or NULL for the pool mode;
 * c_col (int32) and c_val (float) hold c_capacity entries, and nothing is
 * written at or past c_capacity.  row_start (int64[A.rows]) and nnz_row
 * (int32[A.rows]) are outputs.  res is overwritten.  The workspace is the one
 * of spgemm_workspace_size(A, B). */
int spgemm_numeric_into(const spgemm_csr_t* A, const float* a_val, const spgemm_csr_t* B,
                        const float* b_val, const int64_t* alloc_offsets, int32_t* c_col,
                        float* c_val, int64_t c_capacity, int64_t* row_start, int32_t* nnz_row,
                        spgemm_numeric_result_t* res, void* ws, size_t ws_bytes, void* stream);

/* The exact CSR of C from the output of spgemm_numeric_into (same A, B, values,
 * c_col, c_val, c_capacity, row_start, nnz_row): out_rpt = exclusive scan of
 * nnz_row (int64[A.rows + 1], out_rpt[A.rows] = NNZ(C)); out_col/out_val hold
 * out_capacity >= NNZ(C) entries (res->nnz_total after spgemm_numeric_into).
 * res->status gains the bits of this call; its other fields are kept. */
int spgemm_numeric_compact(const spgemm_csr_t* A, const float* a_val, const spgemm_csr_t* B,
                           const float* b_val, const int32_t* c_col, const float* c_val, int64_t c_capacity,
                           const int64_t* row_start, const int32_t* nnz_row, int64_t* out_rpt,
                           int32_t* out_col, float* out_val, int64_t out_capacity,
                           spgemm_numeric_result_t* res, void* ws, size_t ws_bytes, void* stream);

/* Static description of a host return code or of a status bit set. */
const char* spgemm_status_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_PREDICT_H */
