/*
 * lrbatch.h -- C ABI of a GB300 (sm_103a) library for batched small and
 * rectangular FP64 matrix multiplication, C_i += A_i * B_i.
 *
 * The operation is the batched multiplication of low-rank blocks of
 * Deshmukh, Yokota and Bosilca, "Cache Optimization and Performance Modeling
 * of Batched, Small, and Rectangular Matrix Multiplication on Intel, AMD, and
 * Fujitsu Processors" (arXiv 2311.07602):
 *   - a block of shape (m, n, rank) is stored as U S V (Eq. 1, Sec. 2);
 *   - the low-rank product multiplies a "skinny" and a "small" matrix
 *     (Alg. 1; first step C_temp = A_{V^T} B_U), batched over many
 *     independent blocks (Alg. 2, loop 1 over the batch);
 *   - all arithmetic is IEEE binary64 (Sec. 7).
 * Two shapes dominate: the tall-skinny T-form C(b x r) += A(b x b) B(b x r)
 * and the outer O-form C(b x b) += A(b x r) B(r x b); any m, n, k >= 1 is
 * accepted.
 *
 * Conventions for every call:
 *   - Matrices are column-major: element (i, j) of X is X[i + j*ldx].
 *   - Operand pointers in lrb_gemm_desc are DEVICE pointers on the handle's
 *     GPU; descriptor arrays passed to the library are HOST arrays that the
 *     library copies (the caller may free them when the call returns).
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).
 *   - No call aborts, throws or traps.  Failures return a status code and
 *     set a per-thread message readable with lrb_last_error().  Invalid
 *     arguments are rejected before any CUDA call is made.
 */
#ifndef LRBATCH_H
#define LRBATCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lrb_status {
    LRB_OK = 0,
    LRB_ERR_INVALID = 1,      /* bad argument: null pointer, dim <= 0, ld < rows, size overflow */
    LRB_ERR_ALIAS = 2,        /* a C range overlaps another C or any A/B range */
    LRB_ERR_NOMEM = 3,        /* device or host allocation failed */
    LRB_ERR_BUDGET = 4,       /* a request alone exceeds the queue's HBM budget */
    LRB_ERR_QUEUE_FULL = 5,   /* back-pressure: too many requests waiting */
    LRB_ERR_TIMEOUT = 6,      /* a bounded wait ran out */
    LRB_ERR_DEVICE = 7,       /* a CUDA call failed */
    LRB_ERR_UNSUPPORTED = 8   /* valid request this build cannot serve */
} lrb_status;

/* One batch entry: C(m x n) += A(m x k) * B(k x n), binary64, column-major,
 * device pointers.  lda >= m, ldb >= k, ldc >= m.  C must not overlap A, B or
 * the C of another entry (A and B may be shared between entries).
 * T-form: m = b, n = r, k = b.  O-form: m = n = b, k = r. */
typedef struct lrb_gemm_desc {
    const double* A;
    const double* B;
    double* C;
    int32_t m, n, k;
    int32_t lda, ldb, ldc;
} lrb_gemm_desc;

/* Arithmetic of a plan.  FP64: binary64 FMAs (DFMA pipe).  FP64_DMMA_ALLOWED:
 * binary64, and the autotuner may also pick FP64 tensor-core (DMMA) tiles.
 * SPLIT_*: the operands are cut into S BF16/FP16 digit slices per k-chunk,
 * multiplied on the tensor cores with FP32 accumulation and recombined in
 * binary64 (Ozaki-style splitting; not in the paper, which is FP64-only). */
typedef enum lrb_precision {
    LRB_PREC_FP64 = 0,
    LRB_PREC_FP64_DMMA_ALLOWED = 1,
    LRB_PREC_SPLIT_BF16_S3 = 2,
    LRB_PREC_SPLIT_BF16_S4 = 3,
    LRB_PREC_SPLIT_FP16_S3 = 4,
    LRB_PREC_SPLIT_FP16_S4 = 5
} lrb_precision;

typedef struct lrb_plan_opts {
    int32_t precision;      /* lrb_precision */
    int32_t use_graph;      /* 1: lrb_launch replays a captured CUDA graph */
    int32_t tune;           /* 1: time candidate tiles for unseen shape buckets; 0: heuristic */
    int32_t force_variant;  /* >= 0: use this FP64 tile variant for every entry (testing) */
    int32_t check_alias;    /* 1: reject overlapping C ranges (LRB_ERR_ALIAS) */
    int32_t test_stall;     /* testing only, split plans: the kernel waits once on a barrier nothing
                               arrives on, so its bounded wait expires and lrb_plan_status reports
                               LRB_ERR_TIMEOUT (exercises the failure path without a GPU fault) */
    int32_t trans;          /* FP64 plans: bit 0 set -> every entry multiplies A^T, with A stored
                               k x m (lda >= k); bit 1 set -> B^T, with B stored n x k (ldb >= n).
                               m, n, k are always the sizes of the product.  0 = both as stored.
                               Plans with trans != 0 or overwrite != 0 have no plain launch. */
    int32_t overwrite;      /* FP64 plans: 1 -> C = op(A) op(B) (old C is not read); 0 -> C += */
} lrb_plan_opts;

typedef struct lrb_handle lrb_handle;
typedef struct lrb_plan lrb_plan;
typedef struct lrb_queue lrb_queue;

/* Plan summary. */
typedef struct lrb_plan_info {
    int64_t entries;
    int64_t items;          /* output tiles in the device work list */
    int64_t groups;         /* distinct (variant, m, n, k) groups = launches of lrb_launch_plain */
    double flops;           /* sum of 2 m n k */
    double alg_bytes;       /* sum of 8 (m k + k n + 2 m n): each operand once, C read and written */
    int32_t grid;           /* CTAs of the persistent launch */
    int32_t precision;
    int64_t dmma_items;     /* tiles that run on FP64 tensor-core (DMMA) variants */
} lrb_plan_info;

/* ---- handle -------------------------------------------------------------
 * Selects `device` (a CUDA ordinal), loads the tile-tuning cache (path from
 * $LRB_TUNE_CACHE, else none) and owns the streams and scratch it creates.
 * lrb_destroy frees them; it synchronises the device first. */
lrb_status lrb_create(lrb_handle** out, int device);
lrb_status lrb_destroy(lrb_handle* h);

/* ---- plans --------------------------------------------------------------
 * lrb_plan_create copies `count` host descriptors, validates them (the checks of
 * lrb_validate), picks a tile variant per entry (autotuned per shape bucket,
 * cached in the handle), splits every entry into output tiles, orders the
 * tiles longest-first and uploads descriptors and tiles to plan-owned device
 * memory.  opts == NULL means {FP64, no graph, tune, no force, check alias}.
 * C is not touched until a launch.  With tune, a plain FP64 plan (no trans,
 * no overwrite) of two to eight waves of tiles times its own tilings before
 * it returns -- a few launches each of the tuned tiles and of narrower ones (the
 * same per-element results) on its A and B and a scratch C -- and keeps the
 * faster, so A and B must then be readable device memory at creation.
 * Otherwise the operand buffers are not touched until a launch. */
lrb_status lrb_plan_create(lrb_handle* h, const lrb_gemm_desc* host_descs, size_t count,
                           const lrb_plan_opts* opts, lrb_plan** out);

/* Enqueue the whole batch as ONE persistent launch on `stream`: a CTA per SM
 * slot pulls tiles from a device work counter until the list is empty (the
 * counter reset and the kernel are one captured graph when use_graph = 1).
 * Asynchronous; A, B, C must stay valid until the stream passes this point.
 * Re-launching a plan repeats C += A B. */
lrb_status lrb_launch(lrb_plan* p, void* stream);

/* The comparator: one uniform-grid launch per distinct (variant, m, n, k)
 * group, same tile code, hence bitwise the same results as lrb_launch. */
lrb_status lrb_launch_plain(lrb_plan* p, void* stream);

lrb_status lrb_plan_get_info(const lrb_plan* p, lrb_plan_info* info);

/* Synchronises the plan's last stream and reports whether any of its
 * launches hit a bounded device-side wait (the split-precision kernel waits
 * on its tensor-core completion barrier with an iteration limit; on expiry it
 * releases its TMEM, leaves its C tile unwritten and sets a status word):
 * LRB_ERR_TIMEOUT if so (sticky), LRB_OK otherwise. */
lrb_status lrb_plan_status(lrb_plan* p);

/* Diagnostic for split-precision plans of ONE entry: launches the plan once
 * (C += A B as lrb_launch does) and also writes every k-chunk's FP32 level
 * sums P_L (the tensor-core accumulators before recombination) to the
 * device array `dump` laid out as float[chunks][S][m][n], chunks =
 * ceil(k / kc) (kc = 64 for BF16, 32 for FP16), level L = index + 2.
 * LRB_ERR_UNSUPPORTED for FP64 plans or plans of several entries. */
lrb_status lrb_split_dump_levels(lrb_plan* p, float* dump, void* stream);

/* Frees the plan's device memory after synchronising its last stream. */
lrb_status lrb_plan_destroy(lrb_plan* p);

/* Host-buffer form of a whole batch: the descriptors' A, B and C are HOST
 * pointers (pinned memory gives full copy speed; pageable works).  Copies
 * A, B and C into a handle-owned device arena (entries packed with tight
 * leading dimensions; runs of tight blocks that lie less than 256 bytes apart
 * in host memory move in one copy -- the bytes between two C blocks of such a
 * run are copied back unchanged, so they must not change during the call;
 * A and B operands whose host byte ranges overlap -- views into one operand
 * pool, or one block shared by several entries -- are served from a single
 * copy of the union of their ranges and keep their leading dimensions), runs
 * the batch in up to 64 pieces whose copies in, launches and copies out
 * overlap on three streams (each piece's three steps are enqueued together;
 * the layout and plans are cached and reused while the descriptor list
 * repeats), copies every C back and synchronises `stream`.  Returns after host C holds the result.  Not thread-safe per
 * handle; the arena grows to the largest batch seen and is freed by
 * lrb_destroy. */
lrb_status lrb_execute_host(lrb_handle* h, const lrb_gemm_desc* host_descs, size_t count,
                            const lrb_plan_opts* opts, void* stream);

/* Where the time of lrb_execute_host goes.  With timing enabled on a handle
 * (off by default; it adds six timing events per piece), every call records
 * when each piece's copies in, launch and copies out started and ended on the
 * device, and lrb_execute_host_get_timing returns the last call's summary:
 * busy time of each engine (the union of its intervals), the pairwise
 * overlaps, the bytes copied each way (achieved copy rate = bytes / busy
 * time), when the first launch started (the exposed first copy in) and how
 * long the copies ran after the last launch ended.  Times are ms on the
 * device clock; wall_ms spans the first interval's start to the last one's
 * end.  get_timing returns LRB_ERR_INVALID before the first timed call. */
typedef struct lrb_host_timing {
    int32_t valid, pieces;
    double wall_ms;
    double h2d_busy_ms, compute_busy_ms, d2h_busy_ms;
    double h2d_bytes, d2h_bytes;
    double overlap_h2d_compute_ms, overlap_d2h_compute_ms, overlap_h2d_d2h_ms;
    double compute_start_ms;          /* first launch start - first copy start */
    double compute_end_to_last_ms;    /* last copy end - last launch end */
    double first_h2d_ms, first_h2d_bytes;   /* the first piece's copies in */
} lrb_host_timing;
lrb_status lrb_execute_host_set_timing(lrb_handle* h, int32_t enable);
lrb_status lrb_execute_host_get_timing(const lrb_handle* h, lrb_host_timing* out);

/* Measures the FP64 pipe's throughput on `device`: one launch of a kernel in
 * which every thread of a full-GPU grid runs eight independent binary64 FMA
 * chains for `iters` steps, timed with CUDA events (after a short warm-up
 * launch).  Writes the achieved TFLOP/s (2 flops per FMA) and the launch's
 * ms.  The library's FP64 kernels are bound by this pipe, so this is their
 * roofline denominator measured at whatever clock the GPU runs at.
 * Synchronous; allocates no device memory. */
lrb_status lrb_fp64_peak_probe(int device, long long iters, double* tflops, double* ms);

/* Host-only: the argument checks lrb_plan_create performs, without a GPU.
 * LRB_ERR_INVALID for null pointers, count == 0, m/n/k <= 0, ld < rows,
 * element extents that overflow int64, count above 2^31 - 1;
 * LRB_ERR_ALIAS when opts->check_alias and a C range overlaps another C or
 * any A/B range (byte ranges from first to last element). */
lrb_status lrb_validate(const lrb_gemm_desc* host_descs, size_t count, const lrb_plan_opts* opts);

/* Host-only tile list of the planner for forced variant `variant`: writes up
 * to `cap` items as (entry, row0, col0, rows, cols) int32 quintuples in
 * launch order and returns their number in *n_items (for tests of the
 * scheduler invariant: every output element in exactly one tile). */
lrb_status lrb_plan_tiles_host(const lrb_gemm_desc* host_descs, size_t count, int32_t variant,
                               int32_t* out, size_t cap, size_t* n_items);

/* Number of FP64 tile variants and their tile extents (rows x cols). */
int32_t lrb_variant_count(void);
lrb_status lrb_variant_shape(int32_t variant, int32_t* bm, int32_t* bn, int32_t* is_dmma);

/* ---- the low-rank multiplication core (Alg. 1, batched as in Alg. 2) -------
 * For low-rank blocks A = A_U A_X A_{V^T} (rank ra, Eq. 1) and
 * B = B_U B_X B_{V^T} (rank rb) the product is A_U G B_{V^T} with
 *     G = A_X (A_{V^T} B_U) B_X          (ra x rb; A_{V^T}: ra x k, B_U: k x rb)
 * which the paper computes for a batch of independent blocks.  One entry:
 * device pointers, column-major, leading dimensions >= rows; G is WRITTEN
 * (Alg. 1 assigns G_XY), not accumulated; G must not overlap the operands. */
typedef struct lrb_lr_desc {
    const double* AVT;
    const double* BU;
    const double* AX;
    const double* BX;
    double* G;
    int32_t ra, rb, k;
    int32_t ld_avt, ld_bu, ld_ax, ld_bx, ldg;
} lrb_lr_desc;

/* Plans a batch of chains (host descriptor array, copied).  fused = 1: one
 * CTA per block keeps C_temp and E_temp on chip (ranks 1..64, else
 * LRB_ERR_UNSUPPORTED).  fused = 0: the comparator -- three batched
 * multiplications C_temp = A_{V^T} B_U, E_temp = A_X C_temp, G = E_temp B_X
 * through the persistent FP64 path, with temporaries in plan-owned device
 * memory (any ranks).  lrb_launch runs it; lrb_plan_get_info reports the
 * chain's flops (ra rb (2k + 2ra + 2rb) per block; the paper counts
 * 4r^3 + 2r^2 k for ra = rb = r) and bytes. */
lrb_status lrb_lr_plan_create(lrb_handle* h, const lrb_lr_desc* host_descs, size_t count, int32_t fused,
                              lrb_plan** out);

/* ---- several GPUs ----------------------------------------------------------
 * Batch entries are independent (Alg. 2, loop 1 runs over independent
 * blocks), so a batch spreads over GPUs by partitioning its entries; no data
 * moves between devices and no collective is needed.
 *
 * lrb_partition_lpt: host-only longest-processing-time partition of `count`
 * items with costs cost[0..count) (e.g. 2 m n k per entry) into `parts` parts:
 * items in order of decreasing cost (ties: lower index first), each to the
 * part with the least load so far (ties: lower part).  Writes each item's part
 * to part_of[count] and, if part_load is not NULL, every part's total cost to
 * part_load[parts].  Deterministic: every process computes the same partition
 * from the same costs, so ranks agree without exchanging anything.
 * LRB_ERR_INVALID for NULL arrays, count == 0, parts < 1 or a negative or
 * non-finite cost. */
lrb_status lrb_partition_lpt(const double* cost, size_t count, int32_t parts, int32_t* part_of, double* part_load);

/* A batch planned over several devices: entries are partitioned with
 * lrb_partition_lpt over their flops 2 m n k across the `n_handles` handles
 * (handle i gets part i) and each handle plans its share with
 * lrb_plan_create (same opts; the descriptors of part i must point at memory
 * that handle i's device can access -- place each entry's operands by the
 * partition first).  A part that receives no entries has no plan.
 * lrb_multi_launch enqueues every part's launch on streams[i] (a stream of
 * handle i's device; NULL entries mean that device's legacy default stream),
 * with no synchronisation between parts.  lrb_multi_plan_part reports part
 * i's entry count and its plan summary (entries = 0 and a zeroed summary for
 * an empty part). */
typedef struct lrb_multi_plan lrb_multi_plan;
lrb_status lrb_multi_plan_create(lrb_handle* const* handles, int32_t n_handles, const lrb_gemm_desc* host_descs,
                                 size_t count, const lrb_plan_opts* opts, lrb_multi_plan** out);
lrb_status lrb_multi_launch(lrb_multi_plan* mp, void* const* streams);
lrb_status lrb_multi_plan_part(const lrb_multi_plan* mp, int32_t part, lrb_plan_info* info);
lrb_status lrb_multi_plan_destroy(lrb_multi_plan* mp);

/* ---- launch without device allocation -----------------------------------
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc (their GPU memory is owned by a framework pool or a fixed
 * budget, or their loop must not risk the device-wide synchronisation of
 * cudaMalloc/cudaFree).  Runs C += A B for `count` entries (device operand
 * pointers, host descriptor array, same rules as lrb_plan_create) as one
 * persistent FP64 launch on `stream`, with untuned tiles, using only a
 * fixed file-scope device array for the descriptors, tiles and work counter
 * -- nothing is allocated.  Limits: count <= LRB_NOALLOC_MAX_ENTRIES and at
 * most LRB_NOALLOC_MAX_TILES output tiles (64 x 8..64 each); larger batches
 * return LRB_ERR_INVALID before any CUDA call.  The array (about 4.2 MB) is
 * held on every GPU that loads the library until the process exits.  All
 * calls share it, so calls that overlap on the GPU race: order them on one
 * stream (calls from several host threads on one stream are kept whole by
 * an internal lock).  The first call on a device looks up the array's address and the
 * kernel's limits; make it before any stream capture.  Asynchronous like
 * lrb_launch (the descriptor array is copied before the call returns). */
#define LRB_NOALLOC_MAX_ENTRIES 4096
#define LRB_NOALLOC_MAX_TILES 262144
lrb_status lrb_launch_noalloc(const lrb_gemm_desc* host_descs, size_t count, void* stream);

/* ---- serving queue --------------------------------------------------------
 * Continuous batching of multiplication requests (not in the paper, which
 * runs one batch at a time).  A request is a host array of descriptors
 * (device operands, caller-owned, valid until the request completes).
 * lrb_queue_submit is non-blocking: LRB_OK (queued; *ticket set),
 * LRB_ERR_INVALID (bad descriptors), LRB_ERR_BUDGET (the request alone needs
 * more than hbm_budget_bytes: 8 (m k + k n + m n) + 64 bytes per entry) or
 * LRB_ERR_QUEUE_FULL (the waiting FIFO is at its limit: back-pressure).  A
 * worker thread admits waiting requests in FIFO order while their bytes fit
 * in the budget left, launches each wave as one persistent launch on one of
 * `max_inflight` (1..16) stream slots, so waves that arrive while others run
 * overlap on the device, and retires finished waves, releasing their budget.
 * Results are bitwise the same alone or mixed with other requests. */
typedef struct lrb_queue_stats_t {
    uint64_t accepted, rejected_budget, rejected_full, rejected_invalid;
    uint64_t completed, failed, waiting, waves, max_concurrent_waves;
    double mean_wave_entries;
    uint64_t reserved_bytes, peak_reserved_bytes, budget_bytes;
    double p50_ms, p99_ms, mean_ms, max_ms;   /* submission -> completion observed */
    double gflops;                            /* completed flops / (last completion - first submission) */
    double flops_done;
} lrb_queue_stats_t;

lrb_status lrb_queue_create(lrb_handle* h, size_t hbm_budget_bytes, int max_inflight, lrb_queue** out);
/* Waiting-FIFO limit (default 4096 requests) and entries per wave (default
 * 65536; a larger request still forms a wave of its own). */
lrb_status lrb_queue_set_limits(lrb_queue* q, size_t max_waiting, size_t max_wave_entries);
/* Arithmetic of the waves formed from now on (lrb_precision; default FP64).
 * Split-precision waves run the tcgen05 kernel; a bounded device wait that
 * expires fails that wave's requests (LRB_ERR_DEVICE from wait/poll). */
lrb_status lrb_queue_set_precision(lrb_queue* q, int32_t precision);
lrb_status lrb_queue_submit(lrb_queue* q, const lrb_gemm_desc* host_descs, size_t n, uint64_t* ticket);
/* LRB_OK when done, LRB_ERR_TIMEOUT while pending, LRB_ERR_DEVICE if it failed. */
lrb_status lrb_queue_poll(lrb_queue* q, uint64_t ticket);
/* Bounded wait (timeout_ms < 0 means 600 s): LRB_OK, LRB_ERR_TIMEOUT or LRB_ERR_DEVICE. */
lrb_status lrb_queue_wait(lrb_queue* q, uint64_t ticket, int timeout_ms);
/* Latency of a completed request (submission -> completion observed), ms. */
lrb_status lrb_queue_latency(lrb_queue* q, uint64_t ticket, double* latency_ms);
lrb_status lrb_queue_stats(lrb_queue* q, lrb_queue_stats_t* out);
/* Drains the queue (bounded by timeout_ms; < 0 means 600 s), stops the
 * worker and frees everything; LRB_ERR_TIMEOUT if it had to abandon work. */
lrb_status lrb_queue_destroy(lrb_queue* q, int timeout_ms);

/* ---- producers and consumers of low-rank blocks ---------------------------
 * A block of shape (m, n, rank) is stored as U S V (Eq. 1, Sec. 2) with a
 * diagonal S: U is m x r (ldu >= m), S holds r values, V is r x n (ldv >= r);
 * device pointers, column-major.  Sec. 2 names the calls around the batched
 * low-rank product: blocks are produced from dense ones by a randomized SVD
 * (Halko, Martinsson and Tropp), and the low-rank product is the first step
 * of the rounded addition of low-rank blocks.  Each call below plans a batch
 * (host descriptor arrays, copied), runs on lrb_launch as a fixed sequence of
 * batched kernels (the FP64 GEMM path for every product, a Householder QR
 * kernel for the tall-skinny orthonormalisations, a one-sided Jacobi SVD
 * kernel, preconditioned by a pivoted QR, for the small l x l cores), and
 * reports its flops through lrb_plan_get_info.  Singular values come out in
 * descending order; a zero singular value gives a zero row of V (U's columns
 * stay orthonormal).  Outputs are WRITTEN and must not overlap any input or
 * another output.  lrb_plan_status returns LRB_ERR_TIMEOUT when a Jacobi SVD
 * used its whole sweep limit without converging (its last iterate is
 * written).  Limits: l (and r1 + r2) <= LRB_LR_MAX_L, m, n <= LRB_LR_MAX_ROWS,
 * count < 2^30 for the rounded addition (one of its launches covers 2 x count
 * matrices); larger requests return LRB_ERR_UNSUPPORTED before any CUDA call. */
#define LRB_LR_MAX_L 96
#define LRB_LR_MAX_ROWS 8192

typedef struct lrb_lr_block {
    double* U;
    double* S;
    double* V;
    int32_t m, n, r;
    int32_t ldu, ldv;
    int32_t reserved;
} lrb_lr_block;

/* Randomized SVD of one dense block A (m x n, lda >= m): with the Gaussian
 * test matrix Omega (n x l, ldo >= n; the caller draws it, r <= l <= min(m, n))
 *   Y = A Omega, Q = orth(Y); q times: Q~ = orth(A^T Q), Q = orth(A Q~);
 *   A^T Q = Q2 R2;  R2^T = U~ Sigma W^T (Jacobi);  U = Q U~[:, :r],
 *   S = Sigma[:r] (descending),  V = (Q2 W[:, :r])^T
 * which equals stage B's SVD of B = Q^T A = R2^T Q2^T.  out.m, out.n must
 * equal m, n; out.r is the kept rank r. */
typedef struct lrb_rsvd_desc {
    const double* A;
    const double* Omega;
    lrb_lr_block out;
    int32_t l, lda, ldo;
    int32_t reserved;
} lrb_rsvd_desc;
lrb_status lrb_rsvd_plan_create(lrb_handle* h, const lrb_rsvd_desc* host_descs, size_t count,
                                int32_t power_iters, lrb_plan** out);

/* Expansion: D (m x n, ldd >= m) += U diag(S) V, computed as (U diag(S)) V. */
typedef struct lrb_expand_desc {
    lrb_lr_block blk;
    double* D;
    int32_t ldd;
    int32_t reserved;
} lrb_expand_desc;
lrb_status lrb_expand_plan_create(lrb_handle* h, const lrb_expand_desc* host_descs, size_t count,
                                  lrb_plan** out);

/* Rounded addition: out = the rank-out.r truncation of x + y (same m, n):
 *   [x.U diag(x.S), y.U diag(y.S)] = Q1 R1,  [x.V; y.V]^T = Q2 R2,
 *   R1 R2^T = U~ Sigma W^T,  out.U = Q1 U~[:, :r], out.S = Sigma[:r],
 *   out.V = (Q2 W[:, :r])^T;   r <= x.r + y.r <= min(m, n). */
typedef struct lrb_round_add_desc {
    lrb_lr_block x, y, out;
} lrb_round_add_desc;
lrb_status lrb_round_add_plan_create(lrb_handle* h, const lrb_round_add_desc* host_descs, size_t count,
                                     lrb_plan** out);

/* Message of the last failure on the calling thread ("" if none). */
const char* lrb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LRBATCH_H */
