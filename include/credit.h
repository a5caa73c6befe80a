/*
 * credit.h -- C ABI of the GB300 (sm_103a) reduction-reuse row library.
 *
 * The library computes wide "reduction-reuse" row ops (CREDIT, Sec. III-B,
 * Eq. 1): every row of N elements is reduced to a few scalar statistics and
 * the statistics are then applied to every element of the same row.  Three
 * execution paths exist:
 *
 *   CLUSTER   the row is split over the P CTAs of a thread-block cluster
 *             (Eq. 2); each CTA stages its slice once in shared memory with
 *             bulk-async copies, pushes its partial statistics into every
 *             peer's shared memory over DSMEM (Eq. 5), and writes its output
 *             segment from shared memory (no second HBM read, Eq. 4).
 *   ONE_CTA   the whole row is staged in one CTA's shared memory (the
 *             local-SMEM-staged non-DSMEM baseline of Sec. IV-A).
 *   TWO_PASS  the global-reread non-DSMEM baseline of Sec. IV-A: a statistics
 *             sweep over HBM, then a second sweep that rereads the row and
 *             writes the output; with ctas_per_row > 1 the row is split over
 *             several CTAs whose partials go through a device workspace and
 *             a second kernel launch.
 *
 * A planner (Sec. III-D, Eq. 3 and 7-9; optionally a learned latency model)
 * picks a path and cluster size per shape.
 *
 * Conventions shared by every entry point:
 *  - Device pointers are plain device addresses owned by the caller.  The
 *    library owns only a per-device workspace that credit_init() allocates.
 *  - All work is enqueued asynchronously on `stream` (0 = legacy default
 *    stream).  The return value reports argument and launch errors; faults
 *    found on the device (a bounded wait that gave up) are reported later by
 *    credit_device_error().
 *  - Rows are row-major.  Element i of row r lives at base + (r*ld + i)
 *    elements; ld = 0 means ld = cols.  Any element alignment is accepted;
 *    16-byte-aligned rows take the vectorised fast path automatically.
 *  - rows == 0 is a no-op that returns CREDIT_OK.  cols <= 0, a NULL data
 *    pointer, or FP8 data without scales return CREDIT_ERR_INVALID_ARG.
 *  - in == out is allowed for every op except logsumexp; partial overlap of
 *    input and output is undefined.
 *  - Statistics are computed in FP32 from inputs decoded to FP32; outputs are
 *    rounded to nearest even (FP8 saturates to +-448).
 */
#ifndef CREDIT_H_
#define CREDIT_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CREDIT_F32 = 0,
    CREDIT_BF16 = 1,
    CREDIT_FP8_E4M3 = 2,  /* e4m3 "fn": +-448 max, per-row FP32 scale */
    CREDIT_INT8 = 3       /* output of CREDIT_OP_QUANT_INT8 only: int8 codes, per-row FP32 scale */
} credit_dtype;

typedef enum {
    CREDIT_OP_SOFTMAX = 0,    /* y_i = exp(x_i - m) / sum_j exp(x_j - m)            */
    CREDIT_OP_LOGSUMEXP = 1,  /* out[r] = m + ln sum_j exp(x_j - m), FP32 per row    */
    CREDIT_OP_LAYERNORM = 2,  /* y_i = (x_i - mu) / sqrt(var + eps) * g_i + b_i      */
    CREDIT_OP_RMSNORM = 3,    /* y_i = x_i / sqrt(mean(x^2) + eps) * g_i             */
    /* Row-wise int8 quantisation (the "row-wise int8 quantization" workload of
     * Sec. IV-A): s = fl32(max_j |x_j| / 127) (1 for an all-zero row) into
     * out_scale[r]; q_i = clamp(rint(fl32(x_i / s)), -127, 127), ties to even,
     * both quotients correctly rounded in FP32.  in_dtype FP32 or BF16,
     * out_dtype CREDIT_INT8, out_scale required; gamma / beta ignored.  A
     * reduction (amax, q = 1) whose statistic is applied to every element of
     * the row: 5 bytes per FP32 element when the row is read once, 9 with the
     * global reread.  Staged (ONE_CTA / CLUSTER, either retention tier) and
     * TWO_PASS plans.  Planner rule (source 3): the smallest cluster whose
     * slices fit the tensor-memory tier, else two-pass. */
    CREDIT_OP_QUANT_INT8 = 11
} credit_op;

typedef enum {
    CREDIT_PATH_AUTO = -1,
    CREDIT_PATH_ONE_CTA = 0,
    CREDIT_PATH_TWO_PASS = 1,
    CREDIT_PATH_CLUSTER = 2
} credit_path;

/* Where the staged paths (ONE_CTA, CLUSTER) keep a row slice between its
 * reduction and its reuse pass (Sec. III-C, "reuse"; the capacity of Eq. 3).
 *   SMEM  the shared-memory chunk ring (slice <= the opt-in shared memory)
 *   TMEM  tensor memory, two 128-KiB row buffers per SM; shared memory holds
 *         only chunks in flight and gamma / beta.  Softmax, LayerNorm,
 *         RMSNorm and int8 quantisation (not FP8-output norms, not
 *         logsumexp), slice <= 128 KiB of
 *         input, one CTA per SM.  The project's addition; the paper stages
 *         in shared memory only.  A LayerNorm call whose gamma / beta cannot
 *         be staged in shared memory beside the ring (rows off the 16-byte
 *         grid) runs on the SMEM tier instead, also under an explicit TMEM
 *         plan.
 *   AUTO  TMEM where it applies and a slice exceeds 32 KiB, else SMEM
 *         (CREDIT_RETAIN=smem in the environment makes AUTO mean SMEM,
 *         CREDIT_RETAIN=tmem TMEM wherever it applies).  The planners set
 *         SMEM or TMEM explicitly. */
typedef enum {
    CREDIT_RETAIN_AUTO = 0,
    CREDIT_RETAIN_SMEM = 1,
    CREDIT_RETAIN_TMEM = 2
} credit_retain;

typedef enum {
    CREDIT_OK = 0,
    CREDIT_ERR_INVALID_ARG = 1,
    CREDIT_ERR_UNSUPPORTED = 2,      /* illegal cluster size (Eq. 3), dtype or shape   */
    CREDIT_ERR_CUDA = 3,             /* a CUDA runtime call or launch failed           */
    CREDIT_ERR_TIMEOUT = 4,          /* a bounded device wait gave up                  */
    CREDIT_ERR_NOT_INITIALIZED = 5,  /* credit_init() has not run on this device       */
    CREDIT_ERR_CAPTURE = 6,          /* the call would allocate during stream capture  */
    CREDIT_ERR_IO = 7                /* a calibration / model file could not be used   */
} credit_status;

/* Human-readable name of a status code (static storage, never NULL). */
const char *credit_status_string(credit_status s);

/* Version of this library as MAJOR*10000 + MINOR*100 + PATCH. */
int credit_version(void);

/*
 * credit_init -- prepare `device` (sets it current on the calling thread):
 * reads device limits (SM count, opt-in shared memory per block, clock),
 * raises the dynamic-shared-memory and non-portable-cluster attributes of the
 * kernels, and allocates the per-device workspace used by the split-row
 * two-pass path (and the device error word).  Idempotent and thread-safe.
 * The simple entry points call it on first use; call it yourself before any
 * stream capture, because it allocates.
 */
credit_status credit_init(int device);

/*
 * Simple entry points (BASELINE interface).  dtype is both the input and the
 * output type; FP8 needs per-row scales and is only reachable through
 * credit_run_ex (these return CREDIT_ERR_INVALID_ARG for FP8).  LayerNorm
 * uses gamma = 1, beta = 0, eps = 1e-5; RMSNorm gamma = 1, eps = 1e-6.
 * The path is chosen by credit_plan().  Sec. III-B/C; Eq. 1-2, 5.
 *   in   device pointer, rows x cols elements of dtype, contiguous rows
 *   out  device pointer, rows x cols of dtype (logsumexp: rows FP32 values)
 */
credit_status credit_softmax(const void *in, void *out, int64_t rows, int64_t cols,
                             credit_dtype dtype, cudaStream_t stream);
credit_status credit_logsumexp(const void *in, void *out, int64_t rows, int64_t cols,
                               credit_dtype dtype, cudaStream_t stream);
credit_status credit_layernorm(const void *in, void *out, int64_t rows, int64_t cols,
                               credit_dtype dtype, cudaStream_t stream);
credit_status credit_rmsnorm(const void *in, void *out, int64_t rows, int64_t cols,
                             credit_dtype dtype, cudaStream_t stream);

/*
 * Execution plan.  path / cluster_size / ctas_per_row / threads /
 * ring_chunks / chunk_bytes fully decide the launch; the rest is
 * informational.
 *   cluster_size  P of Eq. 2 for CREDIT_PATH_CLUSTER (2..16); 1 otherwise
 *   ctas_per_row  CTAs that share one row: P for CLUSTER, 1 for ONE_CTA,
 *                 G >= 1 for TWO_PASS (G > 1 uses the workspace)
 *   threads       threads per CTA (multiple of 32; 0 = default).  Staged
 *                 paths: reducer + writer threads + one producer warp
 *                 (96..288); two-pass: 64..1024 (default 512 for FP32 rows,
 *                 256 for BF16 / FP8 rows)
 *   reducer_threads  staged paths: threads that reduce and exchange (the rest
 *                 of the non-producer threads write); multiple of 32, 0 =
 *                 default (half)
 *   ring_chunks   staged paths: chunk slots of the shared-memory ring
 *                 (>= chunks of one slice; 0 = default)
 *   chunk_bytes   staged paths: bytes per chunk (multiple of 16; 0 = default)
 *   retain        staged paths: credit_retain (0 = AUTO)
 *   fill_share    CLUSTER only.  A cluster of P CTAs is placed inside one GPC, so
 *                 at P = 8 / 16 only 15 / 7 clusters fit on a GB300 (120 / 112 of
 *                 152 SMs).  With fill_share = f > 0 the last round(f * rows) rows
 *                 run on the split two-pass path (fill_g CTAs per row) on a
 *                 library stream that forks from and joins back into the
 *                 caller's stream, and fills the SMs the clusters leave idle.
 *                 The project's addition; the paper runs one path per launch.
 *   smem_bytes    dynamic shared memory per CTA (S_CTA of Eq. 3), output
 *   predicted_us  model latency for the whole call (0 when not modelled)
 *   source        0 analytic model, 1 learned model, 2 forced by caller or
 *                 environment, 3 built-in heuristic (no calibration loaded)
 */
typedef struct {
    int32_t path;          /* credit_path */
    int32_t cluster_size;
    int32_t ctas_per_row;
    int32_t threads;
    int32_t ring_chunks;
    int32_t chunk_bytes;
    int32_t reducer_threads;
    int32_t retain;        /* credit_retain: where the staged paths keep the slice */
    int64_t smem_bytes;
    float predicted_us;
    int32_t source;
    float fill_share;      /* CLUSTER: share of the rows run by the split two-pass path on the SMs the
                              clusters leave idle, concurrently (0 = none; at most 0.9) */
    int32_t fill_g;        /* CTAs per row of that two-pass part (0 = by row width) */
} credit_plan_t;

/*
 * credit_plan -- choose a plan for (op, rows, cols, in dtype -> out dtype)
 * (Sec. III-D).  Enumerates the legal candidates (Eq. 3 capacity, cluster
 * occupancy > 0), scores them with the loaded calibration (Eq. 7-9) or the
 * learned model, and returns the best one in *out.  Pure host code apart from
 * one-time occupancy queries; deterministic; thread-safe.
 * Environment overrides: CREDIT_FORCE_PATH=one_cta|two_pass|cluster,
 * CREDIT_FORCE_P=<P>, CREDIT_MODEL=analytic|learned.
 */
credit_status credit_plan(credit_op op, int64_t rows, int64_t cols, credit_dtype dtype,
                          credit_plan_t *out);
credit_status credit_plan_ex(credit_op op, int64_t rows, int64_t cols, credit_dtype in_dtype,
                             credit_dtype out_dtype, credit_plan_t *out);

/*
 * Full argument set.
 *   in, out      device pointers (see conventions); out of logsumexp = rows FP32
 *   ld_in/ld_out row strides in elements (0 = cols)
 *   in_scale     FP8 input: rows FP32 scales (x = code * scale); else NULL
 *   out_scale    FP8 output: rows FP32 scales written by the call; else NULL
 *   gamma, beta  LayerNorm / RMSNorm affine, cols FP32 each, NULL = 1 / 0
 *   eps          LayerNorm / RMSNorm epsilon; negative = default (1e-5 / 1e-6)
 */
typedef struct {
    int32_t op;            /* credit_op */
    const void *in;
    void *out;
    int64_t rows, cols, ld_in, ld_out;
    int32_t in_dtype, out_dtype;  /* credit_dtype; logsumexp output is FP32 */
    const float *in_scale;
    float *out_scale;
    const float *gamma;
    const float *beta;
    float eps;
} credit_args;

/*
 * credit_run_ex -- run one op with an explicit plan (NULL = credit_plan's
 * choice).  Returns CREDIT_ERR_UNSUPPORTED for a plan that breaks Eq. 3 or
 * cannot be scheduled on this device, without launching anything.
 */
credit_status credit_run_ex(const credit_args *args, const credit_plan_t *plan,
                            cudaStream_t stream);

/*
 * credit_run_host -- run one op on HOST buffers and return when the output is
 * in host memory.  args as credit_run_ex, except that in / out (and in_scale,
 * out_scale, gamma, beta) are host pointers; pinned memory (cudaHostAlloc /
 * cudaHostRegister) gets the full link bandwidth, pageable memory works but
 * copies slower.  The rows stream through three device staging slots in
 * blocks of about rows / 8 rows (at most 256 MiB per buffer): the copy-in of
 * block b + 1, the op on block b and the copy-out of block b - 1 overlap on
 * three CUDA streams of the library.  Row blocks of pinned buffers (the
 * first and last byte of the rows' range page-locked) are moved by a copy
 * kernel of the library that loads and stores host memory directly; pageable
 * ones by cudaMemcpy(2D)Async; scales and gamma / beta always by the latter.  plan is applied to every block (NULL:
 * credit_plan's choice for the block shape).  Staging buffers are allocated
 * on first use per device and kept (grown when needed); one host call runs
 * per device at a time.  The paper has no counterpart; it is the host-memory
 * form of the same ops (the end-to-end path).
 *   returns  credit_run_ex's statuses; CREDIT_ERR_CUDA if a copy failed
 */
credit_status credit_run_host(const credit_args *args, const credit_plan_t *plan);

/*
 * credit_max_clusters -- how many clusters (CTAs for the one-CTA path) of a
 * staged plan can be resident at once on the current device for these
 * arguments (cudaOccupancyMaxActiveClusters of the kernel the plan selects,
 * with its shared-memory request).  0 if the plan is not a legal staged plan
 * (Eq. 3, scheduling) or not a staged plan at all.  Launches nothing.
 * P * credit_max_clusters() below the SM count means the cluster path leaves
 * SMs idle, which fill_share can use.
 */
int32_t credit_max_clusters(const credit_args *args, const credit_plan_t *plan);

/*
 * credit_plan_check -- CREDIT_OK if `plan` is legal for `args` on the current
 * device (Eq. 3 capacity, cluster size, scheduling), CREDIT_ERR_UNSUPPORTED
 * if not, CREDIT_ERR_INVALID_ARG for bad arguments.  Launches nothing.
 */
credit_status credit_plan_check(const credit_args *args, const credit_plan_t *plan);

/* ------------------------------------------------------------------ backward ops
 * Input gradients of softmax, LayerNorm and RMSNorm: the backward members of
 * the paper's reduction-reuse workload suite (Sec. IV-A).  Like the forward
 * ops, each row is reduced to dot-product statistics that are then applied
 * to every element of the same row; the row now has two arrays (a and dy),
 * so the global-reread path rereads both (Eq. 4: 5 element accesses instead
 * of 3) while the staged paths keep both slices in shared memory.  With
 * g_i = dy_i * gamma_i (gamma = 1 when NULL) and N = cols:
 *   CREDIT_OP_SOFTMAX_BWD    a = y (softmax output), s = sum_j y_j dy_j,
 *                            dx_i = y_i (dy_i - s)
 *   CREDIT_OP_LAYERNORM_BWD  a = x (LayerNorm input), xh_i = (x_i - mean) rstd,
 *                            dx_i = rstd (g_i - sum_j g_j / N - xh_i sum_j g_j xh_j / N)
 *   CREDIT_OP_RMSNORM_BWD    a = x (RMSNorm input), xh_i = x_i rstd,
 *                            dx_i = rstd (g_i - xh_i sum_j g_j xh_j / N)
 * and two gradients with respect to logits z (the "softmax-logits backward"
 * workload), where y = softmax(z) is recomputed from z in the same sweep
 * with online (max, sum exp) statistics instead of being read:
 *   CREDIT_OP_SOFTMAX_LOGITS_BWD  a = z, dy:  dz_i = y_i (dy_i - sum_j y_j dy_j)
 *   CREDIT_OP_XENT_BWD       a = z, dy = t (target weights, soft labels),
 *                            scale = w (per row, NULL = 1): the gradient of
 *                            w * (-sum_j t_j log y_j), dz_i = w (y_i sum_j t_j - t_i)
 * and the gradients of two statistics of a row pair, with scale = g (the
 * upstream gradient per row, NULL = 1) and a second output dx2 (the
 * "weighted-variance backward" and "Pearson-correlation backward" workloads):
 *   CREDIT_OP_WVAR_BWD       a = x, dy = w (weights); v = sum w (x - mu)^2 / W,
 *                            mu = sum w x / W, W = sum w:
 *                            dx_i = g 2 w_i (x_i - mu) / W, dx2_i = dw_i = g ((x_i - mu)^2 - v) / W
 *   CREDIT_OP_PEARSON_BWD    a = x, dy = y; r = Sxy / sqrt(Sxx Syy) (centred sums):
 *                            dx_i = g ((y_i - yb) / sqrt(Sxx Syy) - r (x_i - xb) / Sxx),
 *                            dx2_i = dy_i = g ((x_i - xb) / sqrt(Sxx Syy) - r (y_i - yb) / Syy)
 * (their moments are accumulated about the row's first elements, which keeps
 * the centred sums accurate for rows far from zero mean)
 * mean / rstd are the forward's saved row statistics (rstd = 1/sqrt(var +
 * eps) for LayerNorm, 1/sqrt(sum x^2 / N + eps) for RMSNorm), FP32 per row.
 * Only dx is computed (the parameter gradients dgamma / dbeta are column
 * sums over rows, not row ops).  Statistics accumulate in FP32; dx is
 * rounded to nearest even.
 */
typedef enum {
    CREDIT_OP_SOFTMAX_BWD = 4,
    CREDIT_OP_LAYERNORM_BWD = 5,
    CREDIT_OP_RMSNORM_BWD = 6,
    CREDIT_OP_SOFTMAX_LOGITS_BWD = 7,
    CREDIT_OP_XENT_BWD = 8,
    CREDIT_OP_WVAR_BWD = 9,
    CREDIT_OP_PEARSON_BWD = 10
} credit_bwd_op;

/*
 *   op         credit_bwd_op
 *   dtype      CREDIT_F32 or CREDIT_BF16, for a, dy and dx (FP8: CREDIT_ERR_UNSUPPORTED)
 *   a, dy, dx  device pointers, rows x cols elements with row stride ld
 *              elements (0 = cols).  dx may equal a or dy (in place);
 *              partial overlap is undefined.
 *   gamma      norms: cols FP32, NULL = 1; ignored by softmax
 *   mean       LAYERNORM_BWD: rows FP32 (required)
 *   rstd       LAYERNORM_BWD / RMSNORM_BWD: rows FP32 (required)
 *   scale      XENT_BWD, WVAR_BWD, PEARSON_BWD: rows FP32 upstream gradients of the row losses or
 *              statistics (NULL = 1); ignored otherwise
 *   dx2        WVAR_BWD / PEARSON_BWD: the second gradient (dw or dy), laid out as dx (required); may
 *              equal dy.  Ignored otherwise.
 */
typedef struct {
    int32_t op;
    int32_t dtype;
    const void *a;
    const void *dy;
    void *dx;
    int64_t rows, cols, ld;
    const float *gamma;
    const float *mean;
    const float *rstd;
    const float *scale;
    void *dx2;
} credit_bwd_args;

/*
 * credit_run_bwd -- one backward op with a plan (NULL = credit_plan_bwd's
 * choice).  Plans:
 *   CLUSTER (P = 2..16) / ONE_CTA (P = 1)  each CTA stages its slice of a and
 *       of dy with bulk-async copies, pushes its partial sums to every peer
 *       over DSMEM, and writes its dx segment from shared memory.  ring_chunks
 *       = row buffers per CTA (0: two when they fit, so that the next row
 *       loads while this one is processed, else one, refilled chunk by chunk
 *       behind the write pass; 1 or 2 forced).  The norms also
 *       stage their gamma slice once (when gamma is 16-byte aligned).  Needs 16-byte
 *       aligned rows (a, dy, dx and ld * element size multiples of 16) and
 *       two slices within the opt-in shared memory; otherwise
 *       CREDIT_ERR_UNSUPPORTED, with nothing launched.
 *   TWO_PASS (G = ctas_per_row >= 1)  a statistics sweep over HBM and a
 *       second sweep that rereads a and dy; G > 1 splits a row over G CTAs
 *       whose partials go through the device workspace between two launches.
 *       Any alignment.
 * fill_share and retain must be 0.  Asynchronous on `stream`; the statuses
 * of credit_run_ex.
 */
credit_status credit_run_bwd(const credit_bwd_args *args, const credit_plan_t *plan, cudaStream_t stream);

/*
 * credit_plan_bwd -- a plan for (op, rows, cols, dtype) of the backward ops,
 * assuming 16-byte aligned rows (credit_run_bwd falls back to TWO_PASS for
 * unaligned rows when planning itself): the fused two-pass path for rows of
 * at most 16 KiB per array, else the staged path with the smallest cluster
 * size whose slices (two row buffers of a and dy, and gamma for the norms)
 * fit, else the split two-pass path.  The logits and pair ops, whose per-row
 * merges grow with the cluster size, are staged only for P <= 4 with slices
 * of at most 64 KiB per array.  source = 3 (built-in rule).
 */
credit_status credit_plan_bwd(int32_t op, int64_t rows, int64_t cols, credit_dtype dtype, credit_plan_t *out);

/* CREDIT_OK if `plan` is legal for `args` (see credit_run_bwd), else its error; launches nothing. */
credit_status credit_bwd_plan_check(const credit_bwd_args *args, const credit_plan_t *plan);

/* ------------------------------------------------------------------ ragged batches
 * Rows of uneven width and mixed op in one persistent cluster launch captured
 * in a CUDA graph.  Each row: elements in_base[in_off .. in_off + cols) ->
 * out_base[out_off ..) of the same dtype (offsets in elements; rows may be
 * packed with any alignment); op is CREDIT_OP_SOFTMAX or CREDIT_OP_RMSNORM
 * (gamma = 1, eps = 1e-6).  Each row is staged over the fewest CTAs of the
 * cluster, w = 1, 2, 4, ... P, whose slices fit the staging capacity; P / w
 * rows of one width share the cluster in one work item, the w CTAs of a row
 * exchanging partials over DSMEM (w = 1: the one-CTA path, w = P: the cluster
 * path).  Rows beyond the capacity at w = P stream twice within the cluster.
 * Info: narrow_items counts the items of width 1, wide_items those of width
 * > 1, huge_items the streamed rows.  The project's addition; the paper runs
 * one shape per launch.
 */
typedef struct {
    int64_t in_off, out_off, cols;
    int32_t op;
    int32_t reserved;
} credit_ragged_row;
typedef struct credit_ragged credit_ragged;
typedef struct {
    int32_t cluster_size, threads, staging_bytes, clusters;
    int64_t items, narrow_items, wide_items, huge_items;
    float tuned_us;  /* autotuner's best time for the batch (0 if not tuned) */
    int32_t vector_groups;  /* vector width: 16-byte groups a thread reads per step (1 or 2) */
} credit_ragged_info_t;
/* Build the work list, autotune (tune != 0: cluster size 4/8/16 x staging
 * capacity (48 KiB to 208 KiB) x threads (128, 256) x vector width (1 or 2
 * groups), each timed on this batch -- this launches the kernel
 * and writes out_base), and capture the chosen launch in a CUDA graph.
 * Allocates the device work list; in_base / out_base must stay valid while
 * the handle is used.  BF16 and FP32 only (FP8 rows would need scales). */
credit_status credit_ragged_create(const credit_ragged_row *host_rows, int64_t n, credit_dtype dtype,
                                   const void *in_base, void *out_base, int32_t tune, credit_ragged **out);
/* Replay the captured launch on `stream` (cudaGraphLaunch). */
credit_status credit_ragged_run(credit_ragged *h, cudaStream_t stream);
credit_status credit_ragged_info(const credit_ragged *h, credit_ragged_info_t *out);
void credit_ragged_destroy(credit_ragged *h);

/* ------------------------------------------------------------------ profiling
 * Primitive characterisation (Sec. III-A, Table II) on the current device.
 * Latencies in cycles per dependent load; rates in bytes per cycle per SM;
 * index k of the per-P arrays is P = 2, 4, 8, 16.  The two CTAs of the
 * latency and throughput clusters run on different SMs (distinct_sms = 1
 * when confirmed with %smid).  Every figure is the median of `runs`
 * (<= 0: 15) launches.  Allocates a small device buffer.
 */
typedef struct {
    double lat_local_cycles, lat_remote_cycles;
    double sync_cycles[4];
    double rate_local_read, rate_local_store, rate_remote_read;
    double rate_remote_store[4];
    double sm_clock_mhz;
    int32_t distinct_sms;
} credit_microbench_t;
credit_status credit_microbench(credit_microbench_t *out, int runs);

/*
 * credit_control_time -- median time (us, of `reps` launches) of the
 * work-free control kernel (Sec. III-D): the staged kernel's launch shape
 * (persistent clusters of P CTAs, threads, dynamic shared memory) and its
 * per-row DSMEM push all-gather, with no data work.  T_ctrl(M, N, P) of
 * Eq. 9 = control(P) - control(1).  Allocates a small device buffer.
 */
credit_status credit_control_time(credit_op op, int64_t rows, int64_t cols, credit_dtype dtype, int32_t P,
                                  int32_t reps, float *us_out);

/* ------------------------------------------------------------------ cost model
 * One evaluation of the profitability model for one (M, N, P) (Sec. III-D):
 *   B_eff   = M N b_B / T_B                                   (Eq. 7)
 *   T_save  = T_B b_reread / b_B
 *   W       = ceil(M / active_clusters)                       (Eq. 8; the
 *             paper's floor(S/P) replaced by the queried count)
 *   T_replay = W ceil(N/P) b_keep / (f B_smem_read)
 *   T_DSM   = s W (P-1) q_sum / (f B_dsm_store)
 *   T_deposit = max(0, W ceil(N/P) b_keep / (f B_smem_store) - M N b_in / B_eff)
 *   dT      = T_save - T_ctrl - T_replay - T_deposit - T_DSM    (Eq. 9)
 * ablation = 1 evaluates the "peak bandwidth + serialized staging" model of
 * Table IV instead: T_save = M N b_reread / B_peak and T_deposit = the full
 * staging time.  Times in us, f in MHz, rates in bytes per cycle, B_peak in
 * GB/s.  Pure host arithmetic; no device needed.
 */
typedef struct {
    double M, N, P;
    double T_B_us, T_ctrl_us;
    double b_B, b_reread, b_keep, b_in;
    double s_bytes, q_sum;
    double active_clusters;
    double f_mhz;
    double B_smem_read, B_smem_store, B_dsm_store;
    double B_peak_gbs;
    int32_t ablation;
} credit_model_inputs;
typedef struct {
    double W, B_eff_gbs, T_save_us, T_replay_us, T_dsm_us, T_deposit_us, T_smem_w_us, T_input_us, dT_us;
} credit_model_terms;
credit_status credit_model_eval(const credit_model_inputs *in, credit_model_terms *out);

/*
 * credit_calibrate -- profile the current device and write a calibration
 * file: microbenchmarks, the selected non-DSMEM baseline's time T_B over a
 * (rows, cols) grid per op and dtype, and the control kernel's T_ctrl over a
 * (rows, cols, P) grid (Sec. III-D).  Loads the result for planning too.
 * Slow (seconds to a minute); allocates up to `max_bytes` (<= 0: 4 GiB) of
 * device memory for the timing buffers.  CREDIT_ERR_IO if the file cannot
 * be written.
 */
credit_status credit_calibrate(const char *path, int64_t max_bytes);

/*
 * credit_load_model -- load a calibration file (and, if it names one, the
 * learned model's weights) for the current device.  From then on
 * credit_plan scores candidates with the analytic model (Eq. 7-9), or with
 * the learned model when CREDIT_MODEL=learned and weights are loaded.
 * CREDIT_ERR_IO for a missing or malformed file.
 */
credit_status credit_load_model(const char *path);

/* ------------------------------------------------------------------ learned model
 * A 3 x 64 ReLU MLP predicting log2 of a candidate plan's latency (us) from
 * 21 features (credit_mlp_features), trained on the GPU by the library's own
 * FP32 kernels (forward, backward, Adam; no tensor cores).  With
 * CREDIT_MODEL=learned, credit_plan picks the legal candidate with the
 * smallest predicted latency; the analytic model stays the fallback.  The
 * paper has no learned model; this is the project's addition.
 */
#define CREDIT_MLP_FEATURES 21
int64_t credit_mlp_num_params(void);
/* Features of candidate (path, P, G, retain, fill_share) for (op, dtypes, rows,
 * cols) into out[21]: log2 rows, log2 cols, input dtype one-hot, op one-hot,
 * path one-hot (one-CTA, two-pass, cluster), log2 P, log2 G, log2 algorithmic
 * bytes, output bytes per element, log2 input bytes per CTA, log2 CTAs per
 * SM, 1 when a staged path retains the slice in tensor memory (retain =
 * CREDIT_RETAIN_TMEM; AUTO and SMEM give 0), the fill share of a cluster
 * plan (0 for the other paths), and 1 when cols * element size is a multiple
 * of 16 bytes (contiguous rows all start on the 16-byte grid, where the staged
 * kernels keep gamma / beta in shared memory).  fill_share outside [0, 1]:
 * CREDIT_ERR_INVALID_ARG. */
credit_status credit_mlp_features(int32_t op, int32_t in_dtype, int32_t out_dtype, int64_t rows, int64_t cols,
                                  int32_t path, int32_t P, int32_t G, int32_t retain, float fill_share, float *out);
/* Train one network from scratch on n host samples (X n x 21, y = log2 us),
 * replacing the loaded model: minibatch
 * Adam on the MSE of standardised targets; He-initialised from `seed`.
 * loss_curve (NULL or `epochs` floats) gets the mean training loss per epoch. */
credit_status credit_mlp_train(const float *X, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
                               uint64_t seed, float *loss_curve);
/* An ensemble: `members` (1..16) networks trained as credit_mlp_train with
 * seeds seed, seed + 1, ...; replaces the loaded model.  Predictions and the
 * planner use the mean of the members' log2 latencies.  loss_curve is the
 * first member's. */
credit_status credit_mlp_train_ensemble(const float *X, const float *y, int64_t n, int32_t members, int32_t epochs,
                                        int32_t batch, float lr, uint64_t seed, float *loss_curve);
/* Members of the loaded model (0: none). */
int32_t credit_mlp_members(void);
/* Batched GPU inference: out[i] = predicted log2 us of feature row i (the
 * members' mean). */
credit_status credit_mlp_predict(const float *X, int64_t n, float *out);
/* One GPU forward + backward with explicit parameters on raw inputs: MSE loss
 * and its gradient (host arrays; params and grad have credit_mlp_num_params()
 * floats).  For checking the kernels. */
credit_status credit_mlp_grad(const float *params, const float *X, const float *t, int64_t n, float *grad,
                              float *loss);
/* One Adam step (Kingma & Ba; b1 = 0.9, b2 = 0.999, eps = 1e-8, step = 1, 2,
 * ...) of the training kernel on host arrays of credit_mlp_num_params()
 * floats: params, m and v are updated in place from grad.  For checking the
 * kernel.  CREDIT_ERR_INVALID_ARG for NULL arrays, step < 1 or lr <= 0. */
credit_status credit_mlp_adam_step(float *params, const float *grad, float *m, float *v, int32_t step, float lr);
credit_status credit_mlp_save(const char *path);
credit_status credit_mlp_load(const char *path);

/*
 * credit_set_trace -- phase tracing of the staged kernels.  While a buffer is
 * set, the first 32 CTAs of every staged launch write global-timer stamps (ns)
 * for their first R = bytes / (32 * 8 * 8) rows into it, as uint64
 * [cta][row][8].  Shared-memory retention: 0 row start, 1 stage-1 sweep done,
 * 2 CTA reduction done, 3 DSMEM exchange done, 4 reuse pass done, 5 producer
 * issued the row's last chunk (6, 7 unused).  Tensor-memory retention:
 * 0 reducer row start, 5 its TMEM buffer free, 1 sweep done, 2 warp partial
 * merged and pushed; 6 writer row start, 3 statistics in hand, 4 writes done
 * (7 unused).  device_buf: caller-owned device memory, 8-byte aligned; NULL
 * turns tracing off.  Not thread-safe against concurrent launches; a
 * debugging aid, off by default.
 */
credit_status credit_set_trace(void *device_buf, int64_t bytes);

/*
 * credit_run_two_pass_noalloc -- the split-row two-pass path (ctas_per_row
 * CTAs per row, partials exchanged through device memory between two kernel
 * launches) for callers that cannot allocate device memory: frameworks whose
 * caching allocator owns the device heap and pass a library only finished
 * buffers (a cudaMalloc of the library's own would fragment that heap, or
 * fail once the allocator has reserved it), and embeddings that forbid
 * allocation after start-up.  The paper has no counterpart; it is an
 * interface variant of the non-DSMEM baseline.
 *   args          as credit_run_ex (caller-owned device buffers; FP8 output
 *                 scales included)
 *   ctas_per_row  CTAs per row, 2..4096; outside that: CREDIT_ERR_UNSUPPORTED
 * Allocates nothing and never calls credit_init(): the partials live in a
 * fixed 4 MiB array in the library's device image (on every GPU that loads
 * the library, until the process exits), 262144 (row, CTA) partial sets, so
 * one launch covers floor(262144 / ctas_per_row) rows and longer calls are
 * split into several launches on `stream`.  The first call on a device (and
 * the first after that device's context was reset) looks up the array's
 * device address with cudaGetSymbolAddress; make that first call before any
 * stream capture.  The array keeps the last call's partials; each call writes
 * every partial it reads, so nothing needs clearing.  All calls share the one
 * array: calls that can overlap on the GPU (different streams, no ordering
 * between them) race and corrupt each other's results.
 */
credit_status credit_run_two_pass_noalloc(const credit_args *args, int32_t ctas_per_row,
                                          cudaStream_t stream);

/* ------------------------------------------------------------------ structural screen and negative controls
 * Before any clustered variant is generated, the profitability model rejects
 * three dataflows by construction (Sec. III-D, last paragraph; the negative
 * controls of Sec. IV-C), because a wider row cannot make them profitable:
 *   CREDIT_SCREEN_NO_REUSE      no reduction stage whose statistics every
 *                               element needs, or nothing the global-reread
 *                               baseline reads twice (b_reread = 0: log-sum-exp,
 *                               an elementwise op, a stencil)
 *   CREDIT_SCREEN_ORDERED       the value a CTA applies depends on the CTAs
 *                               before it in order (a scan's carries): the
 *                               barrier count K grows with P instead of 2L
 *   CREDIT_SCREEN_REMOTE_STATE  the CTAs must exchange data that grows with N
 *                               (selection, top-k, medians), not the compact
 *                               q_l statistics of Eq. 6
 * CREDIT_SCREEN_CANDIDATE goes on to the Eq. 7-9 profitability test.
 */
typedef enum {
    CREDIT_OP_SCAN = 12,     /* control: y_i = sum_{j <= i} x_j (inclusive prefix sum per row), FP32 */
    CREDIT_OP_STENCIL = 13,  /* control: y_i = sum_{k=-r..r} w[k + r] x_{i+k}, zero-padded row ends, FP32 */
    CREDIT_OP_SELECT = 14    /* control (screen only, no kernel): row-wise selection, e.g. top-k */
} credit_control_op;
typedef enum {
    CREDIT_SCREEN_CANDIDATE = 0,
    CREDIT_SCREEN_NO_REUSE = 1,
    CREDIT_SCREEN_ORDERED = 2,
    CREDIT_SCREEN_REMOTE_STATE = 3
} credit_screen_verdict;
typedef struct {
    int32_t stages;               /* L: reduction stages before the reuse pass (0: none)                 */
    int32_t ordered;              /* 1: stage results are ordered prefixes over the CTAs of a row        */
    double q_sum;                 /* statistics each CTA exchanges per row, summed over the stages      */
    double b_reread;              /* bytes per element the global-reread baseline reads a second time    */
    double remote_bytes_per_elem; /* data each CTA must exchange per element of its slice (0: compact)   */
} credit_dataflow;
/* The dataflow of a forward op (credit_op), CREDIT_OP_QUANT_INT8 or a control
 * op, for rows of in_dtype.  Pure host code.  CREDIT_ERR_INVALID_ARG for an
 * unknown op. */
credit_status credit_dataflow_of(int32_t op, credit_dtype in_dtype, credit_dataflow *out);
/* The structural screen for cluster size P (1..16): *verdict gets a
 * credit_screen_verdict, *K (may be NULL) the barrier count per row (2L, or
 * 2L(P - 1) for ordered stages).  Pure host code. */
credit_status credit_screen(const credit_dataflow *d, int32_t P, int32_t *verdict, int32_t *K);
/* Plan of a control op (CREDIT_OP_SCAN / CREDIT_OP_STENCIL): the screen's
 * verdict in *verdict (may be NULL), and the non-DSMEM global-memory path
 * (path TWO_PASS: the scan one CTA per row, the stencil a grid over the
 * row).  source = 3. */
credit_status credit_plan_control(int32_t op, int64_t rows, int64_t cols, credit_plan_t *out, int32_t *verdict);
/* Run a control op on FP32 device rows (row strides ld_in / ld_out elements,
 * 0 = cols): the scan (in == out allowed) with one CTA per row, one read and
 * one write of every element; the stencil with weights = 2 radius + 1 FP32
 * values in device memory, radius 0..8, in != out, rows <= 65535.  The sums
 * accumulate in FP32 (the scan's carry across tiles with Kahan
 * compensation).  Asynchronous on `stream`. */
credit_status credit_run_control(int32_t op, const float *in, float *out, int64_t rows, int64_t cols, int64_t ld_in,
                                 int64_t ld_out, const float *weights, int32_t radius, cudaStream_t stream);

/*
 * credit_set_wait_test -- test only: exercises the bounded-wait error path
 * without faulting anything.  wait_ns > 0 sets the limit of the staged
 * reducers' chunk waits (0 restores the default, 2 s).  extra_tx_bytes > 0
 * (a multiple of 16, at most 1 MiB) makes the shared-memory staged kernel's
 * first chunk barrier expect that many bytes more than its bulk copy
 * delivers, so the reducers' wait runs out, sets the device error word and
 * returns; the kernel then finishes (its output for that call is not
 * defined) and credit_device_error() reports CREDIT_ERR_TIMEOUT.  Only
 * accepted for a one-CTA plan on one row of one chunk with shared-memory
 * retention (the barrier is armed once and never reused, and the one copy
 * issued completes); any other staged call returns CREDIT_ERR_UNSUPPORTED
 * while extra_tx_bytes > 0, launching nothing.  Process-wide; not thread-safe
 * against concurrent calls.  The paper has no counterpart.
 */
credit_status credit_set_wait_test(int64_t wait_ns, int32_t extra_tx_bytes);

/*
 * credit_device_error -- synchronise `stream`, then read and clear the
 * device error word of the current device.  Returns CREDIT_ERR_TIMEOUT if a
 * kernel's bounded wait gave up since the last call, CREDIT_OK otherwise.
 */
credit_status credit_device_error(cudaStream_t stream);

/*
 * Capacity of one CTA for a staged slice (Eq. 3): the largest slice, in
 * elements of dtype, that fits the opt-in shared memory of the current device
 * next to the fixed scratch.  0 before credit_init.
 */
int64_t credit_slice_capacity(credit_dtype dtype);

/*
 * Number of kernels this library has launched in this process, all devices
 * (monotonic).  The difference across a region counts the launches in it.
 */
long long credit_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* CREDIT_H_ */
