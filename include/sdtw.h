/*
 * sdtw.h -- C ABI of the GB300 (sm_103a) batched subsequence-DTW library.
 *
 * The operation (paper Section 2, Eq. 1): a query x of length N (one DP row per
 * sample) is aligned against a reference y of length M (one DP column per
 * sample) by
 *
 *     D(i,j) = d(x_i, y_j) + min{ D(i-1,j), D(i,j-1), D(i-1,j-1) },
 *     d(x,y) = (x - y)^2,
 *
 * with a free start in the reference (row 0 holds only the local cost,
 * D(0,j) = d(x_0, y_j)) and a free end: each query returns
 * cost = min_j D(N-1, j) and end = the smallest j attaining it.  Column 0 has
 * only the cell above.  A batch holds many queries against one reference, as
 * in the paper's runSDTW (Section 5): the queries are stored back to back,
 * with no gaps or metadata (Section 5.1), either all of one length N or, with
 * an offsets array, of different lengths.
 *
 * Conventions shared by every entry point:
 *   - Device pointers are CUDA global-memory addresses on the context's device;
 *     the caller owns every buffer it passes and keeps it alive until the work
 *     queued on `stream` has finished.  Host pointers are ordinary (preferably
 *     pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Device-pointer calls are asynchronous: they validate, queue
 *     kernels on `stream` and return.  Host-pointer calls return after their
 *     results are in host memory.
 *   - A status other than SDTW_OK means nothing was queued, except SDTW_E_CUDA
 *     returned after a failed launch.  No C++ exception crosses this ABI.
 *   - Errors found on the device (a query longer than N in a ragged batch, an
 *     end index out of range) are recorded in the context's device status word
 *     and reported by sdtw_last_device_status.  A forward writes the empty
 *     query's outputs for such a query (cost = +inf, or INT32_MAX in SDTW_I8;
 *     end = -1); a backward leaves that query's gradient entries unwritten.
 *   - A context is not thread-safe: use one context per host thread / stream.
 *   - Inputs must be finite.  Inputs are used as given; z-normalisation (the
 *     paper's Eq. 2) is the caller's step (sdtw_znormalize), or the
 *     library's for the queries with SDTW_FLAG_ZNORM_QUERIES.
 */
#ifndef SDTW_H
#define SDTW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SDTW_ABI_VERSION 5

typedef struct sdtw_ctx sdtw_ctx;

typedef enum sdtw_status {
    SDTW_OK = 0,
    SDTW_E_INVALID = 1,     /* bad argument (null pointer, N<1, M<1, B<0, dtype mismatch, size over a configured maximum) */
    SDTW_E_NOMEM = 2,       /* device or host workspace could not be allocated, or would exceed mem_cap_bytes */
    SDTW_E_CUDA = 3,        /* a CUDA runtime call failed; the CUDA error text is kept in the context */
    SDTW_E_TIMEOUT = 4,     /* a bounded device-side wait ran out (the backward's walker and helpers wait on one
                               another in shared memory for at most 2 s each) */
    SDTW_E_UNSUPPORTED = 5  /* a valid request this build does not implement (e.g. backward in int8 mode) */
} sdtw_status;

typedef enum sdtw_dtype {
    SDTW_F32 = 0, /* float inputs, float costs, FP32 arithmetic (fused multiply-add) */
    SDTW_I8 = 1,  /* int8 inputs, int32 costs, exact integer arithmetic */
    SDTW_U8 = 2,  /* uint8 codebook codes (sdtw_codebook_encode), int32 costs in units of the codebook's
                     step^2, exact integer arithmetic */
    SDTW_F16 = 3  /* the paper's precision: IEEE binary16 inputs, every operation of Eq. 1 rounded to binary16
                     (two queries per thread as __half2), float costs holding the binary16 result; uniform
                     batches only (no offsets) */
} sdtw_dtype;

/* sdtw_config.flags (SDTW_I8 and SDTW_U8 contexts run the forward only) */
#define SDTW_FLAG_GRAD 0x1u             /* the context will run sdtw_backward: size checkpoint workspace */
#define SDTW_FLAG_KEEP_CHECKPOINTS 0x2u /* sdtw_forward also stores the checkpoints sdtw_backward needs */
#define SDTW_FLAG_NO_AUTOTUNE 0x4u      /* use the built-in default plan instead of timing candidates */
/* SDTW_F32 only: sdtw_forward, sdtw_backward, sdtw_path and sdtw_autotune
 * z-normalise every query (paper Eq. 2, bit for bit as sdtw_znormalize does on
 * 16-byte-aligned buffers)
 * into a device copy the context owns before the fill, so the caller passes
 * raw queries; sdtw_backward's grad_queries is then the gradient with respect
 * to the raw queries (the normalisation's own derivative applied on the
 * device).  The reference is used as given (normalise it once with
 * sdtw_znormalize).  The copy holds max_total_query_len floats; a ragged
 * query that would reach past it is skipped and reported like a query longer
 * than N. */
#define SDTW_FLAG_ZNORM_QUERIES 0x8u
/* For tests of the device-side timeout only: the backward's helper warps take no
 * work, so the walker's bounded wait for a band it handed out runs out and
 * sdtw_last_device_status reports SDTW_E_TIMEOUT (after about 2 s). */
#define SDTW_FLAG_TEST_IDLE_HELPERS 0x10u

typedef struct sdtw_config {
    sdtw_dtype dtype;
    int32_t device;              /* CUDA device ordinal */
    int64_t max_ref_len;         /* largest M that will be passed */
    int64_t max_total_query_len; /* largest total query samples per call (B*N, or offsets[B]) */
    int32_t max_batch;           /* largest B */
    int32_t max_query_len;       /* largest N (the longest query of a ragged batch) */
    int32_t seg_width;           /* reference columns per thread (the paper's segment width): 8, 16, 20, 24, 28
                                    or 32; 0 = chosen by the library */
    int32_t warps_per_query;     /* warps cooperating on one query; 0 = chosen by the library */
    int32_t ckpt_stride;         /* forward steps between backward wavefront checkpoints: 8, 16, 32 or 64; 0 = chosen by
                                    the library (16 with 4-row tiles, 8 with 8-row tiles, or the autotuner's
                                    choice) */
    int32_t prune_gap;           /* SDTW_I8 / SDTW_U8 only: 0 = off (exact); > 0 = early-INF pruning (paper
                                    Section 8, opt-in, changes results): a cell whose two samples differ by more
                                    than prune_gap costs +inf, and +inf absorbs every sum; a query with no path
                                    left gets cost INT32_MAX and end -1 */
    size_t mem_cap_bytes;        /* cap on device workspace; 0 = 16 GiB */
    uint64_t spin_limit;         /* reserved, must be 0 (the backward's helpers wait on flags in shared memory with
                                    a fixed limit of 2 s each) */
    uint32_t flags;              /* SDTW_FLAG_* */
    int32_t tile_rows;           /* query rows a thread advances per step: 2 or 4, or 8 with
                                    seg_width 16 to 28 (any dtype; with checkpoints, SDTW_F32); 0 = chosen by
                                    the library */
    int32_t bwd_warps;           /* warps per query in sdtw_backward and sdtw_path: 1 = one warp walks the path
                                    and recomputes every band; 2 to 4 = that warp and 1 to 3 helpers that
                                    recompute the bands a path staying on its current row would visit next;
                                    0 = chosen by the library (3, fewer if the CTA's shared memory would not
                                    fit); the results are the same for every value */
} sdtw_config;

/* Description of how a call of a given shape will run (for reports and tests). */
typedef struct sdtw_plan {
    int32_t seg_width;       /* W: reference columns per thread */
    int32_t warps_per_query; /* P: warps in one query's chain of threads */
    int32_t ctas_per_query;  /* CTAs in one query's chain (thread-block cluster size) */
    int32_t persistent;      /* 1 if one persistent launch pulls queries from a device queue */
    int64_t grid;            /* CTAs launched */
    int32_t block;           /* threads per CTA */
    int32_t smem_bytes;      /* dynamic shared memory per CTA */
    int32_t ckpt_stride;     /* forward steps between wavefront checkpoints (0 when none are stored) */
    int32_t tuned;           /* 1 if chosen by timing candidates, 0 if the default */
    int64_t sweep_cols;      /* reference columns covered by one sweep of the chain */
    int32_t tile_rows;       /* query rows a thread advances per step */
    int32_t ckpt_cols;       /* K = 8 * seg_width: columns between boundary-column checkpoints (0 when none) */
    int32_t bwd_warps;       /* warps per query of the backward (0 when the plan has no backward) */
} sdtw_plan;

/* ABI version this library was built with (SDTW_ABI_VERSION). */
int32_t sdtw_abi_version(void);

/* Human-readable name of a status code (static string, never NULL). */
const char* sdtw_status_string(sdtw_status s);

/* Fill *cfg with defaults: F32, device 0, maxima of the paper's batch
 * (512 x 2000 vs 100,000), everything else chosen by the library.
 * Errors: SDTW_E_INVALID if cfg is NULL. */
sdtw_status sdtw_config_init(sdtw_config* cfg);

/* Create a context on cfg->device.  The context owns its device workspace
 * (status word, work queue, checkpoints and gradient scratch when
 * SDTW_FLAG_GRAD is set), sized from the cfg maxima and allocated here.
 * *out receives the context, or NULL on error.
 * Errors: SDTW_E_INVALID (NULL arguments, non-positive maxima, unknown dtype,
 * SDTW_FLAG_GRAD with a dtype other than SDTW_F32, an unsupported seg_width or
 * tile_rows (8 with a seg_width outside 16 to 28), a
 * non-zero spin_limit, a negative ckpt_stride or prune_gap, a prune_gap with
 * SDTW_F32 or SDTW_F16, a bwd_warps outside 0 to 4),
 * SDTW_E_UNSUPPORTED (a ckpt_stride other than 0, 8, 16, 32 or 64, or a
 * max_query_len no forward plan can stage in shared memory),
 * SDTW_E_NOMEM (workspace above mem_cap_bytes, too small for one query's
 * checkpoints, or allocation failure), SDTW_E_CUDA (device unusable). */
sdtw_status sdtw_create(sdtw_ctx** out, const sdtw_config* cfg);

/* Release the context and its workspace (synchronises its device first).
 * NULL is accepted.  Returns SDTW_OK or SDTW_E_CUDA. */
sdtw_status sdtw_destroy(sdtw_ctx* ctx);

/*
 * Forward sDTW of a batch (Section 2, Eq. 1; batch layout of Section 5).
 *   ref      device, M elements: float (SDTW_F32), int8 (SDTW_I8), uint8 codebook
 *            codes (SDTW_U8) or IEEE binary16 (SDTW_F16).
 *   queries  device: uniform batch [B][N] row-major when offsets == NULL;
 *            ragged batch of offsets[B] elements when offsets != NULL
 *            (query q = queries[offsets[q] .. offsets[q+1])).  Same element
 *            type as ref.
 *   offsets  device int64 [B+1], non-decreasing, offsets[0] = 0, or NULL.
 *            Ragged queries must be no longer than N; an empty query returns
 *            cost = +inf (SDTW_F32) or INT32_MAX (SDTW_I8, SDTW_U8) and end = -1.
 *            SDTW_F16 takes uniform batches only (offsets must be NULL).
 *   B        number of queries (0 is a no-op).  N: the query length (uniform)
 *            or an upper bound on every query length (ragged).  M >= 1.
 *   cost     device, B elements: float (SDTW_F32; SDTW_F16, holding the binary16
 *            result exactly) or int32 (SDTW_I8, SDTW_U8).
 *   end      device int64, B elements: the smallest column of the minimum.
 * With SDTW_FLAG_KEEP_CHECKPOINTS the call also stores the checkpoints a
 * following sdtw_backward (or sdtw_path) on the same arguments reuses, when
 * the whole batch's checkpoints fit the context's workspace (otherwise the
 * backward re-runs the forward in chunks of queries).
 * Errors: SDTW_E_INVALID (null pointers with B > 0, N < 1, M < 1, sizes above
 * the context maxima; SDTW_I8 and SDTW_U8 need N <= 32,896 so int32 costs cannot
 * overflow), SDTW_E_UNSUPPORTED (N too long for shared memory, offsets with
 * SDTW_F16), SDTW_E_CUDA.
 */
sdtw_status sdtw_forward(sdtw_ctx* ctx, const void* ref, int64_t M, const void* queries,
                         const int64_t* offsets, int32_t B, int32_t N, void* cost, int64_t* end,
                         void* stream);

/*
 * Gradient of sum_q grad_cost[q] * cost[q] (SDTW_F32 only).
 * The warp path of each query is recovered by walking back from (N_q-1, end[q])
 * (Section 2's walk-back: to the neighbour (i-1,j-1), (i,j-1) or (i-1,j) of
 * smallest D, exact ties to the first of that list, column 0 upwards, stopping
 * at row 0).  The DP is recomputed band by band from checkpoints of the
 * forward: its wavefront (an anti-diagonal staircase of rows, one per thread)
 * every ckpt_stride steps (8, 16, 32 or 64), and the boundary column of every
 * K-column window (K = 8 * seg_width); a band (one window, one stride of
 * steps) is recomputed with the forward's own FP32 operations, so the values
 * are the forward's bit for bit.  A shorter stride makes each band change of
 * the walk cheaper and doubles the checkpoint memory.  The full matrix is
 * never stored.  Under mem_cap_bytes the batch may run in chunks of queries,
 * each re-running its forward with checkpoint stores.
 * Along the path, d cost/d x_i += 2 (x_i - y_j) and d cost/d y_j += -2 (x_i - y_j).
 *   ref, queries, offsets, B, N, M: as in sdtw_forward (float).
 *   end         device int64 [B]: the end columns sdtw_forward returned.
 *   grad_cost   device float [B]: upstream gradient of each cost.
 *   grad_queries device float, same layout as queries: overwritten (with
 *               SDTW_FLAG_ZNORM_QUERIES: the gradient with respect to the raw
 *               queries passed in, through their normalisation).
 *   grad_ref    device float [M]: overwritten with the sum over queries
 *               (summed in query order: deterministic).
 *   path        device int32, NULL or 2 per query sample: for row i of query q
 *               the first and last column of the path in that row
 *               (path[2*(start_q+i)] and path[2*(start_q+i)+1], start_q = q*N or
 *               offsets[q]).  A warp path is monotone, so this fixes it.
 * If the context has SDTW_FLAG_KEEP_CHECKPOINTS and the previous sdtw_forward
 * on this context had the same ref/queries/offsets pointers and sizes, its
 * checkpoints are reused: the caller must not have changed those inputs.
 * Otherwise the forward is re-run with checkpoint stores first.
 * Errors: SDTW_E_UNSUPPORTED (SDTW_I8 context), SDTW_E_INVALID (no
 * SDTW_FLAG_GRAD, bad arguments as for sdtw_forward), SDTW_E_NOMEM, SDTW_E_CUDA.
 */
sdtw_status sdtw_backward(sdtw_ctx* ctx, const float* ref, int64_t M, const float* queries,
                          const int64_t* offsets, int32_t B, int32_t N, const int64_t* end,
                          const float* grad_cost, float* grad_queries, float* grad_ref,
                          int32_t* path, void* stream);

/*
 * The warp path of every query without gradients (the paper's walk-back,
 * Section 2, as in sdtw_backward): for row i of query q, path[2*(start_q+i)]
 * and path[2*(start_q+i)+1] receive the first and last column of the path in
 * that row (start_q = q*N or offsets[q]).
 *   ref, queries, offsets, B, N, M, end: as in sdtw_backward.
 *   path      device int32, 2 per query sample: overwritten.
 * Needs an SDTW_F32 context with SDTW_FLAG_GRAD (it uses the checkpoint
 * workspace); like sdtw_backward it reuses the checkpoints of a kept forward
 * on the same inputs, else re-runs the forward with checkpoint stores.
 * Errors: as sdtw_backward.
 */
sdtw_status sdtw_path(sdtw_ctx* ctx, const float* ref, int64_t M, const float* queries,
                      const int64_t* offsets, int32_t B, int32_t N, const int64_t* end, int32_t* path,
                      void* stream);

/*
 * sdtw_forward from and to host memory (the paper's runSDTW shape: host batch
 * in, host results out).  Copies ref/queries/offsets into context-owned
 * device buffers, runs the forward, copies cost/end back and synchronises
 * `stream`.  Pointers are host pointers with the layouts of sdtw_forward.
 * Errors: as sdtw_forward, plus SDTW_E_NOMEM when staging buffers cannot grow.
 */
sdtw_status sdtw_forward_host(sdtw_ctx* ctx, const void* ref, int64_t M, const void* queries,
                              const int64_t* offsets, int32_t B, int32_t N, void* cost,
                              int64_t* end, void* stream);

/*
 * One differentiable step from and to host memory: forward and backward on
 * staged copies of ref/queries, then cost, end, grad_queries and grad_ref
 * (and path if not NULL) copied back; synchronises `stream`.  grad_cost is a
 * host float [B].  Needs an SDTW_F32 context with SDTW_FLAG_GRAD.
 * Errors: as sdtw_forward and sdtw_backward.
 */
sdtw_status sdtw_forward_backward_host(sdtw_ctx* ctx, const float* ref, int64_t M,
                                       const float* queries, const int64_t* offsets, int32_t B,
                                       int32_t N, const float* grad_cost, float* cost,
                                       int64_t* end, float* grad_queries, float* grad_ref,
                                       int32_t* path, void* stream);

/*
 * Time the candidate plans (segment width, warps per query, tile height) on
 * the given device-resident batch and keep the fastest for calls of this
 * shape class (dtype, ragged or not, N and M buckets, checkpoints) on this
 * context.  On a context with SDTW_FLAG_KEEP_CHECKPOINTS whose workspace holds
 * the batch's checkpoints, each candidate is timed as a forward with
 * checkpoint stores followed by the backward (with zero upstream gradients
 * into scratch it allocates for the call), so the plan serves the
 * differentiable step; the checkpoint stride (8, 16, 32 or 64 steps, unless the
 * config fixes it) is then one more axis, and a stride whose checkpoints do
 * not fit the workspace under mem_cap_bytes is not a candidate.  Runs several forwards on `stream` and synchronises
 * it.  Arguments as sdtw_forward; cost/end are scratch outputs.  *plan (if not
 * NULL) receives the chosen plan.  Errors: as sdtw_forward, and SDTW_E_NOMEM
 * when the backward's scratch cannot be allocated.
 */
sdtw_status sdtw_autotune(sdtw_ctx* ctx, const void* ref, int64_t M, const void* queries,
                          const int64_t* offsets, int32_t B, int32_t N, void* cost,
                          int64_t* end, void* stream, sdtw_plan* plan);

/* The plan a forward (backward = 0) or backward (backward = 1) call of this
 * shape would use.  ragged = 1 for a call with offsets.  No device work.
 * Errors: SDTW_E_INVALID. */
sdtw_status sdtw_get_plan(sdtw_ctx* ctx, int32_t B, int32_t N, int64_t M, int32_t ragged,
                          int32_t backward, sdtw_plan* plan);

/*
 * Batch z-normalisation (paper Section 5.1, Eq. 2): each series becomes
 * (x - mean) / S with its own mean and population standard deviation S (the
 * paper's code divides by n); a series with S == 0 is only centred.  Two
 * passes (the mean, then the centred second moment) in float with compensated
 * sums and float-pair reductions: every output is within 2^-21 (|z| + 1) of
 * the exact value.  This is the standardisation
 * the forward expects of its inputs (the library does not apply it
 * implicitly).
 *   in, out   device float: B series back to back, [B][N] or delimited by
 *             offsets; out may equal in (in place).  Only the series' own
 *             elements are written.
 *   offsets   device int64 [B+1] (ascending) or NULL for B series of length N.
 *             A series with offsets[q+1] <= offsets[q] is left untouched.
 * No context and no allocation; asynchronous on `stream`.
 * Errors: SDTW_E_INVALID (B < 0, N < 1 without offsets, null pointers with
 * B > 0), SDTW_E_CUDA.
 */
sdtw_status sdtw_znormalize(const float* in, float* out, const int64_t* offsets, int32_t B, int32_t N,
                            void* stream);

/*
 * Reference codebook (paper Section 8, future work: quantise below fp16 to
 * uint8 with a codebook built from the reference, dividing the bulk of the
 * reference's value distribution evenly over the 256 codes and clamping
 * outliers to the extreme codes).  The bulk is mean +- sigmas * S of the
 * reference (population spread S); code k covers [lo + k step, lo + (k+1) step)
 * with step = 2 sigmas S / 256.  A forward on a context of dtype SDTW_U8 over
 * codes of the reference and of the queries then returns exact int32 costs
 * sum (code_x - code_y)^2, i.e. the squared-difference cost of the quantised
 * series in units of step^2; the end column follows the same tie rule.
 *
 * sdtw_codebook_fit: from the reference (device float [M], M >= 1) writes the
 *   codebook to params (device float [4]: lo, 1/step, step, 0) on `stream`.
 *   Statistics in double on one CTA.  A reference with zero spread gets
 *   step = 1 and lo = mean - 128.  sigmas > 0 (4 keeps 99.99% of a Gaussian).
 *   Errors: SDTW_E_INVALID (null pointers, M < 1, sigmas not positive and
 *   finite), SDTW_E_CUDA.
 * sdtw_codebook_encode: out[i] = clamp(floor((in[i] - lo) * (1/step)), 0, 255),
 *   the subtraction and the product each rounded to float (device float [n]
 *   in, device uint8 [n] out, params as written by sdtw_codebook_fit or by the
 *   caller).  Asynchronous on `stream`; no allocation.  Errors: SDTW_E_INVALID
 *   (n < 0, null pointers with n > 0), SDTW_E_CUDA.
 */
sdtw_status sdtw_codebook_fit(const float* ref, int64_t M, float sigmas, float* params, void* stream);
sdtw_status sdtw_codebook_encode(const float* in, int64_t n, const float* params, uint8_t* out, void* stream);

/* Largest batch sdtw_forward_noalloc accepts (its fixed device scratch holds
 * the query order for this many queries: 256 KiB per GPU). */
#define SDTW_NOALLOC_MAX_BATCH 65536

/*
 * sdtw_forward without a context and without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- code that runs while a CUDA graph is being
 * captured and must not allocate, plug-ins inside a host process that owns
 * all device memory through its own pool, real-time loops that may not touch
 * the allocator after start-up.  It runs the same persistent forward kernel
 * as sdtw_forward with a fixed plan (32 columns per thread, 4 warps per
 * query, 4 query rows per thread per step); its only scratch (work counter, status word, query order) is one
 * fixed-size array in the library's device memory, which every GPU that
 * loads the library keeps until the process exits.
 *   dtype     SDTW_F32, SDTW_I8, SDTW_U8 or SDTW_F16 (uniform batches only);
 *             ref, queries, offsets, B, N, M, cost and end as in sdtw_forward
 *             (device pointers owned by the caller); no pruning.
 *   stream    the launch stream; the device is the calling thread's current
 *             device.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the one array: calls that overlap on the GPU (on
 * different streams, or from several host threads) race and must not be
 * issued.  Each call clears the counter and status word itself.  Errors found
 * on the device are not reported (there is no context to read them from): a
 * ragged query longer than N gets the empty query's outputs (cost = +inf, or
 * INT32_MAX in the integer modes; end = -1).
 * Errors: SDTW_E_INVALID (bad sizes or null pointers as for sdtw_forward,
 * unknown dtype, B > SDTW_NOALLOC_MAX_BATCH), SDTW_E_UNSUPPORTED (N too long
 * for shared memory, offsets with SDTW_F16), SDTW_E_CUDA.
 */
sdtw_status sdtw_forward_noalloc(sdtw_dtype dtype, const void* ref, int64_t M, const void* queries,
                                 const int64_t* offsets, int32_t B, int32_t N, void* cost, int64_t* end,
                                 void* stream);

/* Synchronise `stream`, then return and clear the device status word: SDTW_OK,
 * SDTW_E_INVALID (a ragged query longer than N, an end index outside [0, M))
 * or SDTW_E_TIMEOUT.  SDTW_E_CUDA if the synchronisation itself failed. */
sdtw_status sdtw_last_device_status(sdtw_ctx* ctx, void* stream);

/* Text of the last CUDA error this context saw ("" if none); valid until the
 * next call on the context. */
const char* sdtw_last_error(sdtw_ctx* ctx);

/* Bytes of device workspace the context currently holds. */
size_t sdtw_workspace_bytes(sdtw_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SDTW_H */
