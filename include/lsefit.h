/*
 * lsefit.h -- C ABI of the GB300 least-squares polynomial fit library.
 *
 * The library computes the matricized least-square-errors polynomial fit of
 * Dasgupta, arXiv 1512.08017, Section II: for data pairs (x_i, y_i),
 * i = 1..n, the polynomial f(x) = a_0 + a_1 x + ... + a_m x^m minimising
 * Pi = sum_i [y_i - f(x_i)]^2 solves the normal equations
 *     sum_i x_i^j y_i = sum_k a_k sum_i x_i^(j+k),   j = 0..m,
 * written as A X = B with the Hankel matrix A[j][k] = S_{j+k},
 * S_k = sum_i x_i^k (k = 0..2m), B[j] = T_j = sum_i x_i^j y_i (k = 0..m) and
 * X = [a_0 .. a_m] (ascending order), solved by Gaussian elimination.
 *
 * Conventions shared by every entry point
 *  - Pointers named "device" must be device (or managed) memory of the
 *    current CUDA device; "host" pointers are ordinary host memory.  The
 *    point arrays x, y of lsefit_powersums may also be pinned, mapped host
 *    memory (the kernel then streams over the host link).
 *  - The caller owns every buffer.  The library allocates no device memory,
 *    frees nothing and keeps no state between calls other than a per-device
 *    cache of launch parameters.
 *  - Every call is asynchronous on `stream` (NULL = the legacy default
 *    stream).  The return value reports argument and launch errors only
 *    (LSEFIT_OK on success).  Data-dependent outcomes (too few points, a
 *    singular or non-finite system, a bad interval) are written per fit to a
 *    device int32 status array with the same codes; coefficients of a
 *    failed fit are NaN.
 *  - Workspaces are caller-provided scratch.  The single-series workspace
 *    must be zero-filled once before its first use; every call leaves it
 *    zeroed again, so it can be reused by later calls on the same stream
 *    (and by CUDA graph replays).  The batched and backward workspaces need
 *    no initialization (their first launch clears what must start at zero).
 *    Two calls that run at the same time must not share a workspace.
 *  - Affine map.  When an interval [lo, hi] is given, every abscissa is
 *    mapped to t = s (x - c) with c = (lo + hi) / 2, s = 2 / (hi - lo),
 *    computed in FP64 and rounded once to the precision the points are
 *    mapped in (FP32 for accum NAIVE/COMP, FP64 for accum F64).  The power
 *    sums are those of t (the "mapped basis"), and the solver returns both
 *    the mapped coefficients Xt (f = sum_k Xt_k t^k) and the coefficients X
 *    of x obtained by expanding (s (x - c))^k in FP64.  Without an interval,
 *    t = x.  The map is not in the paper; it keeps the Hankel system
 *    well-conditioned.
 *  - Degrees: 1 <= m <= LSEFIT_MAX_DEGREE.
 */
#ifndef LSEFIT_H
#define LSEFIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the same handle type). */
typedef struct CUstream_st* lsefit_stream_t;

#define LSEFIT_MAX_DEGREE 8
/* Highest degree of lsefit_fit_general in the Chebyshev basis with FP64 accumulation. */
#define LSEFIT_MAX_DEGREE_CHEBYSHEV 16
#define LSEFIT_ABI_VERSION 4

/* Return and status codes. */
enum {
    LSEFIT_OK = 0,
    LSEFIT_ERR_INVALID_ARG = 1,   /* host: a null pointer, size or enum out of range */
    LSEFIT_ERR_N_TOO_SMALL = 2,   /* per fit: n < m + 1 (the paper's n >= 2 only covers m = 1) */
    LSEFIT_ERR_SINGULAR = 3,      /* per fit: a GE pivot <= (m+1) * eps * max|A| (see lsefit_solve) */
    LSEFIT_ERR_NONFINITE = 4,     /* per fit: a power sum is Inf or NaN */
    LSEFIT_ERR_BAD_INTERVAL = 5,  /* per fit: interval not finite or hi <= lo */
    LSEFIT_ERR_WORKSPACE = 6,     /* host: workspace or plan buffer too small / misaligned */
    LSEFIT_ERR_CUDA = 7,          /* host: a CUDA runtime call or launch failed */
    LSEFIT_ERR_UNSUPPORTED = 8,   /* host: dtype/accum combination not provided */
    LSEFIT_ERR_SCRATCH_LIMIT = 9  /* host: request exceeds the static scratch of lsefit_fit_noalloc */
};

/* Storage type of x and y. */
enum { LSEFIT_F64 = 0, LSEFIT_F32 = 1, LSEFIT_BF16 = 2 };

/* Accumulation of the power sums.
 *  NAIVE: per-point powers and sums in FP32 (per-thread FP32 sums, then an
 *         exact-to-double-float reduction and an FP64 cross-block combine).
 *  COMP:  per-point powers in FP32; per-thread sums kept as compensated
 *         double-float (TwoSum) pairs, folded once per small register batch.
 *  F64:   per-point map, powers and sums in FP64 (the only mode for F64 data). */
enum { LSEFIT_ACCUM_NAIVE = 0, LSEFIT_ACCUM_COMP = 1, LSEFIT_ACCUM_F64 = 2 };

/* Number of doubles in one set of sums for degree m: S_0..S_2m then T_0..T_m. */
#define LSEFIT_SUMS_LEN(m) (3 * (m) + 2)

/* Human-readable name of a return/status code (static string). */
const char* lsefit_status_string(int code);

/* LSEFIT_ABI_VERSION of the loaded library. */
int lsefit_abi_version(void);

/* ------------------------------------------------------------------------
 * Single series
 * ------------------------------------------------------------------------ */

/* Bytes of workspace lsefit_powersums needs for any n on any device (an
 * upper bound, computable without a GPU). */
size_t lsefit_powersums_workspace_size(int m);

/*
 * lsefit_powersums -- the streaming pass that fills A and B (Section II:
 * the entries of A are the sums S_k = sum_i x_i^k, k = 0..2m, and of B the
 * sums T_k = sum_i x_i^k y_i, k = 0..m).
 *
 *  x, y       device (or mapped host) arrays of n points of `dtype`.  Any
 *             element alignment is accepted; 16-byte-aligned arrays with the
 *             same misalignment are streamed with 128-bit loads.
 *  n          number of points, n >= 0 (n = 0 gives zero sums).
 *  dtype      LSEFIT_F64 / LSEFIT_F32 / LSEFIT_BF16.
 *  m          degree, 1..LSEFIT_MAX_DEGREE.
 *  accum      LSEFIT_ACCUM_*; F64 data requires LSEFIT_ACCUM_F64.
 *  interval   device double[2] = {lo, hi} or NULL (t = x).
 *  sums       device double[3m+2], written: S_0..S_2m, T_0..T_m of t.
 *             S_0 = n exactly.  NaN everywhere if the interval is bad.
 *  map        device double[2] or NULL, written: {c, s} as used (the
 *             identity {0, 1} without an interval; NaN if bad).
 *  status     device int32[1] or NULL, written: LSEFIT_OK or
 *             LSEFIT_ERR_BAD_INTERVAL.
 *  workspace  device, >= lsefit_powersums_workspace_size(m) bytes,
 *             256-byte aligned, zero-filled before first use.
 * The result is bitwise reproducible for a given (n, dtype, m, accum,
 * device): per-block partials are combined in FP64 in a fixed order.
 */
int lsefit_powersums(const void* x, const void* y, int64_t n, int dtype, int m, int accum,
                     const double* interval, double* sums, double* map, int32_t* status,
                     void* workspace, size_t workspace_bytes, lsefit_stream_t stream);

/*
 * lsefit_solve -- Gaussian elimination of AX = B (Section II builds A with
 * A[j][k] = S_{j+k} and B[j] = T_j and solves the system by Gaussian
 * elimination), in FP64 with partial pivoting (first row of largest
 * magnitude), back-substitution, then the un-map of the coefficients.
 *
 *  sums    device double[count][3*m_sums+2], each row laid out as written by
 *          lsefit_powersums for degree m_sums.
 *  count   number of independent systems (>= 0).
 *  m_sums  degree the sums were accumulated for (row layout).
 *  m       degree to solve, 1 <= m <= m_sums: the sums of degree m_sums
 *          contain those of every lower degree, so one pass serves several.
 *  accum   the LSEFIT_ACCUM_* the sums were formed with.  It sets the
 *          singularity threshold: a pivot at or below (m+1) * eps * max|A|,
 *          eps = 2^-52 for FP64 accumulation and 2^-23 otherwise (FP32
 *          per-point powers leave pivots of that relative size in a
 *          rank-deficient system).
 *  map     device double[count][2] {c, s} or NULL (identity).
 *  X       device double[count][m+1]: coefficients of x, ascending.
 *  Xt      device double[count][m+1] or NULL: coefficients of t.
 *  status  device int32[count] or NULL: LSEFIT_OK, _N_TOO_SMALL (S_0 < m+1),
 *          _NONFINITE, _SINGULAR or _BAD_INTERVAL (map not finite or s = 0).
 */
int lsefit_solve(const double* sums, int64_t count, int m_sums, int m, int accum,
                 const double* map, double* X, double* Xt, int32_t* status, lsefit_stream_t stream);

/*
 * lsefit_solve_cholesky -- the alternative solver Section V names as future
 * work (a method other than Gaussian elimination): the Hankel normal matrix
 * is symmetric positive definite for distinct abscissae (A = V^T V), so
 * A = L L^T (Cholesky, FP64), then L w = B and L^T X = w, then the un-map.
 * About half the arithmetic of elimination and no pivoting.  A diagonal
 * pivot at or below (m+1) * eps * max|A| is reported as LSEFIT_ERR_SINGULAR.
 * Arguments, layouts and statuses as for lsefit_solve.
 */
int lsefit_solve_cholesky(const double* sums, int64_t count, int m_sums, int m, int accum,
                          const double* map, double* X, double* Xt, int32_t* status,
                          lsefit_stream_t stream);

/*
 * lsefit_fit -- the whole single-series fit in one launch: the streaming
 * pass of lsefit_powersums, then, in the block that completes the
 * reduction, the Gaussian elimination of Section II for every degree
 * d = m_lo..m from the same sums (the sums of degree m contain those of
 * each lower degree), one degree per lane, followed by the un-map.
 *  x..interval, workspace: as for lsefit_powersums.
 *  m_lo    lowest degree to solve, 1 <= m_lo <= m.
 *  X       device double[m-m_lo+1][m+1]: row r holds the x-basis
 *          coefficients of degree m_lo+r, zero beyond that degree.
 *  Xt      device, same shape, or NULL: t-basis coefficients.
 *  sums    device double[3m+2] or NULL.
 *  map     device double[2] or NULL.
 *  status  device int32[m-m_lo+1]: per-degree status as for lsefit_solve.
 */
int lsefit_fit(const void* x, const void* y, int64_t n, int dtype, int m, int m_lo, int accum,
               const double* interval, double* X, double* Xt, double* sums, double* map,
               int32_t* status, void* workspace, size_t workspace_bytes, lsefit_stream_t stream);

/*
 * lsefit_fit_noalloc -- lsefit_fit for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.
 *
 * Who needs it: a service that runs under a fixed device-memory budget and
 * forbids allocation after start-up, or a plugin host that hands its
 * plugins only their input and output buffers and offers no allocator.
 * Such callers pass inputs and outputs only; the reduction's scratch (one
 * ticket word and the per-block FP64 partials) lives in a static device
 * array inside the library.
 *  - Limit: the array has lsefit_fit_noalloc_scratch_bytes() = 819,456
 *    bytes, enough for every degree up to LSEFIT_MAX_DEGREE and the largest
 *    grid the library launches.  Every GPU that loads the library holds it
 *    until the process exits.  A request that would need more returns
 *    LSEFIT_ERR_SCRATCH_LIMIT (it cannot happen with valid degrees).
 *  - The first call on a device looks up the array's device address (with
 *    that device current) and caches it with the device's current driver
 *    context; make that first call before any stream capture.  A call in a
 *    new context of the device (after cudaDeviceReset, or after another
 *    library reset the primary context) looks the address up again, so
 *    its first call there must also precede any capture.
 *  - All calls share the one array.  Calls that overlap on the GPU (on
 *    different streams, or from different threads) race on it; serialise
 *    them.  The call clears the ticket word before its launch; the rest of
 *    the array keeps the previous call's contents and needs no clearing.
 *  - It allocates nothing: no cudaMalloc, cudaFree or allocating library
 *    routine; it issues one 256-byte cudaMemsetAsync and the fit's launch.
 *  Arguments, outputs and errors as for lsefit_fit, without the workspace.
 */
size_t lsefit_fit_noalloc_scratch_bytes(void);
int lsefit_fit_noalloc(const void* x, const void* y, int64_t n, int dtype, int m, int m_lo, int accum,
                       const double* interval, double* X, double* Xt, double* sums, double* map,
                       int32_t* status, lsefit_stream_t stream);

/* ------------------------------------------------------------------------
 * Generalised objective: per-point weights, Chebyshev basis
 * ------------------------------------------------------------------------ */

/* Basis of the fitted polynomial in the mapped variable t. */
enum {
    LSEFIT_BASIS_MONOMIAL = 0,  /* phi_k(t) = t^k (the paper's basis) */
    LSEFIT_BASIS_CHEBYSHEV = 1  /* phi_k(t) = T_k(t): T_0 = 1, T_1 = t, T_{k+1} = 2 t T_k - T_{k-1} */
};

/* Bytes of workspace lsefit_fit_general needs (any n, any device). */
size_t lsefit_fit_general_workspace_size(int m);

/*
 * lsefit_fit_general -- the fit of Section II for the objective
 * sum_i w_i [y_i - f(t_i)]^2 with f(t) = sum_k a_k phi_k(t) (Section V
 * leaves higher-order fits open; weights and the Chebyshev basis are this
 * library's generalisations).  Setting the derivatives by a_j to zero gives
 * G a = b with G[j][k] = sum w phi_j phi_k and b[j] = sum w phi_j y.  One
 * streaming pass accumulates the moments M_p = sum w phi_p(t) (p <= 2m) and
 * T_j = sum w phi_j(t) y (j <= m); G is M_{j+k} (monomial) or
 * (M_{j+k} + M_{|j-k|}) / 2 (Chebyshev: T_j T_k = (T_{j+k} + T_{|j-k|}) / 2).
 * G a = b is solved by Gaussian elimination with partial pivoting in FP64
 * (singular when a pivot is at or below (m+1) * eps * max|G|, eps as in
 * lsefit_solve).
 *
 *  x, y, w    device (or mapped host) arrays of n points of `dtype`; w may be
 *             NULL (every w_i = 1).  Weights are the caller's: zero weights
 *             drop points (and may leave G singular), negative weights give
 *             the stationary point of the objective, not a minimum.
 *  n, dtype, m, m_lo, accum, interval
 *             as lsefit_fit (degrees m_lo..m from the one pass; the map
 *             t = s (x - c) of [lo, hi] onto [-1, 1] or t = x without an
 *             interval).  dtype F64 requires accum F64.  m <= LSEFIT_MAX_DEGREE,
 *             or, in the Chebyshev basis with accum F64 (whose normal matrix
 *             stays well conditioned where the monomial one does not),
 *             m <= LSEFIT_MAX_DEGREE_CHEBYSHEV; a Chebyshev degree above
 *             LSEFIT_MAX_DEGREE with FP32 accumulation is
 *             LSEFIT_ERR_UNSUPPORTED.
 *  basis      LSEFIT_BASIS_MONOMIAL or LSEFIT_BASIS_CHEBYSHEV.
 *  X          device double[(m - m_lo + 1)][m + 1]: monomial coefficients of x
 *             (row d - m_lo for degree d, entries beyond d zero; NaN rows for
 *             failed fits).
 *  Xb         device double[(m - m_lo + 1)][m + 1] or NULL: coefficients a_k in
 *             the basis of t (Chebyshev coefficients with BASIS_CHEBYSHEV).
 *  sums       device double[3m + 2] or NULL: M_0..M_2m then T_0..T_m (without
 *             weights M_0 = n).
 *  map        device double[2] or NULL: (c, s) used.
 *  status     device int32[m - m_lo + 1]: per-degree status.
 *  workspace  device, >= lsefit_fit_general_workspace_size(m) bytes,
 *             256-byte aligned, zero-filled once before first use (each call
 *             leaves it zeroed).  One workspace serves one call at a time.
 * Returns LSEFIT_OK or a host error; w == NULL with the monomial basis runs
 * lsefit_fit itself (Xb is then the mapped-basis coefficients Xt).
 */
int lsefit_fit_general(const void* x, const void* y, const void* w, int64_t n, int dtype, int m, int m_lo,
                       int accum, int basis, const double* interval, double* X, double* Xb, double* sums,
                       double* map, int32_t* status, void* workspace, size_t workspace_bytes,
                       lsefit_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched ragged series (one persistent launch)
 * ------------------------------------------------------------------------ */

typedef struct lsefit_batch {
    const void* x;            /* device, concatenated points of all series, dtype */
    const void* y;            /* device, same layout as x */
    const int64_t* offsets;   /* device int64[num_series+1]; series s is [offsets[s], offsets[s+1]) */
    const int32_t* degree;    /* device int32[num_series], each in 1..m_max */
    const double* interval;   /* device double[num_series][2] {lo, hi}, or NULL (t = x) */
    int64_t num_series;
    int32_t m_max;            /* row stride of X/Xt is m_max+1, of sums 3*m_max+2 */
    int32_t dtype;            /* LSEFIT_F32 / LSEFIT_BF16 / LSEFIT_F64 */
    int32_t accum;            /* LSEFIT_ACCUM_* */
    int32_t basis;            /* LSEFIT_BASIS_MONOMIAL (0, the paper's fit) or LSEFIT_BASIS_CHEBYSHEV:
                                 the basis of t the fit is computed in (see lsefit_fit_general);
                                 Chebyshev needs accum COMP or F64 (F32/BF16 storage) or F64 */
} lsefit_batch;

/* Tuning of the batched schedule (0 in a field = library default). */
typedef struct lsefit_tuning {
    int32_t warp_max_len;     /* series up to this length are reduced by one warp */
    int32_t chunk_len;        /* longer series are cut into chunks of about this many points,
                                 each reduced by one block; a series with one chunk is finished
                                 by its block, others by the block that completes them last */
    int32_t block_threads;    /* reserved (the batched kernel runs 512 threads per block) */
    int32_t blocks_per_sm;    /* reserved (one persistent block per SM) */
    int32_t task_order;       /* order of the warp tasks in the plan (schedules 1 and 2):
                                 1 = longest first; 2 (0 = default) = grouped by degree
                                 when degrees are given, longest first within a degree */
    int32_t schedule;         /* how warps take warp tasks:
                                 1 = from one queue, in plan order;
                                 2 = fixed snake order (round r gives warp w task r*W + w,
                                     or r*W + W-1-w on odd rounds; W warps in the grid,
                                     numbered warp-major: w = warp * blocks + block, so a
                                     partly filled round is shared evenly by the SMs);
                                 3 (0 = default) = one queue per degree class, longest
                                     first; every block starts on a class (blocks shared
                                     out in proportion to the classes' points times a
                                     per-degree cost per point) and moves
                                     to the next class with tasks left when its class runs
                                     dry, so the warps of an SM run the code of one degree.
                                 In 1 and 3 a warp's first three tasks of its first queue
                                 are snake rounds over that queue's warps; later tasks
                                 come from an atomic counter. */
    int32_t reserved[2];
} lsefit_tuning;

/* Host-side schedule of one batch layout (built by lsefit_plan_build).  The two
 * task arrays must be copied to device memory by the caller, who stores the
 * device pointers in block_tasks / warp_tasks before calling lsefit_fit_batched. */
typedef struct lsefit_plan {
    int64_t num_series;
    int64_t total_points;
    int32_t n_block_tasks;    /* entries of block_tasks (4 int32 each) */
    int32_t n_warp_tasks;     /* entries of warp_tasks (4 int32 each) */
    int32_t n_split_series;   /* series cut into more than one chunk */
    int32_t m_max;
    lsefit_tuning tuning;     /* resolved values */
    int32_t grid;             /* persistent grid size */
    int32_t num_sms;
    const int32_t* block_tasks;  /* device int32[n_block_tasks][4]: series, chunk, nchunks, first task */
    const int32_t* warp_tasks;   /* device int32[n_warp_tasks][4]: series, first point (low and
                                    high 32 bits), length */
    int32_t class_begin[LSEFIT_MAX_DEGREE + 2];  /* schedule 3: warp tasks of degree class c
                                    (c = the degree, 0 = a degree outside 1..LSEFIT_MAX_DEGREE
                                    or no degrees given) are [class_begin[c], class_begin[c+1]) */
    int64_t class_points[LSEFIT_MAX_DEGREE + 1]; /* schedule 3: points of each class */
    int64_t warp_task_len;    /* the common length of every warp task, or 0 when they differ
                                 (lsefit_backward then splits their points evenly over its warps) */
} lsefit_plan;

/*
 * lsefit_plan_build -- split a batch layout into block tasks (series longer
 * than tuning.warp_max_len, cut into chunks) and warp tasks (the shorter
 * series).  Block tasks are ordered longest first.  Warp tasks are ordered
 * as tuning.schedule and tuning.task_order say: by degree class and longest
 * first within a class (schedule 3, the default), so that the warps of an SM
 * run the code of one degree while the longest series start first.  Host
 * only; no GPU needed.
 *  offsets_host  host int64[num_series+1] (nondecreasing, offsets[0] = 0).
 *  degree_host   host int32[num_series] or NULL (the same degrees the fits
 *                will use; only the order of the tasks depends on them).
 *  tuning        host, or NULL for defaults.
 *  num_sms       SM count of the target device (> 0).
 *  plan          host, written.
 *  block_tasks_host / warp_tasks_host  host buffers of capacity
 *                block_cap and warp_cap entries of 4 int32 each, written.
 *                A warp task's length must fit an int32 (warp_max_len <= 2^31-1).
 *                Pass NULL with zero capacity to query: plan->n_block_tasks
 *                and plan->n_warp_tasks are still set, and the call returns
 *                LSEFIT_ERR_WORKSPACE.
 */
int lsefit_plan_build(const int64_t* offsets_host, const int32_t* degree_host, int64_t num_series,
                      int m_max, const lsefit_tuning* tuning, int num_sms, lsefit_plan* plan,
                      int32_t* block_tasks_host, int64_t block_cap,
                      int32_t* warp_tasks_host, int64_t warp_cap);

/*
 * lsefit_plan_class_blocks -- the degree class each persistent block of
 * lsefit_fit_batched starts on under schedule 3 (the same sharing the fit
 * uses).  The `grid` blocks are shared out over the classes in proportion to
 * each class's points times the relative time per point of its degree; block
 * b starts on the class holding (b + 1/2) / grid of the total.  Class 0 (a
 * degree outside 1..LSEFIT_MAX_DEGREE) costs nothing, unless it holds every
 * point (a plan built without degrees): its blocks then cover the grid.  Host
 * only; no GPU needed.
 *  plan       host, from lsefit_plan_build.
 *  grid       persistent blocks (> 0; lsefit_fit_batched uses at most one per SM).
 *  cls_block  host int32[LSEFIT_MAX_DEGREE + 2], written: blocks
 *             [cls_block[c], cls_block[c+1]) start on class c (none when equal).
 * Returns LSEFIT_OK, or LSEFIT_ERR_INVALID_ARG for a NULL pointer or grid < 1.
 */
int lsefit_plan_class_blocks(const lsefit_plan* plan, int grid, int32_t* cls_block);

/* Bytes of workspace lsefit_fit_batched needs for `plan`. */
size_t lsefit_batched_workspace_size(const lsefit_plan* plan);

/*
 * lsefit_fit_batched -- every step of the fit (map, power sums, Hankel
 * system, Gaussian elimination, un-map; Section II) for each series of a
 * ragged batch, in one persistent launch.  Series are reduced by a warp or,
 * when longer, by one or more blocks (chunk partials combined in FP64 in a
 * fixed order by the block that completes the series), and each series is
 * solved right after its reduction.
 *  batch     host descriptor (device arrays inside).
 *  plan      host, from lsefit_plan_build for this layout, with device task arrays.
 *  X         device double[num_series][m_max+1]; row s holds degree[s]+1
 *            coefficients, the rest of the row is zero.
 *  Xt        device, same shape, or NULL: the coefficients in the basis of t
 *            (t^k, or T_k(t) when batch->basis is LSEFIT_BASIS_CHEBYSHEV).
 *  sums      device double[num_series][3*m_max+2] or NULL: S_0..S_2d, T_0..T_d
 *            of degree d = degree[s] at the start of the row (needed by
 *            lsefit_backward), rest zero; in the Chebyshev basis the moments
 *            sum T_p(t) and sum T_j(t) y.
 *  map       device double[num_series][2] or NULL: {c, s} used per series.
 *  status    device int32[num_series]: per-series status.
 *  workspace device, >= lsefit_batched_workspace_size(plan), 256-byte aligned;
 *            no initialization needed.
 */
int lsefit_fit_batched(const lsefit_batch* batch, const lsefit_plan* plan, double* X,
                       double* Xt, double* sums, double* map, int32_t* status,
                       void* workspace, size_t workspace_bytes, lsefit_stream_t stream);

/* ------------------------------------------------------------------------
 * Autotuning of the batched schedule
 * ------------------------------------------------------------------------ */

/* Largest candidate list lsefit_plan_autotune accepts. */
#define LSEFIT_AUTOTUNE_MAX_CANDIDATES 32

/* Copies the built-in candidate tunings into out[0 .. min(cap, count) - 1]
 * (out may be NULL) and returns their count: every series a warp task under
 * each of the three schedules, and the degree-class schedule with block tasks
 * above 4,096 or 65,536 points in chunks of 65,536 or 262,144.  Host only. */
int lsefit_autotune_candidates(lsefit_tuning* out, int cap);

/* Device buffer sizes lsefit_plan_autotune needs for one layout: *task_ints
 * = int32 elements of the largest task arrays over the candidates (block
 * tasks then warp tasks), *workspace_bytes = the largest batched workspace.
 * candidates NULL = the built-in list (n_candidates ignored).  Host only;
 * num_sms as for lsefit_plan_build. */
int lsefit_plan_autotune_sizes(const int64_t* offsets_host, const int32_t* degree_host, int64_t num_series,
                               int m_max, const lsefit_tuning* candidates, int n_candidates, int num_sms,
                               int64_t* task_ints, size_t* workspace_bytes);

/*
 * lsefit_plan_autotune -- measure candidate schedules of lsefit_fit_batched
 * on the caller's batch and return the fastest (the batched fit computes the
 * same Section II fit under every schedule; only the assignment of series to
 * warps and blocks changes).  For each candidate: the plan is built on the
 * host for the layout (offsets_host, degree_host), its task arrays copied
 * into tasks_device, one warm-up fit on `stream`, then the fit captured in a
 * CUDA graph (on a private stream) and `reps` replays of it timed with CUDA
 * events on `stream` -- the way a caller that replays graphs runs the fit;
 * timed as plain back-to-back calls, schedules can differ by less than the
 * noise while their graph replays do not.  Synchronous: returns after the
 * last measurement.  Outputs of
 * the trial fits land in X and status (their content is the last
 * candidate's fit).  Build the final plan with lsefit_plan_build(*best).
 *  batch          host descriptor of the device batch (as lsefit_fit_batched).
 *  offsets_host, degree_host   host copies of the layout (degree may be NULL).
 *  candidates     host array of n_candidates tunings, or NULL for the
 *                 built-in list (lsefit_autotune_candidates).
 *  reps           timed fits per candidate, >= 1.
 *  tasks_device   device int32[task_ints], 16-byte aligned (from
 *                 lsefit_plan_autotune_sizes); overwritten per candidate.
 *  workspace      device, >= the size lsefit_plan_autotune_sizes gives,
 *                 256-byte aligned.
 *  X, status      device outputs as for lsefit_fit_batched.
 *  best           host, written: the resolved tuning of the fastest candidate.
 *  ms_per_candidate  host float[n_candidates] or NULL: mean ms per fit.
 * Allocates no device memory of its own: two CUDA events, a stream and one
 * graph per candidate are created and destroyed.
 */
int lsefit_plan_autotune(const lsefit_batch* batch, const int64_t* offsets_host, const int32_t* degree_host,
                         const lsefit_tuning* candidates, int n_candidates, int reps, int32_t* tasks_device,
                         int64_t task_ints, void* workspace, size_t workspace_bytes, double* X,
                         int32_t* status, lsefit_stream_t stream, lsefit_tuning* best, float* ms_per_candidate);

/* CUDA driver version (cudaDriverGetVersion) the library sees, 0 if none;
 * part of the key under which measured tunings are cached. */
int lsefit_driver_version(void);

/* Bytes of workspace lsefit_range needs for `plan`. */
size_t lsefit_range_workspace_size(const lsefit_plan* plan);

/*
 * lsefit_range -- interval prepass: writes, per series, the smallest and
 * largest abscissa, for fits whose caller does not know the interval of the
 * affine map (not in the paper; the map keeps the Hankel system of
 * Section II well-conditioned).  Exact (minimum and maximum do not depend on
 * the order of evaluation); NaN points are ignored.  Reads x once (the
 * prepass costs the bytes of x on top of the fit).
 *  batch     as for lsefit_fit_batched (y, degree and interval unused).
 *  plan      from lsefit_plan_build for the layout, device task arrays set.
 *  interval  device double[num_series][2], written {lo, hi}; {NaN, NaN} for
 *            a series without a non-NaN point (its fit then reports
 *            LSEFIT_ERR_BAD_INTERVAL).
 *  workspace device, >= lsefit_range_workspace_size(plan), 256-byte aligned,
 *            zero-filled before first use (each call leaves it zeroed).
 */
int lsefit_range(const lsefit_batch* batch, const lsefit_plan* plan, double* interval,
                 void* workspace, size_t workspace_bytes, lsefit_stream_t stream);

/* Bytes of workspace lsefit_residuals needs for `plan`. */
size_t lsefit_residuals_workspace_size(const lsefit_plan* plan);

/*
 * lsefit_residuals -- fitted values and residual errors of a batched fit
 * (Section III judges a fit by its residuals e_i = y_i - f(x_i) and their sum
 * of squares, Table V).  One more pass over the points:
 *   SSE_s = sum_i r_i^2,  (V^T r)_{s,k} = sum_i t_i^k r_i  (k = 0..m),
 * with r_i = y_i - f(t_i), f(t) = sum_k Xt_k t^k by Horner's rule on the
 * mapped abscissae t_i = s (x_i - c).  V^T r vanishes at the least-squares
 * solution (the normal equations of Section II), so it measures how well a
 * fit satisfies them.  FP32 per point, compensated double-float sums, FP64
 * chunk combine; FP64 throughout for FP64 data.  For a fit in the Chebyshev
 * basis, f(t) = sum_k Xt_k T_k(t) (Clenshaw's recurrence) and
 * (V^T r)_{s,k} = sum_i T_k(t_i) r_i.
 *  batch     as for lsefit_fit_batched (interval unused: the map is `map`);
 *            basis as in the fit that produced Xt (LSEFIT_BASIS_MONOMIAL or
 *            LSEFIT_BASIS_CHEBYSHEV, else LSEFIT_ERR_INVALID_ARG).
 *  plan      the layout's plan, device task arrays set.
 *  Xt        device double[num_series][m_max+1] (from lsefit_fit_batched):
 *            coefficients in the mapped basis, monomial or Chebyshev.
 *  map       device double[num_series][2] {c, s} or NULL (identity).
 *  r         device array like y or NULL: per-point residuals (FP32 for
 *            F32/BF16 data, FP64 for F64 data).
 *  sse       device double[num_series]: NaN for a series whose fit failed.
 *  vtr       device double[num_series][m_max+1] or NULL: entries k <= m, NaN
 *            for a failed fit; entries k > m are 0; a degree outside
 *            1..m_max gives a row of NaN.
 *  workspace device, >= lsefit_residuals_workspace_size(plan), 256-byte
 *            aligned; no initialization needed.
 */
int lsefit_residuals(const lsefit_batch* batch, const lsefit_plan* plan, const double* Xt,
                     const double* map, void* r, double* sse, double* vtr, void* workspace,
                     size_t workspace_bytes, lsefit_stream_t stream);

/* ------------------------------------------------------------------------
 * Adjoint
 * ------------------------------------------------------------------------ */

/* Bytes of workspace lsefit_backward needs for `plan`. */
size_t lsefit_backward_workspace_size(const lsefit_plan* plan);

/*
 * lsefit_backward -- gradient of a loss L(X) with respect to the points,
 * given gX = dL/dX.  Not in the paper; derived from its normal equations
 * (Section II) by the chain rule, with the map constants held fixed:
 *   gt = M^T gX (M maps t-basis to x-basis coefficients);
 *   lambda solves A lambda = gt (A symmetric), in FP64;
 *   dL/dy_i = lambda(t_i);
 *   dL/dx_i = s * [lambda'(t_i) (y_i - f(t_i)) - lambda(t_i) f'(t_i)],
 *   with f(t) = sum_k Xt_k t^k; powers are recomputed, not stored.
 * Two launches: the lambda solves (one series per thread), then a second
 * pass over the points with the forward plan's tasks.
 *  batch     as for lsefit_fit_batched (same layout and degrees); basis must
 *            be LSEFIT_BASIS_MONOMIAL (else LSEFIT_ERR_UNSUPPORTED).
 *  plan      the forward's plan (same layout), device task arrays set.
 *  sums      device double[num_series][3*m_max+2] from lsefit_fit_batched.
 *  Xt        device double[num_series][m_max+1] from lsefit_fit_batched.
 *  map       device double[num_series][2] from lsefit_fit_batched, or NULL
 *            (identity map).
 *  gX        device double[num_series][m_max+1]; entries beyond a series'
 *            degree are ignored.
 *  dx, dy    device arrays laid out like x, y: FP32 for F32/BF16 data, FP64
 *            for F64 data.
 *  status    device int32[num_series], written: LSEFIT_OK, or the reason the
 *            adjoint system has no solution (_N_TOO_SMALL, _NONFINITE,
 *            _SINGULAR, _BAD_INTERVAL, _INVALID_ARG for a bad degree); such
 *            series get zero gradients.
 *  workspace device, >= lsefit_backward_workspace_size(plan), 256-byte aligned;
 *            no initialization needed.
 */
int lsefit_backward(const lsefit_batch* batch, const lsefit_plan* plan, const double* sums,
                    const double* Xt, const double* map, const double* gX, void* dx, void* dy,
                    int32_t* status, void* workspace, size_t workspace_bytes, lsefit_stream_t stream);

/* ------------------------------------------------------------------------
 * Diagnostics
 * ------------------------------------------------------------------------ */

/*
 * lsefit_check_reciprocal -- out[i] = the reciprocal 1/a[i] exactly as the
 * Gaussian eliminations and Cholesky factorisations of this library form it
 * (Newton-Raphson refinement of an FP32 seed; within about an ulp of the
 * IEEE quotient, not always correctly rounded).  Not in the paper; exposed so
 * that tests can hold it to its error bound.
 *  a, out  device double[n]; n >= 0.
 */
int lsefit_check_reciprocal(const double* a, double* out, int64_t n, lsefit_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LSEFIT_H */
