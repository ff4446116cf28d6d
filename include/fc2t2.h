/*
 * fc2t2.h -- C ABI of the GB300 (sm_103a) FC2T2 transform library.
 *
 * The library computes the multi-level uniform-grid Taylor transform of
 * Lange & Kutz, "FC^2T^2: The Fast Continuous Convolutional Taylor Transform"
 * (arXiv 2111.00110):
 *
 *     y_m  ~=  sum_n psi(p_n - q_m) w_n                       (Sec. 3, Eq. 1)
 *
 * for N sources p_n with weights w_n and M queries q_m in D = 2 or 3 dimensions,
 * by P2M -> M2M -> M2L -> L2L -> L2P on a uniform grid (Sec. 3), truncated at total
 * degree rho (Sec. 3, Eq. 2), and its adjoints with respect to w and p (Sec. 4.1).
 *
 * Conventions shared by every entry point:
 *  - Every array pointer is a DEVICE pointer owned by the caller, unless stated.
 *    Inputs are never modified.  Arrays are dense, row-major, float32, with C =
 *    fc2t2_plan_desc.channels weights per source (channel-major, as the paper's
 *    w of shape (B, C, N), Sec. 3, "How to use the implementation?"):
 *      p    [N][dim]   source positions        w     [C][N]    source weights
 *      q    [M][dim]   query positions         y     [C][M]    transform values
 *      ybar [C][M]     cotangent of y          wbar  [C][N]    dL/dw
 *      pbar [N][dim]   dL/dp (summed over the channels)
 *      qbar [M][dim]   dL/dq (summed over the channels)
 *    Channel c is the transform of the weights w[c]: the channels share the
 *    points (and their sort) and are otherwise independent.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *    Calls are asynchronous with respect to the host: they enqueue kernels on
 *    `stream` and return.  The only host synchronisation is in fc2t2_plan_create and,
 *    when check_domain is set, at the end of fc2t2_forward / fc2t2_backward.
 *  - A plan owns its operator tables and its device workspace; calls on one plan must
 *    not overlap in time (enqueue them on one stream).  Different plans are independent.
 *  - Every function returns a status code; nothing aborts or throws across the ABI.
 *    fc2t2_last_error() returns the text of the last failure on the calling thread.
 *  - Domain: [lo, hi)^dim.  The cell of a coordinate x at a level with n cells per
 *    dimension is decided in FP32: t = (x - lo) * (n / (hi - lo)), cell = floor(t),
 *    clamped to [0, n-1], each step rounded to FP32.  Points outside the domain are
 *    clamped into the edge cell, or rejected with FC2T2_ERR_DOMAIN when check_domain
 *    is set (the paper requires points inside the domain, Sec. 3.2).
 */
#ifndef FC2T2_H
#define FC2T2_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FC2T2_API __attribute__((visibility("default")))
#else
#define FC2T2_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FC2T2_OK = 0,
    FC2T2_ERR_INVALID_ARG = 1,   /* a NULL pointer, a size out of range, a bad descriptor */
    FC2T2_ERR_UNSUPPORTED = 2,   /* a valid request this build does not implement */
    FC2T2_ERR_OOM = 3,           /* device allocation failed in fc2t2_plan_create */
    FC2T2_ERR_DOMAIN = 4,        /* check_domain set and a point lies outside [lo, hi)^dim */
    FC2T2_ERR_CUDA = 5,          /* a CUDA runtime error (text in fc2t2_last_error) */
    FC2T2_ERR_TIMEOUT = 6        /* a bounded device-side wait gave up */
} fc2t2_status;

typedef enum {
    /* psi(x) = exp(-|x|^2 / (2 sigma^2)): the kernel of every experiment in the paper
     * (Sec. 3.3, written there as exp(-alpha |x|^2), alpha = 1 / (2 sigma^2)). */
    FC2T2_KERNEL_GAUSSIAN = 0,
    /* psi(x) = sum_a c_a x^a, coefficients in graded multi-index order (degree, then the
     * exponent of x_0 descending, then of x_1 descending); any degree.  For degree <= order
     * the series is exact.  The backward pass assumes psi(-x) = psi(x) (Sec. 4.1). */
    FC2T2_KERNEL_POLY = 1
} fc2t2_kernel;

/* Arithmetic of the M2L translation, the dominant step.  The tensor-core forms apply to 3D
 * plans; 2D plans run the CUDA-core M2L whatever is asked.  SEPARABLE needs the Gaussian kernel
 * and dim = 3 (plan creation returns UNSUPPORTED otherwise). */
typedef enum {
    FC2T2_M2L_FP32 = 0,          /* FP32 on the CUDA cores */
    FC2T2_M2L_TF32 = 1,          /* tcgen05 tensor cores, TF32 operands, FP32 accumulation */
    FC2T2_M2L_BF16 = 2,          /* tcgen05 tensor cores, BF16 operands, FP32 accumulation */
    FC2T2_M2L_TF32X3 = 3,        /* tcgen05, each operand split into TF32 high + low parts,
                                    three products (hi*hi + hi*lo + lo*hi): FP32 accuracy */
    FC2T2_M2L_BF16X3 = 4,        /* as TF32X3 with BF16 parts (~16 significant bits per operand,
                                    half the MMA instructions): within the FP32 error bar */
    FC2T2_M2L_SEPARABLE = 5,     /* FP32 on the CUDA cores, the Gaussian's derivative table
                                    factored per dimension: three one-dimensional passes per
                                    level (same operator and interaction lists, far fewer flops) */
    FC2T2_M2L_OCCUPIED = 6       /* FP32 on the CUDA cores, the direct operator over occupied
                                    cells only: a target cell with targets below it takes the
                                    terms of the source cells of its interaction list that hold
                                    sources (the others' moments are zero; the other targets'
                                    series are never read).  The same terms as FP32 for every
                                    series that is read; the work scales with the occupied cell
                                    pairs, not the grid (clustered points).  Any kernel, 2D and 3D.
                                    One persistent launch over a device work queue per call (per
                                    batched call for the plans of one dimension and order).  The
                                    local series of cells with no target are left unspecified, so
                                    fc2t2_expand and the ray calls take every cell as a target. */
} fc2t2_m2l_prec;

typedef struct fc2t2_plan_s *fc2t2_plan;

typedef struct {
    int dim;                     /* 2 or 3 */
    int grid;                    /* finest cells per dimension n: a power of two, 4 <= n <= 1024
                                    (levels = log2(n) - 1, coarsest level 4 cells; Sec. 3.2) */
    int order;                   /* rho, total-degree truncation, 1 <= rho <= 8 */
    fc2t2_kernel kernel;
    double sigma;                /* Gaussian width (> 0); ignored for FC2T2_KERNEL_POLY */
    const double *poly_coef;     /* HOST pointer, n_poly coefficients; copied at plan creation */
    int n_poly;                  /* must equal C(deg + dim, dim) for some degree deg */
    double lo, hi;               /* domain [lo, hi)^dim, hi > lo */
    int channels;                /* weights per source C, 1 <= C <= 4096 */
    fc2t2_m2l_prec m2l;
    int check_domain;            /* nonzero: reject points outside the domain (synchronises) */
    int64_t max_sources;         /* workspace bound on N (>= 0) */
    int64_t max_queries;         /* workspace bound on M (>= 0) */
    int fit;                     /* 0: M2L uses the kernel's Taylor coefficients about each cell-pair
                                    offset c (Sec. 3).  1: least-squares fitted ones (Sec. 3.1): the
                                    polynomial of total degree `order` closest to psi over the pair's
                                    separations c + [-h, h]^dim in the discrete L2 norm of the tensor
                                    Gauss-Legendre grid of order + 2 points per dimension (more
                                    accurate when cells are wide next to the kernel).  Not with the
                                    SEPARABLE M2L (UNSUPPORTED): the fit does not factor per
                                    dimension. */
    int tile;                    /* SEPARABLE M2L, finest level: the cells per CTA along a pass's
                                    axis (the line segment a CTA stages and computes).  0: 64 where
                                    a CTA's shared memory allows it, else the longest that does;
                                    16, 32 or 64: at most that many.  Other values: INVALID_ARG.  A
                                    tuning knob only (every value gives the same result); ignored by
                                    the other M2L forms. */
} fc2t2_plan_desc;

/* Build a plan: validate `desc`, build the M2L operator tables (the kernel's derivatives per
 * level and offset, or their least-squares fits) in FP64 on the host (Sec. 3: the kernel
 * derivatives are a once-per-plan preprocessing step, cf. Sec. 3.1; the M2M / L2L shifts need no
 * table), cast them to the M2L precision, and allocate the device workspace for
 * max_sources / max_queries points.  Synchronises the current device.
 * On success *out receives the plan; on failure *out is set to NULL.
 * A plan with C > 1 channels also holds C finest-level local series for fc2t2_expand.
 * Errors: INVALID_ARG (desc or out NULL, values out of range), UNSUPPORTED
 * (an M2L precision this build lacks for the kernel or dimension), OOM, CUDA. */
FC2T2_API fc2t2_status fc2t2_plan_create(const fc2t2_plan_desc *desc, fc2t2_plan *out);

/* Release a plan and its device memory.  NULL is accepted and ignored.  The caller
 * must make sure no call on the plan is still running on the device. */
FC2T2_API fc2t2_status fc2t2_plan_destroy(fc2t2_plan plan);

/* Forward transform (Sec. 3): y[c][m] = sum_n psi(p[n] - q[m]) w[c][n] through the series.
 * 0 <= N <= max_sources, 0 <= M <= max_queries; N = 0 gives y = 0.  y must not alias
 * an input.  The points are sorted once; each channel runs its own expansion.
 * Errors: INVALID_ARG, DOMAIN (check_domain), CUDA. */
FC2T2_API fc2t2_status fc2t2_forward(fc2t2_plan plan, void *stream,
                           const float *p, const float *w, int64_t N,
                           const float *q, int64_t M, float *y);

/* Backward pass of y = forward(p, w, q) for a cotangent ybar (Sec. 4.1):
 *   wbar[c][n] = sum_m psi(q[m] - p[n]) ybar[c][m]          (the transposed transform)
 *   pbar[n][i] = sum_c w[c][n] * d/dx_i sum_m psi(x - q[m]) ybar[c][m] at x = p[n]
 * computed as a second transform with sources q, weights ybar and targets p, whose local
 * series is evaluated (wbar) and differentiated (pbar) at p with the binning of p held
 * fixed.  Either output may be NULL to skip it.  The kernel must be even.
 * Errors: INVALID_ARG, DOMAIN (check_domain), CUDA. */
FC2T2_API fc2t2_status fc2t2_backward(fc2t2_plan plan, void *stream,
                            const float *p, const float *w, int64_t N,
                            const float *q, int64_t M, const float *ybar,
                            float *wbar, float *pbar);

/* Exact evaluation of Sec. 3, Eq. 1 by brute force, y[m] = sum_n psi(p[n] - q[m]) w[n], in
 * O(N M) on the device (one thread per query, compensated FP32 summation): the sum the series
 * approximates, for measuring a plan's truncation error on a sample of queries.  Uses
 * desc->dim, desc->kernel (Gaussian only) and desc->sigma; no plan.  Device arrays as in
 * fc2t2_forward, with desc->channels channels (w [C][N], y [C][M]); asynchronous on `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED (polynomial kernel), CUDA. */
FC2T2_API fc2t2_status fc2t2_direct(const fc2t2_plan_desc *desc, void *stream, const float *p, const float *w,
                                    int64_t N, const float *q, int64_t M, float *y);

/* Synchronise `stream` and report the device-side conditions raised on `plan`: TIMEOUT if a
 * bounded device-side wait (the staging of P2M, L2P or the M2L, or the tensor-core M2L's pipeline;
 * every such wait gives up after 0.2 s) gave up in any call since the last check (the outputs of
 * that call are then incomplete; the condition is cleared by this check), DOMAIN if
 * check_domain is set and the last call saw a point outside the domain.  Forward and backward
 * make the same check themselves when check_domain is set.  Errors: INVALID_ARG, CUDA, and the
 * two conditions above. */
FC2T2_API fc2t2_status fc2t2_plan_check(fc2t2_plan plan, void *stream);

/* fc2t2_backward after a forward call on the same plan with the same p, w, q arrays (same
 * pointers and sizes, contents unchanged -- what an autograd layer guarantees for its saved
 * inputs): reuses that call's sorts of p and q instead of sorting again (the cotangent is
 * gathered into the existing order of q).  The plan checks that its sorts were made from these
 * pointers and sizes and otherwise runs fc2t2_backward; it cannot see changed contents, which is
 * the caller's promise.  Same results and errors as fc2t2_backward. */
FC2T2_API fc2t2_status fc2t2_backward_reuse(fc2t2_plan plan, void *stream,
                                            const float *p, const float *w, int64_t N,
                                            const float *q, int64_t M, const float *ybar,
                                            float *wbar, float *pbar);

/* Gradient with respect to the query positions for a cotangent ybar:
 *   qbar[m][i] = sum_c ybar[c][m] * d/dx_i y_c(x) at x = q[m],   y_c(x) = the forward series of
 *                (p, w[c])
 * (the derivative of the local series, the binning of q held fixed -- the same reading as pbar).
 * Sec. 4.1 derives the adjoints for p and w; the query gradient is what the paper's accessor
 * exposes as the field's first partial derivatives (Sec. 3, "How to use the implementation?"),
 * and what a layer whose q comes from a network needs (Sec. 4's usage example); ybar = 1 gives
 * the field's gradient at q.  Recomputes the forward expansion.  qbar is [M][dim].
 * Errors: INVALID_ARG, DOMAIN (check_domain), CUDA. */
FC2T2_API fc2t2_status fc2t2_backward_q(fc2t2_plan plan, void *stream,
                                        const float *p, const float *w, int64_t N,
                                        const float *q, int64_t M, const float *ybar, float *qbar);

/* ---- The accessor (Sec. 3, "How to use the implementation?"): an expansion of (p, w) kept in
 * the plan and queried at continuous positions for the field's value, first partials and second
 * partials, at a list of points or on the meshgrid of per-axis coordinates (the paper's `vol`). */

/* What an evaluation returns per point and channel (K values):
 *   VALUE      K = 1        y_c(x)
 *   PARTIALS   K = dim      d y_c / dx_i, i = 0 .. dim-1
 *   PARTIALS2  K = dim (dim + 1) / 2   d^2 y_c / dx_i dx_k for i <= k, row-major:
 *              (00, 01, 11) in 2D, (00, 01, 02, 11, 12, 22) in 3D
 * The partials are those of the finest-level local series of the cell that holds x (the
 * binning rule of the conventions above), the same reading as pbar and qbar. */
typedef enum {
    FC2T2_EVAL_VALUE = 0,
    FC2T2_EVAL_PARTIALS = 1,
    FC2T2_EVAL_PARTIALS2 = 2
} fc2t2_eval;

/* Expand sources (p, w) (w [C][N]) into the plan: P2M, M2M, M2L and L2L of every channel (the
 * paper's `expand`).  The expansion stays in the plan for fc2t2_evaluate / fc2t2_evaluate_grid
 * until the next call of any transform entry point on the plan (forward, backward,
 * backward_reuse, backward_q, expand), which replaces it.  0 <= N <= max_sources; N = 0 gives
 * the zero field.  Errors: INVALID_ARG, DOMAIN (check_domain), CUDA. */
FC2T2_API fc2t2_status fc2t2_expand(fc2t2_plan plan, void *stream, const float *p, const float *w, int64_t N);

/* Evaluate the held expansion at M points q [M][dim]: out [C][M][K] (K from `what`).  The points
 * are sorted by cell for locality (0 <= M <= max_queries).  Errors: INVALID_ARG (no expansion
 * held, bad `what`, NULL array, M out of range), DOMAIN (check_domain), CUDA. */
FC2T2_API fc2t2_status fc2t2_evaluate(fc2t2_plan plan, void *stream, const float *q, int64_t M,
                                      fc2t2_eval what, float *out);

/* Evaluate the held expansion on the meshgrid of per-axis coordinates (the paper's `vol`):
 * axis is a HOST array of dim DEVICE pointers, axis[i] holding count[i] >= 0 coordinates
 * (count a HOST array of dim entries); the point (x_0, .., x_{dim-1}) = (axis[0][i_0], ..)
 * gives out[c][i_0][i_1]([i_2])[k] (last index fastest).  No point array is formed and no
 * sort is made: consecutive outputs step along the last axis.  Coordinates outside the domain
 * are clamped into the edge cell (check_domain is not applied here).  Errors: INVALID_ARG (no
 * expansion held, bad `what`, NULL array, negative count), CUDA. */
FC2T2_API fc2t2_status fc2t2_evaluate_grid(fc2t2_plan plan, void *stream, const float *const *axis,
                                           const int64_t *count, fc2t2_eval what, float *out);

/* ---- Ray integrals (Sec. 6, the integral-implicit layer, "Line Integral": a transform integrated
 * along rays, each box's series first restricted to the ray (line2poly, Sec. 5, "Line to polynomial"); the
 * building block of the paper's rendering and ray-sampled losses).  Rays are R records of 8
 * floats [R][8]: origin o (3), direction r (3), t0, t1; ray q covers x(t) = o + t r for t in
 * [t0, t1] (the parameter, not arc length, is integrated), clipped to the domain box [lo, hi)^3.
 * A ray is cut at the faces of the finest cells it crosses and each segment is integrated exactly
 * (up to rounding) with the series of the cell that holds it (the cell of its midpoint by the
 * binning rule), by Gauss-Legendre quadrature with ceil((order + 1) / 2) nodes.  3D plans only
 * (UNSUPPORTED otherwise). */

/* y[c][q] = int_{t0}^{t1} f_c(o_q + t r_q) dt,  f_c the series of (p, w[c]).  Any R >= 0 (no
 * workspace bound).  Errors: INVALID_ARG, UNSUPPORTED, DOMAIN (check_domain, for p), CUDA. */
FC2T2_API fc2t2_status fc2t2_ray_forward(fc2t2_plan plan, void *stream, const float *p, const float *w,
                                         int64_t N, const float *rays, int64_t R, float *y);

/* The adjoint of fc2t2_ray_forward for a cotangent ybar [C][R] (Sec. 6, "Line Integral JVP"): the
 * rays become the sources, each
 * segment adding ybar_q times its integral of the scaled monomials to its cell's moments (the
 * paper's ray2M), and the transform is evaluated and differentiated at the sources p:
 *   wbar[c][n] = sum_q ybar[c][q] int T(p_n, x_q(t)) dt,
 *   pbar[n][i] = sum_c w[c][n] d/dp_{n,i} (the same),  T the series' kernel.
 * The moments are summed with float atomics (rays in any order): results are reproducible to
 * rounding, not bit for bit.  Either output may be NULL.  Errors: as fc2t2_ray_forward. */
FC2T2_API fc2t2_status fc2t2_ray_backward(fc2t2_plan plan, void *stream, const float *p, const float *w,
                                          int64_t N, const float *rays, int64_t R, const float *ybar,
                                          float *wbar, float *pbar);

/* Batched forms (independent instances of uneven size, e.g. many small point sets): instance i
 * uses plans[i] and the device arrays p[i], w[i], q[i], y[i] (host arrays of device pointers,
 * each of n_inst entries) with N[i] sources and M[i] queries.  The call forks `stream` into one
 * stream per distinct plan (each plan owns one): a plan's instances run on its stream in order,
 * instances of different plans side by side (small instances fill the GPU together), and every
 * plan stream is joined back into `stream` before the call returns, so work enqueued on `stream`
 * afterwards sees all results.  The call is equivalent to n_inst calls of fc2t2_forward /
 * fc2t2_backward and can be captured into a CUDA graph by the caller (with check_domain off: the
 * fork / join become parallel branches).  Instances whose plan has the OCCUPIED M2L (one channel,
 * points on both sides, a plan that serves no other instance of the call) share the M2L: each runs
 * its sorts, P2M, occupancy and M2M on its plan's stream, then one persistent launch on `stream`
 * takes the occupied cell pairs of all of them (one launch per dimension and order, per 64
 * instances) from a device work queue, then each runs L2L and L2P on its stream.  Errors:
 * INVALID_ARG (n_inst < 0, a NULL array or plan), and any error of the single-instance call, for
 * the first failing instance (the remaining instances are not enqueued; the plan streams are
 * joined all the same). */
FC2T2_API fc2t2_status fc2t2_forward_batched(int n_inst, const fc2t2_plan *plans, void *stream,
                                             const float *const *p, const float *const *w, const int64_t *N,
                                             const float *const *q, const int64_t *M, float *const *y);
FC2T2_API fc2t2_status fc2t2_backward_batched(int n_inst, const fc2t2_plan *plans, void *stream,
                                              const float *const *p, const float *const *w, const int64_t *N,
                                              const float *const *q, const int64_t *M,
                                              const float *const *ybar, float *const *wbar, float *const *pbar);
/* fc2t2_backward_batched after fc2t2_forward_batched on the same plans and arrays (the batched
 * form of fc2t2_backward_reuse: an instance whose plan's sorts were made from these pointers and
 * sizes reuses them, the cotangent gathered into the existing order of q; the caller promises
 * unchanged contents).  Same results and errors as fc2t2_backward_batched. */
FC2T2_API fc2t2_status fc2t2_backward_batched_reuse(int n_inst, const fc2t2_plan *plans, void *stream,
                                                    const float *const *p, const float *const *w, const int64_t *N,
                                                    const float *const *q, const int64_t *M,
                                                    const float *const *ybar, float *const *wbar,
                                                    float *const *pbar);

/* What a plan computes per transform (forward or backward), for performance accounting. */
typedef struct {
    int levels;                  /* grid levels (finest n, coarsest 4 cells per dimension) */
    int coefficients;            /* P = C(order + dim, dim) per cell */
    int m2l_tensor_cores;        /* 1: the finest level's M2L runs on tcgen05 */
    double m2l_cell_pairs;       /* interacting (target, source) cell pairs over all levels */
    double m2l_useful_flops;     /* 2 x #{(k, b): |k| + |b| <= order} x m2l_cell_pairs */
    double m2l_issued_flops;     /* multiply-add work (x2) the M2L kernels issue, incl. the zeros
                                    inside the dense tensor-core blocks; = useful on CUDA cores.
                                    For the OCCUPIED form both figures are those of every cell
                                    pair: an upper bound (it runs the occupied pairs only, which
                                    the points decide) */
    int64_t device_bytes;        /* device memory owned by the plan */
    int m2l_classes_per_cta;     /* target parity classes one tensor-core CTA accumulates (1, 2 or
                                    4; 0 when the M2L runs on the CUDA cores) */
} fc2t2_plan_info;

/* Fill *info for `plan`.  Errors: INVALID_ARG (NULL argument). */
FC2T2_API fc2t2_status fc2t2_plan_query(fc2t2_plan plan, fc2t2_plan_info *info);

/* Pipeline stages, for fc2t2_profile_read. */
typedef enum {
    FC2T2_STAGE_SORT = 0,        /* binning + counting sort of sources and queries */
    FC2T2_STAGE_P2M = 1,
    FC2T2_STAGE_M2M = 2,
    FC2T2_STAGE_M2L = 3,
    FC2T2_STAGE_L2L = 4,
    FC2T2_STAGE_L2P = 5,         /* L2P, and the L2P gradient of the backward pass */
    FC2T2_STAGE_M2L_PACK = 6,    /* rewrite of the moments into the tensor-core operand layout */
    FC2T2_NUM_STAGES = 7
} fc2t2_stage;

/* Diagnostics, not part of the transform: while enabled, every call on `plan` records CUDA
 * events around each stage's kernels on the call's stream.  The plan always counts the
 * kernels it launches per stage.  Errors: INVALID_ARG (plan NULL), CUDA. */
FC2T2_API fc2t2_status fc2t2_profile_enable(fc2t2_plan plan, int enable);

/* Accumulated device time (ms, from the recorded events) and kernel launches per stage since
 * the last reset; either array may be NULL, each holds FC2T2_NUM_STAGES entries.  Waits for the
 * recorded events (synchronises with the streams they were recorded on).  reset != 0 clears
 * the accumulators after reading.  Errors: INVALID_ARG, CUDA. */
FC2T2_API fc2t2_status fc2t2_profile_read(fc2t2_plan plan, double *ms, int64_t *launches, int reset);

/* Forward transform that allocates no device memory and needs no plan.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc when they need
 * the transform -- for example code inside a framework that owns all device memory through its
 * own pool, or a real-time loop that must not allocate after start-up.
 * It computes exactly what fc2t2_forward computes for a plan built from `desc` (same kernels),
 * but keeps every intermediate (cell sort, coefficients of all levels, operator tables) in one
 * static device array inside the library, about 6.1 MB, which every GPU that loads the library
 * holds until the process exits.  Limits: Gaussian kernel, one channel, FP32 M2L,
 * grid^dim <= 4096 finest cells (64^2 or 16^3), 1 <= order <= 4, 0 <= N, M <= 65536; larger
 * requests return FC2T2_ERR_INVALID_ARG (or FC2T2_ERR_UNSUPPORTED for other kernels) before any
 * work is queued.  desc->max_sources / max_queries are ignored; desc->check_domain must be 0
 * (UNSUPPORTED otherwise: this path clamps points outside the domain into the edge cells and
 * never reports them, where a plan built with check_domain returns FC2T2_ERR_DOMAIN).
 * Every call looks up the array's device address on the current device (cudaGetSymbolAddress);
 * the first call on a device also loads the library's device code there, so make that first
 * call outside any stream capture.  The call queues its work on `stream` and returns without
 * waiting for it: the operator tables are built on the device inside the array, and no host
 * memory is read after the call returns.  All calls share the array and it keeps the last
 * call's contents (each call clears what must start from zero): calls whose work overlaps on
 * the GPU -- on different streams or from different threads -- race and give wrong results, so
 * issue them on one stream, one after the other.  Pointers as for fc2t2_forward.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
FC2T2_API fc2t2_status fc2t2_forward_noalloc(const fc2t2_plan_desc *desc, void *stream,
                                             const float *p, const float *w, int64_t N,
                                             const float *q, int64_t M, float *y);

/* Static text for a status code. */
FC2T2_API const char *fc2t2_status_string(fc2t2_status status);

/* Copy the message of the last failure on the calling thread into buf (NUL-terminated,
 * truncated to n bytes) and return its status (FC2T2_OK if none). buf may be NULL. */
FC2T2_API fc2t2_status fc2t2_last_error(char *buf, size_t n);

#ifdef __cplusplus
}
#endif

#endif /* FC2T2_H */
