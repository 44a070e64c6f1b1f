/*
 * spline_project.h -- C ABI of the GB300 spline x-ray projector.
 *
 * The library computes the x-ray transform of an image written as a sum of
 * shifted tensor-product B-splines, and its exact adjoint (backprojection),
 * over any list of lines ("Generalized Ray Tracing with Basis Functions for
 * Tomographic Projections", arXiv 2503.20907).
 *
 * Image model (eq. def_f, eq. xrtbasis, Sec. III.C):
 *   f(x) = sum_k c_k phi((x - x_k)/h),  phi(x1, x2) = beta^n(x1) beta^n(x2),
 *   node k = (i, j) at x_k = (cx + (i - (nx-1)/2) h, cy + (j - (ny-1)/2) h),
 *   beta^n the centred B-spline of degree n = 0..3 (or the 3-direction
 *   box-spline of Sec. III.D, see sp_basis).
 * Lines (eq. rayparam): {t theta + y theta^perp}, theta = (cos, sin),
 *   theta^perp = (sin, -cos).
 * Forward (eq. xray with eq. xrtbasis, discretised operator of Sec. IV.A):
 *   p_m = h * sum_k c_k phi_{theta_m}((y_m - <x_k, theta_m^perp>)/h)
 * Adjoint (Sec. II.B, "exactly matched"):
 *   c'_k = h * sum_m p_m phi_{theta_m}((y_m - <x_k, theta_m^perp>)/h)
 * phi_theta is the exact x-ray transform of phi (Prop. 1, eq. xsa).
 *
 * Conventions shared by every entry point:
 *   - Array pointers are DEVICE pointers owned by the caller; the library keeps
 *     no reference to them after the call returns.
 *   - Coefficient images are float32 [ny][nx], row j (x2) major, i (x1) fastest.
 *   - Sinograms are float32 [m]; for the structured kinds the ray index is
 *     view * n_det + bin (view-major, bin fastest).
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream) and runs asynchronously; the call returns after enqueueing.
 *   - Argument errors detectable on the host return SP_EINVAL before anything
 *     is enqueued.  A CUDA error returns SP_ECUDA.  sp_last_error() gives a
 *     message for the last failing call on the calling thread.
 *   - Internal workspace (per-line records and footprint tables) is cached per
 *     device and grows on demand; sp_release_workspace() frees it.  Calls on
 *     one device must not overlap from several host threads.
 *   - Lines that miss the support of every basis give 0.  Lines with
 *     non-finite parameters give unspecified values.
 */
#ifndef SPLINE_PROJECT_H
#define SPLINE_PROJECT_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sp_status {
    SP_OK = 0,
    SP_EINVAL = -1,        /* invalid argument (checked on the host) */
    SP_ENOMEM = -2,        /* device allocation of the workspace failed */
    SP_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed */
    SP_EUNSUPPORTED = -5   /* valid request that this build does not support */
} sp_status;

/* Basis functions (Sec. III.D).
 *   SP_BASIS_BSPLINE: phi(x1, x2) = beta^n(x1) beta^n(x2), the tensor-product
 *     B-spline of degree n = grid.degree (0..3).
 *   SP_BASIS_BOX3: the 3-direction box-spline with directions e1, e2,
 *     e1 + e2 and centred unit rectangles as factors: the piecewise-linear
 *     hat M(x) = max(0, 1 + min(x1, x2, 0) - max(x1, x2, 0)) on the
 *     triangulation by x1, x2, x1 - x2 in Z (grid.degree must be 1).  Its
 *     x-ray transform is the convolution of three boxes of widths |sin|,
 *     |cos| and |sin - cos| (|<theta^perp, u_d>|, Prop. 1 with D = 3). */
typedef enum sp_basis {
    SP_BASIS_BSPLINE = 0,
    SP_BASIS_BOX3 = 1
} sp_basis;

/* Coefficient grid: nx x ny nodes, spacing h > 0, centre (cx, cy), basis. */
typedef struct sp_grid {
    int32_t nx, ny;        /* 1 <= nx, ny <= 16384 */
    int32_t degree;        /* B-spline degree n, 0..3 (1 for SP_BASIS_BOX3) */
    int32_t basis;         /* sp_basis */
    float h;               /* grid spacing */
    float cx, cy;          /* grid centre */
} sp_grid;

typedef enum sp_lines_kind {
    SP_LINES_THETA_Y = 0,  /* line m = (theta[m], y[m]) (eq. rayparam) */
    SP_LINES_POINTS = 1,   /* infinite line through src[m] and dst[m] */
    SP_LINES_PARALLEL = 2, /* line (v, j) = (view[v], det0 + j*ddet) */
    SP_LINES_FAN = 3       /* flat-detector fan beam, see below */
} sp_lines_kind;

/*
 * A line list.  Fields not used by `kind` are ignored.
 *
 * SP_LINES_FAN: for view v with source angle beta = view[v], the source is at
 * dso*(cos beta, sin beta); the detector is the line through
 * -dod*(cos beta, sin beta) with direction (-sin beta, cos beta), and bin j is
 * centred at offset det0 + j*ddet along it.  Ray (v, j) joins the source to
 * the centre of bin j.  (The paper's fan geometry is not specified in closed
 * form; this is the flat-detector fan of its experiments, Sec. IV.B/IV.C.)
 */
typedef struct sp_lines {
    int32_t kind;          /* sp_lines_kind */
    int32_t n_view;        /* PARALLEL, FAN: number of views (>= 1) */
    int32_t n_det;         /* PARALLEL, FAN: bins per view (>= 1) */
    int32_t reserved;      /* must be 0 */
    int64_t m;             /* THETA_Y, POINTS: number of lines (>= 0);
                              PARALLEL, FAN: 0 or n_view*n_det */
    const float *theta;    /* THETA_Y: device [m] angles (radians) */
    const float *y;        /* THETA_Y: device [m] offsets */
    const float *src;      /* POINTS: device [m][2] first point */
    const float *dst;      /* POINTS: device [m][2] second point (!= src) */
    const float *view;     /* PARALLEL: device [n_view] line angles;
                              FAN: device [n_view] source angles */
    float det0, ddet;      /* PARALLEL, FAN: offset of bin 0 and bin spacing */
    float dso, dod;        /* FAN: source-origin and origin-detector distances */
} sp_lines;

/* Number of lines described by `lines` (-1 if the description is invalid). */
int64_t sp_lines_count(const sp_lines *lines);

/*
 * Forward projection (Sec. II, Algorithm 2's output for every line):
 *   sino[m] = h * sum_k coef[k] * phi_{theta_m}((y_m - <x_k, theta_m^perp>)/h).
 * coef: device float [ny][nx] (read only).  sino: device float [m] (written).
 */
sp_status spline_project_fwd(const sp_grid *grid, const float *coef,
                             const sp_lines *lines, float *sino, void *stream);

/*
 * Adjoint (backprojection), the exact transpose of spline_project_fwd
 * (Sec. II.B): coef_out[k] = h * sum_m sino[m] * phi_{theta_m}(...).
 * sino: device float [m] (read only).  coef_out: device float [ny][nx],
 * overwritten (not accumulated into).
 */
sp_status spline_project_adj(const sp_grid *grid, const float *sino,
                             const sp_lines *lines, float *coef_out, void *stream);

/*
 * Line setup on its own (the first step of the hot path, eq. rayparam):
 * writes theta_out[m] and y_out[m] (device float) for every line, with
 * theta in (-pi, pi] the direction angle and y = <P, theta^perp> for a point
 * P of the line.  Either output may be NULL.
 */
sp_status spline_lines_expand(const sp_lines *lines, float *theta_out, float *y_out,
                              void *stream);

/*
 * The footprint phi_theta(yt) on the unit grid (Prop. 1, eq. xsa) as the
 * projector evaluates it: out[r] = phi_{theta[r]}(yt[r]) for r < count, for
 * the basis and degree of *grid (its other fields are not used).
 * theta, yt, out: device float [count].  For testing and inspection.
 */
sp_status spline_footprint_eval(const sp_grid *grid, int64_t count, const float *theta,
                                const float *yt, float *out, void *stream);

/*
 * The nonzero (line, node) pairs the projector visits, i.e. the pairs with
 * |y~| < w, w = (n+1)(|cos|+|sin|)/2 (closed for degree 0 along an axis).
 * counts: device int32 [m], written with the number of pairs of each line.
 * If offsets != NULL (device int64 [m], exclusive prefix sums of counts) and
 * nodes != NULL, nodes[offsets[m] ...] receives each line's node indices
 * j*nx + i, in the projector's own order (unordered within a line).
 */
sp_status spline_visited(const sp_grid *grid, const sp_lines *lines, int32_t *counts,
                         const int64_t *offsets, int32_t *nodes, void *stream);

/*
 * Plans.  A plan keeps the per-line records and footprint tables of one
 * (grid, lines) pair in its own device memory, so that repeated projections
 * (iterative reconstruction, autograd) skip the setup.  The steps of one pass
 * of the projector are then separate calls:
 *   spline_plan_prepare  line setup (eq. rayparam) and footprint tables
 *                        (Prop. 1, eq. xsa), for THETA_Y and POINTS lists
 *                        the strip kernels' line order, and, where the plan keeps
 *                        them, the row records: for every major-axis row of
 *                        every line, the position of its run of nodes and
 *                        the argument of its footprint polynomials (the
 *                        traversal of Algorithm 2), sorted by polynomial;
 *   spline_plan_fwd      forward projection (Algorithms 1-2);
 *   spline_plan_adj      adjoint.
 * Row records (spline_plan_set_records) are for plans that project many
 * times per prepare (iterative reconstruction): the projections then read
 * them instead of recomputing the rows, with the same results (the forward
 * bit for bit), at the price of a longer prepare and about 8 bytes per line
 * and row of device memory (2.7 GB for 720 x 768 lines on a 512 x 512
 * grid).  New plans keep none.
 * spline_plan_create allocates (cudaMalloc on the current device) and copies
 * the descriptors but enqueues no work; the device arrays that `lines` points
 * to must stay valid until the last spline_plan_prepare on the plan has run.
 * A plan is used on the device that was current at creation.  Calls on one
 * plan must be ordered (same stream, or synchronised).
 */
typedef struct sp_plan sp_plan;

sp_status spline_plan_create(const sp_grid *grid, const sp_lines *lines, sp_plan **plan);
sp_status spline_plan_prepare(sp_plan *plan, void *stream);
sp_status spline_plan_fwd(const sp_plan *plan, const float *coef, float *sino, void *stream);
sp_status spline_plan_adj(const sp_plan *plan, const float *sino, float *coef_out, void *stream);
/*
 * Least squares with the plan's projector A: conjugate gradients on the
 * normal equations A^T A x = A^T b (CGLS), the reconstruction step of Sec. V,
 * where the system is solved by conjugate gradients.  With x_0 the initial x:
 *   r = b - A x_0;  s = A^T r;  p = s;  gamma = <s, s>
 *   for k = 1..iters:
 *     q = A p;  alpha = gamma / <q, q>;  x += alpha p;  r -= alpha q;
 *     s = A^T r;  gamma' = <s, s>;  p = s + (gamma' / gamma) p;  gamma = gamma'.
 * x_k minimises ||b - A x|| over x_0 + span{A^T r_0, (A^T A) A^T r_0, ...}.
 *   b           device float32 [m], the data (not modified).
 *   x           device float32 [ny][nx]: x_0 on entry, x_iters on return.
 *               Must not overlap b.
 *   iters       number of iterations, >= 0 (0 only evaluates gamma_0).
 *   gamma_hist  NULL, or device double [iters + 1]: gamma_k =
 *               ||A^T (b - A x_k)||^2 for k = 0..iters; the relative residual
 *               of the normal equations is sqrt(gamma_k / gamma_0).
 * Vectors are FP32; dot products accumulate in FP64 with a fixed summation
 * order (results are reproducible run to run).  A step whose <q, q> or gamma
 * is 0 leaves x unchanged.  Scalars stay on the device: the call enqueues the
 * whole solve on `stream` without waiting.  Workspace (2 m + 2 ny nx floats)
 * is allocated in the plan on first use (cudaMalloc, which synchronises the
 * device) and freed with the plan.
 */
sp_status spline_plan_cgls(sp_plan *plan, const float *b, float *x, int32_t iters,
                           double *gamma_hist, void *stream);
/*
 * Kernel choice of a plan, per direction: 0 = automatic (the strip kernels
 * for degree >= 1, else the general kernels; THETA_Y and POINTS lists reach
 * the strip kernels through an order that prepare sorts them into: by major
 * axis, direction and offset, so that 32 consecutive lines are nearly
 * parallel neighbours),
 * 1 = strip kernels where they apply (ray-driven: the adjoint scatters into
 * shared-memory strips), 2 = general kernels (warp per line; the adjoint
 * scatters with global atomics), and for the adjoint only 3 = pixel-driven
 * gather (thread per node over every view, no atomics; PARALLEL and FAN
 * lines of degree >= 1, else as 0).  All give the same results within
 * rounding (no paper counterpart: this is an implementation choice).
 */
sp_status spline_plan_set_paths(sp_plan *plan, int32_t fwd_path, int32_t adj_path);
/*
 * Autotuner: times the forward with both kernel families and the adjoint
 * with all three (strip scatter, warp-per-line scatter, pixel-driven gather)
 * on the caller's data (coef: device [ny][nx], sino: device [m]; neither is
 * modified; outputs go to temporary buffers) and keeps the fastest per
 * direction (spline_plan_set_paths).  Writes the choices to *fwd_path and
 * *adj_path and, if ms != NULL, the mean times ms[0..4] = forward strip,
 * forward general, adjoint strip, adjoint general, adjoint gather (0 when
 * not measured).
 * Synchronises the stream; allocates and frees m + ny*nx floats.
 */
sp_status spline_plan_autotune(sp_plan *plan, const float *coef, const float *sino, void *stream,
                               int32_t *fwd_path, int32_t *adj_path, float *ms);

/*
 * Batches: several independent instances (each its own grid, basis, degree
 * and line list, sizes free) projected together.  Instances on the strip
 * kernels (any line list; degree >= 1 unless the path is set or
 * tuned to them; path not forced to the
 * general kernels) share one persistent launch that takes chunks of 32
 * lines of any of them from a work queue; the others are forked over 8
 * internal streams; all are joined on the caller's stream.  The first call
 * for a given set of data pointers records that as a CUDA graph (after
 * uploading the queue, which synchronises the device), later calls with the
 * same pointers replay it (one launch).
 *   spline_batch_create   count >= 1 instances from grids[count], lines[count]
 *                         (each as spline_plan_create; all pointers of
 *                         lines must stay valid while the batch is prepared)
 *   spline_batch_prepare  line setup and tables of every instance
 *   spline_batch_fwd      sino[i] = A_i coef[i] for every i; coef and sino
 *                         are HOST arrays of count DEVICE pointers
 *   spline_batch_adj      coef_out[i] = A_i^T sino[i]
 *   spline_batch_autotune spline_plan_autotune on each instance, then, per
 *                         direction, the whole batch timed with those
 *                         choices against the strip kernels wherever they
 *                         apply (the faster is kept); paths (NULL or host
 *                         int32 [2 count]) receives the forward and adjoint
 *                         choice of each; uses temporary device buffers
 *                         (cudaMalloc) for the outputs; drops recorded graphs
 *   spline_batch_destroy  frees everything (synchronises the device)
 * Calls on one batch must be ordered; capture of the graph needs the
 * device not to be capturing on the calling thread already.
 */
typedef struct sp_batch sp_batch;
sp_status spline_batch_create(int32_t count, const sp_grid *grids, const sp_lines *lines, sp_batch **batch);
sp_status spline_batch_prepare(sp_batch *batch, void *stream);
sp_status spline_batch_fwd(sp_batch *batch, const float *const *coef, float *const *sino, void *stream);
sp_status spline_batch_adj(sp_batch *batch, const float *const *sino, float *const *coef_out, void *stream);
sp_status spline_batch_autotune(sp_batch *batch, const float *const *coef, const float *const *sino,
                                void *stream, int32_t *paths);
/* Number of instances (-1 if batch is NULL). */
int32_t spline_batch_count(const sp_batch *batch);
/* Number of instances that the last recorded forward (adjoint != 0: adjoint)
 * graph runs through the work queue (-1 if batch is NULL). */
int32_t spline_batch_queued(const sp_batch *batch, int32_t adjoint);
sp_status spline_batch_destroy(sp_batch *batch);

/* Number of lines of the plan (-1 if plan is NULL). */
int64_t spline_plan_lines(const sp_plan *plan);
/* Device bytes of the plan's row records (0: the plan keeps none and its
 * projections traverse the rows themselves; -1 if plan is NULL). */
int64_t spline_plan_record_bytes(const sp_plan *plan);
/*
 * keep = 1: the plan keeps row records, written by every later
 * spline_plan_prepare (the plan must be prepared again before it projects);
 * SP_EUNSUPPORTED unless the degree is >= 1, SP_ENOMEM if they would take more than a quarter of the device's
 * free memory or 16 GiB (cudaMalloc).  keep = 0 frees them (synchronises the
 * device).
 */
sp_status spline_plan_set_records(sp_plan *plan, int32_t keep);
/*
 * Diagnostics of the plan's forward projections so far (synchronises):
 * slow_rows = rows whose run of nodes fell outside the shared-memory window
 * staged for their group of lines and were read from global memory instead
 * (results are the same; only speed differs).
 */
sp_status spline_plan_stats(const sp_plan *plan, int64_t *slow_rows);
/* Free the plan and its device memory (synchronises the device first). */
sp_status spline_plan_destroy(sp_plan *plan);

/*
 * Forward projection that allocates nothing (this entry point has no
 * counterpart in the paper; it gives the same result as spline_project_fwd,
 * always through the warp-per-line kernels: the strip kernels need a
 * transposed image that the fixed scratch does not hold, so it runs at that
 * path's speed, not at the strip path's).
 *
 * For callers that cannot let the library allocate device memory: programs
 * that reserve the device's memory up front for their own pool, where a
 * foreign cudaMalloc fails or fragments it, and latency-bound pipelines that
 * cannot take the device-wide synchronisation of cudaFree or of growing a
 * cached workspace.  Its scratch (per-line records and footprint tables) is a
 * fixed 48 MiB array in the library's device memory, which every GPU that
 * loads the library holds until the process exits.  Calls neither cudaMalloc
 * nor cudaFree.
 *
 * Limit: 64 bytes per line plus 1312 bytes per footprint table (one per line;
 * one per view for SP_LINES_PARALLEL) must fit in 48 MiB, i.e. about 36,000
 * lines with their own tables; larger lists return SP_EINVAL with the byte
 * count in sp_last_error().  The first call with a nonempty line list on a
 * device looks up the array's device address (cudaGetSymbolAddress); under
 * lazy module loading (CUDA_MODULE_LOADING=LAZY, PyTorch's default) that
 * lookup is also when the CUDA driver loads the array and reserves its 48 MiB on
 * that device (and the kernels' code).  So make one such call first (a
 * one-line list suffices), before the rest of the device memory goes to the
 * caller's own pool and before any stream capture; later calls take no
 * device memory.  All calls on a device share the one array, and every call
 * rewrites the part it uses before reading it: calls that overlap on the GPU
 * (other streams, or before the previous call's kernels finished) race.
 * Arguments, outputs and errors as spline_project_fwd.
 */
sp_status spline_project_fwd_noalloc(const sp_grid *grid, const float *coef,
                                     const sp_lines *lines, float *sino, void *stream);

/* Free the cached workspace of the current device (synchronises the device). */
sp_status sp_release_workspace(void);

/* Message of the last failing call on this thread ("" if none). */
const char *sp_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int32_t sp_version(void);

/*
 * FP32 throughput of the current device, measured (the denominator of the
 * projector's roofline; no paper counterpart): a kernel of independent
 * fused multiply-add chains on every SM, as scalar fma.rn.f32 (packed = 0)
 * or packed fma.rn.f32x2 (packed = 1), timed with CUDA events on `stream`
 * after one warm-up launch (best of three).  *tflops receives the FLOP/s
 * (an FMA counts 2) in units of 1e12, *ms (if not NULL) the time of one
 * launch.  Synchronises the stream; uses the cached workspace (1 float per
 * thread of the launch).
 */
sp_status sp_fp32_peak(int32_t packed, double *tflops, float *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SPLINE_PROJECT_H */
