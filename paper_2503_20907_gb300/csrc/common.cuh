// Internal declarations shared by the CUDA translation units of the projector.
//
// Geometry of one line in grid units.  For node (i, j) the offset of the line
// is y~ = (y - <x_k, theta^perp>)/h (Sec. IV.A), and u = y~ + w with
// w = (n+1)(a+b)/2 the half-width of the support of phi_theta, a = max(|cos|,
// |sin|), b = min(|cos|, |sin|) (Prop. 1 with D = 2).  A pair is nonzero iff
// u is in (0, 2w).
//
// Rows follow the major axis of the line's direction (x2 for "mainly
// vertical" lines, x1 otherwise, as in Algorithm 2) and columns the minor
// axis, so that along a row u moves by +-a per column and by rho (|rho| = b)
// per row.  In row r the nonzero columns form one run of at most K <= 2(n+1)
// consecutive columns (Lemma 1 with K = n neighbours each side of the crossed
// cells).  Writing u_0 in (0, a] for the smallest u of the run, candidate i of
// the run sits at u_0 + i a.
//
// Footprint tables.  phi_theta is a piecewise polynomial of degree 2n+1 with
// breakpoints p a + q b (p, q = 0..n+1) in u.  As a function of u_0, the
// value at candidate i, phi(u_0 + i a), changes polynomial only where u_0
// crosses one of the points s_q = (q b) mod a, so (0, a] splits into at most
// n+2 intervals (s_sigma, s_{sigma+1}].  The table holds, for every interval
// sigma and candidate i, the polynomial T[sigma][i](t) = phi(s_sigma + i a + t)
// in t = u_0 - s_sigma: evaluating a pair is one Horner scheme of degree 2n+1.
// It is built per line (per view for parallel beams) in FP32, stably:
//   - derivatives n+1..2n+1 at each breakpoint directly from
//     phi^{(n+1+e)}(u) = a^{-(n+1)} sum_p (-1)^p C(n+1,p) B^{(e)}(u - p a),
//     B the B-spline of width (n+1) b (no cancellation);
//   - derivatives 0..n carried from piece to piece by Taylor shifts whose
//     lengths are formed from the integer breakpoint coordinates (p, q),
//     walking only up to the centre of the support, the other half by the
//     symmetry phi(u) = phi(2w - u).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/spline_project.h"

namespace spx {

constexpr int kMaxDeg = 3;
constexpr int kMaxM = kMaxDeg + 1;            // n + 1
constexpr int kMaxSig = kMaxM + 1;            // u_0 intervals
constexpr int kMaxK = 2 * kMaxM;              // candidate slots per row
constexpr int kNC = 2 * kMaxDeg + 2;          // coefficients of one polynomial
constexpr int kSigStride = kMaxK * kNC;       // 64 floats
constexpr int kTabHead = 8;                   // s_1..s_m (padded with FLT_MAX), a, b
constexpr int kTabMode = 5;                   // head slot of the footprint kind (TabMode)
constexpr int kTabA = 6;                      // head slot of the a the table was built with
constexpr int kTabB = 7;                      // head slot of its b
constexpr int kTabFloats = kTabHead + kMaxSig * kSigStride;   // 328 floats
constexpr float kBMin = 1e-7f;                // below this b is taken as 0 (Dirac)

// Offset of the polynomial of (interval sg, candidate i) in a table: its
// kNC coefficients (ascending powers of t) are contiguous, 32-byte aligned.
__host__ __device__ constexpr int tab_poly(int sg, int i)
{
    return kTabHead + sg * kSigStride + i * kNC;
}

// Footprint kinds (table head slot kTabMode).
enum TabMode : int {
    kModeBspline = 0,   // beta^n_a * beta^n_b (Prop. 1, D = 2)
    kModeBoxSame = 1,   // 3-direction box-spline, sin and cos of equal sign: boxes b, a, a - b
    kModeBoxOpp = 2,    // 3-direction box-spline, opposite signs: boxes b, a, a + b
};

enum LineFlags : int {
    kVert = 1,        // rows are x2 (index j), columns x1 (index i)
    kKapNeg = 2,      // u decreases with the column index
    kDeg0Axis = 4,    // degree 0 and b == 0: rectangle, midpoint value at its edges
    kEmpty = 8,       // the line meets no support
};

// Per-line record (64 bytes).  u(r, q) = U0 + (r - r_ref) rho + (q - q_ref) kappa,
// kappa = +-a; rho and a are carried as hi + lo pairs whose hi parts make the
// products with row and step counts exact.
struct __align__(16) LineHdr {
    float U0;              // u at (r_ref, q_ref), in (0, a]
    float rho_hi, rho_lo;  // u step per row
    float a_hi, a_lo;      // a = a_hi + a_lo
    float a;               // |kappa| as one float
    float two_w;           // 2w
    int r_ref, q_ref;
    int r_begin, r_end;    // rows to visit, [r_begin, r_end)
    int flags;
    int tab;               // index of the footprint table
    int K;                 // candidate slots per row
    float U0_lo;           // U0 = U0 (above) + U0_lo exactly enough for degree 0
    float a_corr;          // |kappa| minus the a the footprint table was built with
};
static_assert(sizeof(LineHdr) == 64, "LineHdr layout");

struct GridDev {
    int nx, ny, degree;
    int basis;   // sp_basis
    int kdeg;    // degree the kernels are instantiated for: degree, or 2 for the box-spline
    float h, cx, cy;
};

struct LinesDev {
    int kind, n_view, n_det;
    int64_t m;
    const float *theta, *y, *src, *dst, *view;
    float det0, ddet, dso, dod;
    // Free line lists (THETA_Y, POINTS) on the strip kernels: the line indices
    // in chunk order (sorted by major axis, direction and offset; order.cu),
    // else NULL (parallel and fan beams take their lines view by view).
    const int *order;
};

// The chunk layout of the strip kernels: n_view "views" of n_det lines each,
// cut into chunks of 32 consecutive lines.  A sorted free list is one view
// of m lines.
__host__ __device__ __forceinline__ int64_t chunk_views(const LinesDev &L) { return L.order ? 1 : L.n_view; }
__host__ __device__ __forceinline__ int64_t chunk_bins(const LinesDev &L) { return L.order ? L.m : L.n_det; }

// Exactly-rounded u_0 of row r for a given step count k:
// u_0 = U0 + dr*rho - k*a, with the hi products exact.
__device__ __forceinline__ float row_u0(const LineHdr &H, int dr, int k)
{
    float fr = (float)dr, fk = (float)k;
    float big = __fsub_rn(__fmul_rn(fr, H.rho_hi), __fmul_rn(fk, H.a_hi));
    float small = __fmaf_rn(fr, H.rho_lo, __fmul_rn(-fk, H.a_lo));
    return __fadd_rn(__fadd_rn(H.U0, small), big);
}

// Row setup: the step count k and u_0 in (0, a] of row r.
__device__ __forceinline__ float row_start(const LineHdr &H, float inv_a, int r, int &k)
{
    int dr = r - H.r_ref;
    float V = __fmaf_rn((float)dr, H.rho_hi + H.rho_lo, H.U0);
    k = (int)ceilf(V * inv_a) - 1;
    float u0 = row_u0(H, dr, k);
    if (u0 <= 0.0f) { k -= 1; u0 = row_u0(H, dr, k); }
    else if (u0 > H.a) { k += 1; u0 = row_u0(H, dr, k); }
    return u0;
}

// Degree 0 near an axis has footprint ramps of width b, which can be far
// narrower than one float ulp of u.  For that degree u_0 is carried as an
// unevaluated sum hi + lo.
struct U0DF {
    float hi, lo;
};

__device__ __forceinline__ U0DF row_u0_df(const LineHdr &H, int dr, int k)
{
    float fr = (float)dr, fk = (float)k;
    float big = __fsub_rn(__fmul_rn(fr, H.rho_hi), __fmul_rn(fk, H.a_hi));   // exact
    float small = __fadd_rn(__fmaf_rn(fr, H.rho_lo, __fmul_rn(-fk, H.a_lo)), H.U0_lo);
    float s = __fadd_rn(H.U0, big);                                             // two-sum
    float bb = __fsub_rn(s, H.U0);
    float err = __fadd_rn(__fsub_rn(H.U0, __fsub_rn(s, bb)), __fsub_rn(big, bb));
    float lo = __fadd_rn(err, small);
    float hi = __fadd_rn(s, lo);
    lo = __fsub_rn(lo, __fsub_rn(hi, s));
    return U0DF{hi, lo};
}

// u_0 - c for a float c, as one float (accurate when the result is small).
__device__ __forceinline__ float df_minus(U0DF u, float c) { return __fadd_rn(__fsub_rn(u.hi, c), u.lo); }

__device__ __forceinline__ U0DF row_start_df(const LineHdr &H, float inv_a, int r, int &k)
{
    int dr = r - H.r_ref;
    float V = __fmaf_rn((float)dr, H.rho_hi + H.rho_lo, H.U0);
    k = (int)ceilf(V * inv_a) - 1;
    U0DF u = row_u0_df(H, dr, k);
    // u_0 in (0, |kappa|], |kappa| = a_hi + a_lo
    if (__fadd_rn(u.hi, u.lo) <= 0.0f) { k -= 1; u = row_u0_df(H, dr, k); }
    else if (__fadd_rn(__fsub_rn(u.hi, H.a_hi), __fsub_rn(u.lo, H.a_lo)) > 0.0f) {
        k += 1;
        u = row_u0_df(H, dr, k);
    }
    return u;
}

// ------------------------------------------------------------------ row evaluation
// Horner scheme of a table polynomial (see tab_poly).
template <int DEG>
__device__ __forceinline__ float horner(const float *T, float t)
{
    constexpr int NC = 2 * DEG + 2;
    float s = T[NC - 1];
#pragma unroll
    for (int d = NC - 2; d >= 0; --d) s = __fmaf_rn(s, t, T[d]);
    return s;
}

template <int DEG>
__device__ __forceinline__ int sigma_of(const float *s, float u0, float &s_lo)
{
    int sg = 0;
    s_lo = 0.f;
#pragma unroll
    for (int q = 0; q <= DEG; ++q) {
        float v = s[q];
        if (v < u0) { sg = q + 1; s_lo = v; }
    }
    return sg;
}

// Row r of a line: first column q0, interval sigma, polynomial argument t of
// candidate 0, and for degree 0 the argument shift per candidate and the
// midpoint tie of an axis-aligned rectangle.
struct RowEval {
    int q0, sg;
    float t;
    bool tie;
    float uhi, ulo;   // degree 0: u_0 as a float pair
};

template <int DEG>
__device__ __forceinline__ RowEval row_eval(const LineHdr &H, const float *s, float inv_a, int sgn, int r)
{
    RowEval e;
    int k;
    if constexpr (DEG == 0) {
        U0DF u = row_start_df(H, inv_a, r, k);
        e.sg = (df_minus(u, s[0]) > 0.f) ? 1 : 0;
        e.t = df_minus(u, e.sg ? s[0] : 0.f);
        e.tie = (H.flags & kDeg0Axis) &&
                __fadd_rn(__fsub_rn(u.hi, H.a_hi), __fsub_rn(u.lo, H.a_lo)) == 0.f;
        e.uhi = u.hi;
        e.ulo = u.lo;
    } else {
        float u0 = row_start(H, inv_a, r, k);
        float s_lo;
        e.sg = sigma_of<DEG>(s, u0, s_lo);
        e.t = u0 - s_lo;
        e.tie = false;
        e.uhi = u0;
        e.ulo = 0.f;
    }
    e.q0 = H.q_ref - sgn * k;
    return e;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Kernel launchers (kernels.cu).
cudaError_t launch_setup(const GridDev &g, const LinesDev &L, LineHdr *hdr, float *tabs, cudaStream_t s);
cudaError_t launch_tables(const GridDev &g, const LinesDev &L, float *tabs, int64_t n_tab,
                          cudaStream_t s);
// Line setup and tables (one fused kernel where each line has its own
// B-spline table and there are enough lines, else launch_setup then
// launch_tables).
cudaError_t launch_prepare(const GridDev &g, const LinesDev &L, LineHdr *hdr, float *tabs, int64_t n_tab,
                           cudaStream_t s);
cudaError_t launch_fwd(const GridDev &g, const LineHdr *hdr, const float *tabs, int64_t m,
                       const float *coef, float *sino, cudaStream_t s);
cudaError_t launch_adj(const GridDev &g, const LineHdr *hdr, const float *tabs, int64_t m,
                       const float *sino, float *coef_out, cudaStream_t s);
cudaError_t launch_visited(const GridDev &g, const LineHdr *hdr, const float *tabs, int64_t m,
                           int32_t *counts, const int64_t *offsets, int32_t *nodes,
                           cudaStream_t s);
cudaError_t launch_expand(const LinesDev &L, float *theta_out, float *y_out, cudaStream_t s);

// Sorted row records of every line, kept by a plan so that its projections
// skip the per-row traversal (strip.cu): line_bytes per line, line-major.
struct StripRec {
    unsigned char *base;
    long long line_bytes;
};

// Free line lists in strip-kernel order (order.cu): the key of every line
// (major axis, then direction, then the position of its run at the grid's
// middle row) and a stable radix sort of the line indices by it.  `area`
// holds line_order_bytes(m); the order (m ints) is at its start, the rest is
// scratch of the sort.
size_t line_order_bytes(int64_t m);
cudaError_t launch_line_order(const GridDev &g, const LinesDev &L, const LineHdr *hdr, void *area, cudaStream_t s);
// Whether the strip kernels take the lines of L through a sorted order.
inline bool strip_needs_order(const LinesDev &L) { return L.kind == SP_LINES_THETA_Y || L.kind == SP_LINES_POINTS; }

// Forward projection with coefficient strips in shared memory (strip.cu), for
// parallel and fan beams and sorted free line lists (any degree; L.order set
// for the latter).  `scratch` holds strip_scratch_bytes;
// `slow_rows` counts rows whose run fell outside the staged window.  With
// `rec` (written by launch_strip_record for the same lines) the row records
// are read instead of recomputed.
bool strip_supported(const GridDev &g, const LinesDev &L);
size_t strip_scratch_bytes(const GridDev &g);
long long strip_rec_line_bytes(const GridDev &g);
cudaError_t launch_fwd_strip(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                             const float *coef, void *scratch, float *sino, int *slow_rows, cudaStream_t s,
                             const StripRec *rec = nullptr);
// Adjoint with strip accumulators; coef_out is overwritten.  `defer` holds
// 2 + strip_chunk_count(L) words (chunks deferred to float strips).
int64_t strip_chunk_count(const LinesDev &L);
cudaError_t launch_adj_strip(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                             const float *sino, void *scratch, float *coef_out, int *slow_rows, cudaStream_t s,
                             const StripRec *rec, unsigned *defer);
// Pixel-driven adjoint (gather.cu): thread per node over all views, no
// atomics; parallel and fan beams of degree >= 1.  coef_out is overwritten.
bool gather_supported(const GridDev &g, const LinesDev &L);
cudaError_t launch_adj_gather(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                              const float *sino, float *coef_out, cudaStream_t s);
// The row records of every line of (g, L) into rec (after line setup and tables).
cudaError_t launch_strip_record(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                                const StripRec &rec, cudaStream_t s);

// One instance of the persistent strip kernel's work queue: the arguments of
// one strip projection and the index of its first chunk in the queue.
struct StripJob {
    GridDev g;
    LinesDev L;
    const LineHdr *hdr;
    const float *tabs;
    const float *coef;     // forward input (NULL for the adjoint)
    float *coefT;          // scratch: transposed input (forward) ...
    float *sino;
    float *out, *outT;     // ... or output and transposed output (adjoint)
    int *err;
    int cpv;               // chunks per view
    int vec;               // 16-byte staging and flushing
    long long chunk0;
};
// The job of one strip projection (adj: img_out receives the adjoint of sino;
// forward: sino receives the projection of img_in).  chunk0 is left 0.
StripJob make_strip_job(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs, bool adj,
                        const float *img_in, float *sino, float *img_out, void *scratch, int *err);
int64_t strip_job_chunks(const StripJob &J);
// Before the queue kernel: transposed copy of the input (forward) or cleared
// outputs (adjoint); after it: the transposed output added in (adjoint).
cudaError_t launch_strip_pre(const StripJob &J, bool adj, cudaStream_t s);
cudaError_t launch_strip_post(const StripJob &J, bool adj, cudaStream_t s);
// The persistent kernel over jobs[0..njobs) (device array, chunk0 ascending,
// `total` chunks in all, every job of kernel degree deg in 0..3); counter is
// three device words, reset here.  The adjoint defers chunks that need float
// strips to `defer` (device, room for `total` chunk indices) and runs them in
// a second launch.
cudaError_t launch_strip_queue(int deg, bool adj, const StripJob *jobs, int njobs, int64_t total,
                               unsigned long long *counter, long long *defer, cudaStream_t s);
cudaError_t launch_footprint_eval(const GridDev &g, int64_t count, const float *theta, const float *yt,
                                  float *out, float *scratch, cudaStream_t s);


// FP32 throughput probe (peak.cu): FLOPs of one launch, and the launch.
int64_t fp32_peak_flops(int packed, int blocks, int iters);
cudaError_t launch_fp32_peak(int packed, int blocks, int iters, float *out, cudaStream_t s);

// Argument errors and the thread-local message of the C ABI (api.cu), for the
// entry points defined in other translation units.
sp_status record_error(sp_status st, const char *msg);
void clear_error();

// CGLS (cg.cu).  The projector is passed as callbacks so that cg.cu does not
// depend on how a plan runs its projections.
struct CgOps {
    void *ctx;
    cudaError_t (*fwd)(void *ctx, const float *coef, float *sino, cudaStream_t s);
    cudaError_t (*adj)(void *ctx, const float *sino, float *coef_out, cudaStream_t s);
};
size_t cg_workspace_bytes(int64_t n, int64_t m);
cudaError_t run_cgls(const CgOps &ops, int64_t n, int64_t m, const float *b, float *x, int iters, double *hist,
                     void *ws, cudaStream_t s);

}  // namespace spx
