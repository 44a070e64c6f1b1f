// Kernels of the spline x-ray projector: line setup, footprint tables,
// forward projection, adjoint, visited-set listing, line expansion and a
// footprint probe.  The method is that of "Generalized Ray Tracing with Basis
// Functions for Tomographic Projections" (arXiv 2503.20907); see common.cuh
// for the geometry and the table layout.
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace spx {
namespace {

// Left-anchored B-spline beta^n on [0, n+1] (Sec. III.C, centred beta^n
// shifted by (n+1)/2), piece l on x = l + tau, tau in [0, 1): coefficients of
// tau^0..tau^n, from beta^n(x) = 1/n! sum_k (-1)^k C(n+1,k) (x-k)_+^n.
// Read with lane-dependent l, so it sits in global memory (L1), not in the
// constant bank.
__device__ const float kBPiece[4][4][4] = {
    {{1.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}},
    {{0.f, 1.f, 0.f, 0.f}, {1.f, -1.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}},
    {{0.f, 0.f, 0.5f, 0.f}, {0.5f, 1.f, -1.f, 0.f}, {0.5f, -1.f, 0.5f, 0.f}, {0.f, 0.f, 0.f, 0.f}},
    {{0.f, 0.f, 0.f, 1.f / 6.f}, {1.f / 6.f, 0.5f, 0.5f, -0.5f}, {2.f / 3.f, 0.f, -1.f, 0.5f},
     {1.f / 6.f, -0.5f, 0.5f, -1.f / 6.f}},
};

// Binomial coefficient C(n, k) (exact in float for n < 25); folded to a
// constant wherever its arguments are.
__host__ __device__ constexpr float binomf(int n, int k)
{
    if (k < 0 || k > n) return 0.f;
    float r = 1.f;
    for (int i = 1; i <= k; ++i) r = r * (float)(n - k + i) / (float)i;
    return r;
}

__device__ __forceinline__ float factf(int n)
{
    float r = 1.f;
    for (int i = 2; i <= n; ++i) r *= (float)i;
    return r;
}

// Unit direction (dx, dy) and a point (px, py) of line r, in double.  For
// parallel and fan beams, vs / vc (if not NULL) hold sin and cos of the view
// angle of line r, computed as below.
__device__ void line_geometry(const LinesDev &L, int64_t r, double &dx, double &dy, double &px,
                              double &py, const double *vs = nullptr, const double *vc = nullptr)
{
    switch (L.kind) {
    case SP_LINES_THETA_Y: {
        double th = (double)L.theta[r], yy = (double)L.y[r], s, c;
        sincos(th, &s, &c);
        dx = c; dy = s; px = yy * s; py = -yy * c;
        break;
    }
    case SP_LINES_POINTS: {
        double sx = L.src[2 * r], sy = L.src[2 * r + 1];
        double vx = (double)L.dst[2 * r] - sx, vy = (double)L.dst[2 * r + 1] - sy;
        double inv = 1.0 / sqrt(vx * vx + vy * vy);
        dx = vx * inv; dy = vy * inv; px = sx; py = sy;
        break;
    }
    case SP_LINES_PARALLEL: {
        int64_t v = r / L.n_det, j = r - v * L.n_det;
        double s, c;
        if (vs) { s = *vs; c = *vc; }
        else sincos((double)L.view[v], &s, &c);
        double yy = (double)L.det0 + (double)j * (double)L.ddet;
        dx = c; dy = s; px = yy * s; py = -yy * c;
        break;
    }
    default: {  // SP_LINES_FAN
        int64_t v = r / L.n_det, j = r - v * L.n_det;
        double sb, cb;
        if (vs) { sb = *vs; cb = *vc; }
        else sincos((double)L.view[v], &sb, &cb);
        double sx = (double)L.dso * cb, sy = (double)L.dso * sb;
        double off = (double)L.det0 + (double)j * (double)L.ddet;
        double ex = -(double)L.dod * cb - off * sb, ey = -(double)L.dod * sb + off * cb;
        double vx = ex - sx, vy = ey - sy;
        double inv = 1.0 / sqrt(vx * vx + vy * vy);
        dx = vx * inv; dy = vy * inv; px = sx; py = sy;
        break;
    }
    }
}

// The footprint parameters a, b as the table uses them.  For degree >= 1 a
// b below kBMin changes phi by less than about 2 kBMin and is taken as the
// Dirac of Prop. 1; degree 0 keeps any representable b (its ramps have slope
// 1/(a b), so dropping b would move mass by O(1) near cell edges).
__device__ __forceinline__ void footprint_ab(int degree, double dx, double dy, float &af, float &bf)
{
    af = (float)fmax(fabs(dx), fabs(dy));
    bf = (float)fmin(fabs(dx), fabs(dy));
    if (bf < (degree == 0 ? 1e-30f : kBMin)) bf = 0.f;
}

__device__ __forceinline__ float two_w_of(int m, float af, float bf)
{
    return (float)((double)m * ((double)af + (double)bf));
}

__device__ __forceinline__ int slots_of(int m, float af, float bf, float two_w)
{
    if (bf == 0.f) return m;
    int K = (int)floorf(two_w / af) + 1;
    return K < 2 * m ? K : 2 * m;
}

// Support of phi_theta in u = y~ + w: its length 2w (float, as the kernels
// compare it), w (double), and the candidate slots K of a row.  B-splines:
// 2w = (n+1)(a+b).  Box-spline: the three box widths b, a, a -+ b add up to
// 2a (sin and cos of equal sign) or 2(a+b) (opposite signs).
__device__ __forceinline__ void support_params(int kdeg, float af, float bf, int mode, float &two_w, double &w,
                                               int &K)
{
    if (mode == kModeBspline) {
        const int m = kdeg + 1;
        two_w = two_w_of(m, af, bf);
        w = 0.5 * m * ((double)af + (double)bf);
        K = slots_of(m, af, bf, two_w);
    } else {
        const double W = (mode == kModeBoxSame) ? 2.0 * (double)af : 2.0 * ((double)af + (double)bf);
        two_w = (float)W;
        w = 0.5 * W;
        const int k = (int)floorf(two_w / af) + 1;
        K = k < 2 * (kdeg + 1) ? k : 2 * (kdeg + 1);
    }
}

__device__ __forceinline__ int footprint_mode(int basis, double dx, double dy)
{
    if (basis != SP_BASIS_BOX3) return kModeBspline;
    return (dx * dy >= 0.0) ? kModeBoxSame : kModeBoxOpp;
}

// Split x into hi + lo with hi carrying `bits` significant bits.
__device__ void split_hi_lo(double x, int bits, float &hi, float &lo)
{
    if (x == 0.0) { hi = 0.f; lo = 0.f; return; }
    int e;
    frexp(x, &e);
    const double sc = ldexp(1.0, bits - e), isc = ldexp(1.0, e - bits);   // powers of two: exact
    double xh = rint(x * sc) * isc;
    hi = (float)xh;
    lo = (float)(x - xh);
}

// ------------------------------------------------------------------ setup
constexpr int kSetupThreads = 128;

// Line setup of line r: its record hdr[r] (see LineHdr) and the footprint's
// a, b and kind.  vs, vc: sin and cos of the line's view for parallel and fan
// beams (NULL: computed here).
__device__ void setup_line(const GridDev &g, const LinesDev &L, int64_t r, LineHdr *hdr, const double *vs,
                           const double *vc, float &af, float &bf, int &mode)
{
    double dx, dy, px, py;
    line_geometry(L, r, dx, dy, px, py, vs, vc);
    LineHdr H;
    H.U0_lo = 0.f;
    H.a_corr = 0.f;
    H.tab = (L.kind == SP_LINES_PARALLEL) ? (int)(r / L.n_det) : (int)r;
    footprint_ab(g.kdeg, dx, dy, af, bf);
    mode = footprint_mode(g.basis, dx, dy);
    double w;
    support_params(g.kdeg, af, bf, mode, H.two_w, w, H.K);
    const bool vert = fabs(dy) >= fabs(dx);
    const double A = fmax(fabs(dx), fabs(dy));
    const double B = fmin(fabs(dx), fabs(dy));
    const double h = (double)g.h;
    const double Yhat = ((px - (double)g.cx) * dy - (py - (double)g.cy) * dx) / h;
    const double ic = 0.5 * (g.nx - 1), jc = 0.5 * (g.ny - 1);
    double kap, rho, rc, qc;
    int Nr, Nq;
    if (vert) { kap = -dy; rho = dx; rc = jc; qc = ic; Nr = g.ny; Nq = g.nx; }
    else { kap = dx; rho = -dy; rc = ic; qc = jc; Nr = g.nx; Nq = g.ny; }
    const int sgn = kap > 0.0 ? 1 : -1;
    // w as the table sees it (support_params, with the table's a and b)
    int flags = (vert ? kVert : 0) | (sgn < 0 ? kKapNeg : 0);
    if (g.degree == 0 && B == 0.0) flags |= kDeg0Axis;

    // Rows whose support run meets the columns [0, Nq): the column of the
    // support centre (u = w) moves linearly with the row.
    const double lo = -w / A - 2.0, hi = (double)(Nq - 1) + w / A + 2.0;
    const double c0 = qc - (Yhat - rc * rho) / kap;   // centre column at row 0
    const double gam = -rho / kap;
    int rb = 0, re = 0;
    if (fabs(gam) < 1e-300) {
        if (c0 >= lo && c0 <= hi) { rb = 0; re = Nr; }
    } else {
        double t0 = (lo - c0) / gam, t1 = (hi - c0) / gam;
        if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
        t0 = fmax(floor(t0) - 1.0, 0.0);
        t1 = fmin(ceil(t1) + 2.0, (double)Nr);
        if (t1 > t0) { rb = (int)t0; re = (int)t1; }
    }
    if (rb >= re || !(Yhat == Yhat)) {
        H.flags = flags | kEmpty;
        H.U0 = H.rho_hi = H.rho_lo = H.a_hi = H.a_lo = 0.f;
        H.a = af;
        H.r_ref = H.q_ref = H.r_begin = H.r_end = 0;
        hdr[r] = H;
        return;
    }
    const int r_ref = (rb + re) / 2;
    // u at (r_ref, q = 0), then the reference column with U0 in (0, a].
    const double Ur = Yhat + w + ((double)r_ref - rc) * rho - qc * kap;
    double qr = (sgn > 0) ? floor(-Ur / A) + 1.0 : ceil(Ur / A) - 1.0;
    double U0 = Ur + qr * kap;
    if (U0 <= 0.0) { qr += sgn; U0 = Ur + qr * kap; }
    else if (U0 > A) { qr -= sgn; U0 = Ur + qr * kap; }
    // hi parts exact against |row offset| and |step count|, both < maxc
    int maxc = (re - rb) + 8;
    int nb = 0;
    while ((1 << nb) <= maxc) ++nb;
    const int bits = 23 - nb;
    H.U0 = (float)U0;
    H.U0_lo = (float)(U0 - (double)H.U0);
    split_hi_lo(rho, bits, H.rho_hi, H.rho_lo);
    split_hi_lo(A, bits, H.a_hi, H.a_lo);
    H.a = af;
    H.a_corr = (float)(A - (double)af);
    H.r_ref = r_ref;
    H.q_ref = (int)qr;
    H.r_begin = rb;
    H.r_end = re;
    H.flags = flags;
    hdr[r] = H;
}

__global__ void __launch_bounds__(kSetupThreads) setup_kernel(GridDev g, LinesDev L, LineHdr *hdr, float *tabs, int64_t M)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // parallel and fan beams: sin and cos of each view once per block (the
    // block's lines span at most blockDim.x views)
    __shared__ double vsin[kSetupThreads], vcos[kSetupThreads];
    const bool views = (L.kind == SP_LINES_PARALLEL || L.kind == SP_LINES_FAN);
    int64_t v0 = 0;
    if (views) {
        const int64_t r0 = (int64_t)blockIdx.x * blockDim.x;
        const int64_t r1 = min(r0 + (int64_t)blockDim.x, M) - 1;
        v0 = r0 / L.n_det;
        const int64_t nv = r1 / L.n_det - v0 + 1;
        if (threadIdx.x < nv) sincos((double)L.view[v0 + threadIdx.x], &vsin[threadIdx.x], &vcos[threadIdx.x]);
        __syncthreads();
    }
        if (r >= M) return;
    float af, bf;
    int mode;
    if (views) {
        const int k = (int)(r / L.n_det - v0);
        setup_line(g, L, r, hdr, &vsin[k], &vcos[k], af, bf, mode);
    } else {
        setup_line(g, L, r, hdr, nullptr, nullptr, af, bf, mode);
    }
    const int tab = (L.kind == SP_LINES_PARALLEL) ? (int)(r / L.n_det) : (int)r;
    if (L.kind != SP_LINES_PARALLEL || r % L.n_det == 0) {
        // the owner of table tab hands a, b and the footprint kind to the table builder
        tabs[(int64_t)tab * kTabFloats + kTabA] = af;
        tabs[(int64_t)tab * kTabFloats + kTabB] = bf;
        tabs[(int64_t)tab * kTabFloats + kTabMode] = (float)mode;
    }
}

// ------------------------------------------------------------------ tables
// Derivatives e = 0..N of B-spline piece l at tau, times b^-(1+e).
template <int N>
__device__ __forceinline__ void bspline_piece_derivs(int l, float tau, float binv, float *D)
{
    float sc = binv;
#pragma unroll
    for (int e = 0; e <= N; ++e) {
        float acc = 0.f;
#pragma unroll
        for (int k = N; k >= e; --k) {
            float ff = 1.f;   // k!/(k-e)!
#pragma unroll
            for (int t = 0; t < e; ++t) ff *= (float)(k - t);
            acc = acc * tau + kBPiece[N][l][k] * ff;
        }
        D[e] = acc * sc;
        sc *= binv;
    }
}

// Sign of (pa + qb) - (p2 a + q2 b) + extra, formed from the integer
// differences so that it is accurate whatever the size of a and b.
__device__ __forceinline__ float sym_diff(int dp, int dq, float a, float b, float extra)
{
    return __fmaf_rn((float)dp, a, __fmaf_rn((float)dq, b, extra));
}

// Build the footprint table of one direction (see common.cuh), degree N, on
// one half-warp: l is the lane within the half (0..15) and gmask the half's
// lanes.  sm is the half's shared scratch of kBuildScratch floats; the table
// is assembled there and then written to out (if out is not NULL).  Every
// phase fits 16 lanes (at most 15 pieces start before the centre of the
// support; 25 breakpoints are ranked two per lane), so a warp builds two
// tables at once.
constexpr int kBuildScratch = kTabFloats + 32 + 32 + 25 * 8 + 8 + 8 + 8;
constexpr int kTabWarps = 8;

template <int N>
__device__ void build_table_half(float a, float b, float *out, float *sm, int l, unsigned gmask)
{
    constexpr int n = N, m = N + 1, nc = 2 * N + 2;
    constexpr int G = 16;
    float *tab = sm;
    float *bv = tab + kTabFloats;                       // sorted breakpoint values
    int *bpq = reinterpret_cast<int *>(bv + 32);        // and their (p, q), p | q << 8
    float *P = reinterpret_cast<float *>(bpq + 32);     // piece polynomials [25][8]
    float *sv = P + 25 * 8;                             // sorted u_0 interval ends
    int *sq = reinterpret_cast<int *>(sv + 8);
    int *sf = sq + 8;
    for (int k = l; k < kTabFloats / 4; k += G) reinterpret_cast<float4 *>(tab)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp(gmask);
    const float two_w = two_w_of(m, a, b);
    const float ainv = 1.0f / a;
    if (b == 0.f) {
        // Dirac factor (Prop. 1): phi(u) = beta^n(u/a)/a on the a-knots.
        if (l < kTabHead) tab[l] = l == kTabA ? a : (l == kTabB ? 0.f : (l < m ? a : FLT_MAX));
        if (l < m * (n + 1)) {
            const int i = l / (n + 1), e = l - i * (n + 1);
            float sc = ainv;
            for (int k = 0; k < e; ++k) sc *= ainv;
            tab[tab_poly(0, i) + e] = kBPiece[n][i][e] * sc;
        }
    } else {
        // breakpoints p a + q b, ranked (ties by p, then q)
        constexpr int NB = (m + 1) * (m + 1);
        constexpr int NI = (NB + G - 1) / G;   // breakpoints per lane: l and l + 16
        // all values in the scratch of the pieces (filled later), read back
        // four at a time; ties go by index, which orders (p, q) lexicographically
        float *vr = P;
        int p[NI], q[NI];
        float v[NI];
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int idx = l + G * it;
            p[it] = 0; q[it] = 0; v[it] = 0.f;
            if (idx < NB) {
                p[it] = idx / (m + 1);
                q[it] = idx - p[it] * (m + 1);
                v[it] = __fmaf_rn((float)p[it], a, (float)q[it] * b);
                vr[idx] = v[it];
            }
        }
        __syncwarp(gmask);
        int rank[NI];
#pragma unroll
        for (int it = 0; it < NI; ++it) rank[it] = 0;
#pragma unroll
        for (int j4 = 0; j4 < (NB + 3) / 4; ++j4) {
            const float4 w4 = reinterpret_cast<const float4 *>(vr)[j4];
            const float vj[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 4 * j4 + u;
                if (j < NB)
#pragma unroll
                    for (int it = 0; it < NI; ++it)
                        rank[it] += (vj[u] < v[it]) || (vj[u] == v[it] && j < l + G * it);
            }
        }
        __syncwarp(gmask);
#pragma unroll
        for (int it = 0; it < NI; ++it)
            if (l + G * it < NB) { bv[rank[it]] = v[it]; bpq[rank[it]] = p[it] | (q[it] << 8); }
        __syncwarp(gmask);
        // pieces that start at or before the centre w: the leading sorted run
        // (the last breakpoint, at 2w, is always beyond it)
        int mp = 0, mq = 0;
        unsigned outside = 0u;
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int idx = l + G * it;
            int ip = 0, iq = 0;
            if (idx < NB) { ip = bpq[idx] & 255; iq = bpq[idx] >> 8; }
            if (it == 0) { mp = ip; mq = iq; }
            const unsigned bal = __ballot_sync(gmask, idx >= NB || sym_diff(2 * ip - m, 2 * iq - m, a, b, 0.f) > 0.f);
            outside |= ((bal >> (threadIdx.x & 16)) & 0xFFFFu) << (G * it);
        }
        int nh = __ffs(outside) - 1;
        if (nh < 1) nh = 1;
        // derivatives n+1..2n+1 of every piece directly (right-sided at its start)
        const float binv = 1.0f / b;
        float am = 1.f;
#pragma unroll
        for (int k = 0; k < m; ++k) am *= ainv;
        if (l < nh) {
            const int p0 = mp, q0 = mq;
            float hi[n + 1];
#pragma unroll
            for (int e = 0; e <= n; ++e) hi[e] = 0.f;
#pragma unroll
            for (int pp = 0; pp <= m; ++pp) {
                int piece;
                float tau;
                if (pp == p0) {
                    if (q0 >= m) continue;
                    piece = q0; tau = 0.f;
                } else {
                    const float vv = __fmaf_rn((float)(p0 - pp), a, (float)q0 * b);
                    if (vv < 0.f) continue;
                    const float t = __fdiv_rn(vv, b);   // exact when vv is a multiple of b
                    piece = (int)floorf(t);
                    if (piece < 0 || piece >= m) continue;
                    tau = t - (float)piece;
                }
                float D[n + 1];
                bspline_piece_derivs<n>(piece, tau, binv, D);
                const float wp = binomf(m, pp) * ((pp & 1) ? -1.f : 1.f);
#pragma unroll
                for (int e = 0; e <= n; ++e) hi[e] = __fmaf_rn(wp, D[e], hi[e]);
            }
#pragma unroll
            for (int e = 0; e <= n; ++e) P[l * 8 + n + 1 + e] = hi[e] * am / factf(n + 1 + e);
            if (l == 0)
#pragma unroll
                for (int d = 0; d <= n; ++d) P[d] = 0.f;
        }
        __syncwarp(gmask);
        // derivatives 0..n carried from piece to piece (lane d computes coefficient d);
        // C(k, l) held in registers (a lane-dependent index into a constant
        // table would serialise the warp's constant loads)
        float cb[nc];
#pragma unroll
        for (int k = 0; k < nc; ++k) {
            float c = 0.f;
#pragma unroll
            for (int d = 0; d <= n; ++d)
                if (l == d) c = binomf(k, d);
            cb[k] = c;
        }
        // lane pi holds the length of piece pi - 1 (the step to piece pi); the
        // low coefficients of the previous piece travel in registers (lane d
        // holds coefficient d), the top ones come from the scratch
        float dlv = 0.f;
        if (l >= 1 && l < nh) {
            const int cur = bpq[l], prev = bpq[l - 1];
            dlv = sym_diff((cur & 255) - (prev & 255), (cur >> 8) - (prev >> 8), a, b, 0.f);
        }
        float low = 0.f;   // piece 0 starts the support: its coefficients 0..n vanish
        for (int pi = 1; pi < nh; ++pi) {
            const float dl = __shfl_sync(gmask, dlv, pi, G);
            float c[nc];
#pragma unroll
            for (int k = 0; k <= n; ++k) c[k] = __shfl_sync(gmask, low, k, G);
#pragma unroll
            for (int k = n + 1; k < nc; ++k) c[k] = P[(pi - 1) * 8 + k];
            float sacc = 0.f;
#pragma unroll
            for (int k = nc - 1; k >= 0; --k)
                if (k >= l) sacc = __fmaf_rn(sacc, dl, cb[k] * c[k]);
            low = sacc;
            if (l <= n) P[pi * 8 + l] = sacc;
        }
        __syncwarp(gmask);
        // u_0 interval ends s_q = (q b) mod a in (0, a], sorted (stable in q)
        float rq = 0.f;
        int fq = 0;
        if (l >= 1 && l <= m) {
            fq = (int)floorf((float)l * b * ainv);
            rq = __fmaf_rn((float)(-fq), a, (float)l * b);
            if (rq <= 0.f) { fq -= 1; rq = __fmaf_rn((float)(-fq), a, (float)l * b); }
            else if (rq > a) { fq += 1; rq = __fmaf_rn((float)(-fq), a, (float)l * b); }
        }
        int srank = 1;
#pragma unroll
        for (int j = 1; j <= m; ++j) {
            const float rj = __shfl_sync(gmask, rq, j, G);
            srank += (j < l) ? (rj <= rq) : (j > l ? (rj < rq) : 0);
        }
        if (l >= 1 && l <= m) { sv[srank] = rq; sq[srank] = l; sf[srank] = fq; }
        if (l == 0) { sv[0] = 0.f; sq[0] = 0; sf[0] = 0; }
        __syncwarp(gmask);
        if (l < kTabHead) tab[l] = l == kTabA ? a : (l == kTabB ? b : (l < m ? sv[l + 1] : FLT_MAX));
        const int K = slots_of(m, a, b, two_w);
        // entry e = (sigma, candidate) = (e / 8, e % 8), two sigmas per pass
#pragma unroll
        for (int pass = 0; pass < ((m + 1) * 8 + G - 1) / G; ++pass) {
            const int e = l + G * pass;
            const int sg = e >> 3, i = e & 7;
            if (sg > m || i >= K) continue;
            const float hw = 0.5f * (((sg < m) ? sv[sg + 1] : a) - sv[sg]);
            // interval start u_lo = (i - f) a + q b; midpoint u_lo + hw
            const int pl = i - sf[sg], ql = sq[sg];
            if (sym_diff(pl - m, ql - m, a, b, hw) >= 0.f) continue;          // beyond 2w
            const bool mirror = sym_diff(2 * pl - m, 2 * ql - m, a, b, 2.f * hw) > 0.f;
            // last piece (of the nh sorted ones) starting at or before the
            // midpoint of the entry (mirrored into the left half if needed):
            // binary search, the predicate being monotone in the piece index
            const int pq = mirror ? m - pl : pl, qq = mirror ? m - ql : ql;
            const float hs = mirror ? -hw : hw;
            int pi = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int c = pi + st;
                if (c < nh && sym_diff(pq - (bpq[c] & 255), qq - (bpq[c] >> 8), a, b, hs) >= 0.f) pi = c;
            }
            const int bp = bpq[pi] & 255, bq = bpq[pi] >> 8;
            const float X = mirror ? sym_diff(m - pl - bp, m - ql - bq, a, b, 0.f) : sym_diff(pl - bp, ql - bq, a, b, 0.f);
            float *T = tab + tab_poly(sg, i);
            float c[8];
            {
                const float4 c0 = reinterpret_cast<const float4 *>(P + pi * 8)[0];
                const float4 c1 = reinterpret_cast<const float4 *>(P + pi * 8)[1];
                c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
                c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
            }
            float r[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) r[d] = 0.f;   // slots beyond nc stay zero
            if (X != 0.f) {
                // Taylor shift of the piece to the interval start
#pragma unroll
                for (int d = 0; d < nc; ++d) {
                    float sacc = 0.f;
#pragma unroll
                    for (int k = nc - 1; k >= d; --k) sacc = __fmaf_rn(sacc, X, binomf(k, d) * c[k]);
                    r[d] = (mirror && (d & 1)) ? -sacc : sacc;
                }
            } else {
#pragma unroll
                for (int d = 0; d < nc; ++d) r[d] = (mirror && (d & 1)) ? -c[d] : c[d];
            }
            reinterpret_cast<float4 *>(T)[0] = make_float4(r[0], r[1], r[2], r[3]);
            reinterpret_cast<float4 *>(T)[1] = make_float4(r[4], r[5], r[6], r[7]);
        }
    }
    __syncwarp(gmask);
    if (out)
        for (int k = l; k < kTabFloats / 4; k += G)
            reinterpret_cast<float4 *>(out)[k] = reinterpret_cast<const float4 *>(tab)[k];
    __syncwarp(gmask);
}

// Table of the 3-direction box-spline (Sec. III.D), same layout as the
// B-spline tables of kernel degree 2 (polynomials of degree <= 2 in t).
// phi_theta is the convolution of the boxes of widths b, a and a -+ b
// (Prop. 1 with D = 3): piecewise quadratic, C^1, with breakpoints at the
// sums of subsets of the widths, each carrying the sign (-1)^(subset size);
// phi'' = (sum of the signs passed) / (product of the widths).  Built
// stably like the B-spline tables: phi and phi' are carried from piece to
// piece with piece lengths formed from the integer coordinates (p, q) of the
// breakpoints p a + q b, so a narrow box never divides a large sum.  A width
// below kBMin (b near an axis, a - b near a diagonal) is a Dirac: the
// remaining two boxes give a piecewise-linear phi.
__device__ void build_table_box(float a, float b, int mode, float *out, float *sm, int lane)
{
    constexpr int K2 = 2, NSMAX = 3;          // kernel degree 2: up to 3 interval ends in the head
    float *tab = sm;
    float *pc = tab + kTabFloats;             // pieces: [8][3] (phi, phi', top derivative)
    int *bp = reinterpret_cast<int *>(pc + 24);   // sorted breakpoints p | q << 8 (q biased by 4)
    float *sv = reinterpret_cast<float *>(bp + 8);
    int *sq = reinterpret_cast<int *>(sv + 4);
    int *sf = sq + 4;
    int *nbp = sf + 4;
    for (int k = lane; k < kTabFloats; k += 32) tab[k] = 0.f;
    __syncwarp();
    if (lane == 0) {
        // box widths with their coordinates: b = (0,1), a = (1,0), a -+ b = (1,-+1)
        const int q3 = (mode == kModeBoxSame) ? -1 : 1;
        float wv[3] = {b, a, (mode == kModeBoxSame) ? a - b : (float)((double)a + (double)b)};
        int wp[3] = {0, 1, 1}, wq[3] = {1, 0, q3};
        int used[3], nu = 0;
        for (int d = 0; d < 3; ++d)
            if (wv[d] >= kBMin) used[nu++] = d;
        float prod = 1.f;
        for (int u = 0; u < nu; ++u) prod *= wv[used[u]];
        // all subset sums, sorted by value (ties by p, then q)
        const int nb = 1 << nu;
        int P[8], Q[8], S[8];
        float V[8];
        for (int e = 0; e < nb; ++e) {
            int pp = 0, qq = 0, c = 0;
            for (int u = 0; u < nu; ++u)
                if ((e >> u) & 1) { pp += wp[used[u]]; qq += wq[used[u]]; ++c; }
            int k = e;
            const float v = __fmaf_rn((float)pp, a, (float)qq * b);
            while (k > 0 && (V[k - 1] > v || (V[k - 1] == v && (P[k - 1] > pp || (P[k - 1] == pp && Q[k - 1] > qq))))) {
                V[k] = V[k - 1]; P[k] = P[k - 1]; Q[k] = Q[k - 1]; S[k] = S[k - 1];
                --k;
            }
            V[k] = v; P[k] = pp; Q[k] = qq; S[k] = (c & 1) ? -1 : 1;
        }
        // walk the pieces: phi, phi' and the top derivative (phi'' for three
        // boxes, phi' for two) on each
        float f0 = 0.f, f1 = 0.f;
        int acc = 0;
        for (int j = 0; j < nb; ++j) {
            acc += S[j];
            const float D = (float)acc / prod;
            bp[j] = P[j] | ((Q[j] + 4) << 8);
            pc[3 * j] = f0;
            pc[3 * j + 1] = (nu == 3) ? f1 : D;
            pc[3 * j + 2] = (nu == 3) ? 0.5f * D : 0.f;
            if (j + 1 < nb) {
                const float dl = sym_diff(P[j + 1] - P[j], Q[j + 1] - Q[j], a, b, 0.f);
                if (nu == 3) {
                    f0 = __fmaf_rn(__fmaf_rn(0.5f * D, dl, f1), dl, f0);
                    f1 = __fmaf_rn(D, dl, f1);
                } else {
                    f0 = __fmaf_rn(D, dl, f0);
                }
            }
        }
        *nbp = nb;
        // interval ends s = (q b) mod a in (0, a] for the q of the widths used
        int qs[2], nq = 0;
        for (int u = 0; u < nu; ++u) {
            const int qq = wq[used[u]];
            if (qq != 0 && (nq == 0 || qs[0] != qq)) qs[nq++] = qq;
        }
        if (mode == kModeBoxOpp && nu == 3) qs[nq++] = 2;   // b + (a + b) = a + 2b
        const float ainv = 1.0f / a;
        float rs[3];
        int fs[3], qv[3];
        for (int t = 0; t < nq; ++t) {
            const int qq = qs[t];
            int fq = (int)floorf((float)qq * b * ainv);
            float rq = __fmaf_rn((float)(-fq), a, (float)qq * b);
            if (rq <= 0.f) { fq -= 1; rq = __fmaf_rn((float)(-fq), a, (float)qq * b); }
            else if (rq > a) { fq += 1; rq = __fmaf_rn((float)(-fq), a, (float)qq * b); }
            int k = t;
            while (k > 0 && rs[k - 1] > rq) { rs[k] = rs[k - 1]; fs[k] = fs[k - 1]; qv[k] = qv[k - 1]; --k; }
            rs[k] = rq; fs[k] = fq; qv[k] = qq;
        }
        sv[0] = 0.f; sq[0] = 0; sf[0] = 0;
        for (int t = 0; t < nq; ++t) { sv[t + 1] = rs[t]; sq[t + 1] = qv[t]; sf[t + 1] = fs[t]; }
        for (int t = nq + 1; t <= NSMAX; ++t) { sv[t] = a; sq[t] = 0; sf[t] = -1; }
        for (int t = 0; t < kTabHead; ++t) tab[t] = FLT_MAX;
        for (int t = 0; t < nq; ++t) tab[t] = rs[t];
        tab[kTabMode] = (float)mode;
        tab[kTabA] = a;
        tab[kTabB] = b;
    }
    __syncwarp();
    // entries: lane = (interval sg, candidate i)
    const int nb = *nbp;
    const int sg = lane >> 3, i = lane & 7;
    const int nsg = NSMAX;   // intervals (s_sg, s_sg+1], sg = 0..2
    if (sg < nsg && i < 2 * (K2 + 1)) {
        const float hw = 0.5f * (sv[sg + 1] - sv[sg]);
        const int pl = i - sf[sg], ql = sq[sg];
        const int top = bp[nb - 1];
        const int ptop = top & 255, qtop = (top >> 8) - 4;
        // entry inside the support: its midpoint below the last breakpoint.
        // Empty intervals (hw = 0) are filled too, with the expansion just
        // right of their start: rows step by the exact |kappa|, which can
        // exceed the table's float a by an ulp, and a u_0 in that gap lands
        // in an empty last interval.
        if (sym_diff(pl - ptop, ql - qtop, a, b, hw) < 0.f) {
            int pi = 0;
#pragma unroll
            for (int st = 4; st > 0; st >>= 1) {
                const int c = pi + st;
                if (c < nb - 1) {
                    const int bc = bp[c];
                    if (sym_diff(pl - (bc & 255), ql - ((bc >> 8) - 4), a, b, hw) >= 0.f) pi = c;
                }
            }
            const int bc = bp[pi];
            const float X = sym_diff(pl - (bc & 255), ql - ((bc >> 8) - 4), a, b, 0.f);
            const float c0 = pc[3 * pi], c1 = pc[3 * pi + 1], c2 = pc[3 * pi + 2];
            float *T = tab + tab_poly(sg, i);
            T[0] = __fmaf_rn(__fmaf_rn(c2, X, c1), X, c0);
            T[1] = __fmaf_rn(2.f * c2, X, c1);
            T[2] = c2;
        }
    }
    __syncwarp();
    if (out)
        for (int k = lane; k < kTabFloats / 4; k += 32)
            reinterpret_cast<float4 *>(out)[k] = reinterpret_cast<const float4 *>(tab)[k];
    __syncwarp();
}

// Two tables per warp, one per half-warp (box-spline tables: one after the
// other on the full warp).  a, b and the footprint kind were written into the
// table head by the line setup (FP64 geometry stays there, once per line).
template <int DEG>
__global__ void __launch_bounds__(kTabWarps * 32) tables_kernel(float *tabs, int64_t n_tab)
{
    __shared__ __align__(16) float scratch[2 * kTabWarps][kBuildScratch];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4;
    const int64_t t0 = ((int64_t)blockIdx.x * kTabWarps + warp) * 2;
    if (t0 >= n_tab) return;
    const int nt = (t0 + 1 < n_tab) ? 2 : 1;
    const int mode0 = (int)tabs[t0 * kTabFloats + kTabMode];
    __syncwarp();
    if (DEG == 2 && mode0 != kModeBspline) {
        // box-spline tables (one basis per grid, so both are): full warp each
        for (int k = 0; k < nt; ++k) {
            float *out = tabs + (t0 + k) * (int64_t)kTabFloats;
            const float af = out[kTabA], bf = out[kTabB];
            const int mode = (int)out[kTabMode];
            __syncwarp();
            if (mode != kModeBspline) build_table_box(af, bf, mode, out, scratch[2 * warp], lane);
            else if (half == 0) build_table_half<DEG>(af, bf, out, scratch[2 * warp], lane, 0x0000FFFFu);
            __syncwarp();
        }
        return;
    }
    if (half >= nt) return;
    float *out = tabs + (t0 + half) * (int64_t)kTabFloats;
    const float af = out[kTabA], bf = out[kTabB];
    build_table_half<DEG>(af, bf, out, scratch[2 * warp + half], lane & 15, half ? 0xFFFF0000u : 0x0000FFFFu);
}

// Line setup and tables in one pass, for B-spline footprints with one table
// per line (fan beams, point pairs, (theta, y) lists): each warp sets up 32
// lines, one per lane (the FP64 geometry at full width), then builds their
// 32 tables two at a time, one per half-warp.  Warps at the FP64 stage and
// warps at the table stage share the SMs, so the two overlap.
template <int DEG>
__global__ void __launch_bounds__(kTabWarps * 32) setup_tables_kernel(GridDev g, LinesDev L, LineHdr *hdr, float *tabs,
                                                                      int64_t M)
{
    __shared__ __align__(16) float scratch[2 * kTabWarps][kBuildScratch];
    __shared__ double vsin[kTabWarps * 32], vcos[kTabWarps * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t r = r0 + threadIdx.x;
    // fan beams: sin and cos of each view once per block (at most blockDim.x views)
    const bool views = (L.kind == SP_LINES_FAN);
    int64_t v0 = 0;
    if (views) {
        const int64_t r1 = min(r0 + (int64_t)blockDim.x, M) - 1;
        v0 = r0 / L.n_det;
        const int64_t nv = r1 / L.n_det - v0 + 1;
        if (threadIdx.x < nv) sincos((double)L.view[v0 + threadIdx.x], &vsin[threadIdx.x], &vcos[threadIdx.x]);
        __syncthreads();
    }
    float af = 0.f, bf = 0.f;
    int mode = 0;
    if (r < M) {
        if (views) {
            const int k = (int)(r / L.n_det - v0);
            setup_line(g, L, r, hdr, &vsin[k], &vcos[k], af, bf, mode);
        } else {
            setup_line(g, L, r, hdr, nullptr, nullptr, af, bf, mode);
        }
    }
    // the warp's 32 tables (table index = line index), two at a time
    const int half = lane >> 4, hl = lane & 15;
    const unsigned gmask = half ? 0xFFFF0000u : 0x0000FFFFu;
    const int64_t rw = r0 + (int64_t)warp * 32;
    for (int k = 0; k < 16; ++k) {
        const int src = 2 * k + half;   // the lane that set up this half's line
        const float a = __shfl_sync(0xffffffffu, af, src);
        const float b = __shfl_sync(0xffffffffu, bf, src);
        const int64_t rr = rw + src;
        if (rr < M) build_table_half<DEG>(a, b, tabs + rr * kTabFloats, scratch[2 * warp + half], hl, gmask);
        __syncwarp();
    }
}

// ------------------------------------------------------------------ evaluation
// Visit every candidate of every row of one line; `op(node, phi)` is called
// for in-grid candidates (phi may be 0 beyond the support).
template <int DEG, typename Op>
__device__ __forceinline__ void walk_line(const LineHdr &H, const float *tab, const GridDev &g,
                                          int lane, Op op)
{
    const bool vert = H.flags & kVert;
    const int sgn = (H.flags & kKapNeg) ? -1 : 1;
    const int Nq = vert ? g.nx : g.ny;
    const float inv_a = 1.0f / H.a;
    float s[DEG + 1];
#pragma unroll
    for (int q = 0; q <= DEG; ++q) s[q] = tab[q];
    for (int r = H.r_begin + lane; r < H.r_end; r += 32) {
        const RowEval e = row_eval<DEG>(H, s, inv_a, sgn, r);
        for (int i = 0; i < H.K; ++i) {
            int q = e.q0 + sgn * i;
            if ((unsigned)q < (unsigned)Nq) {
                float ti = (DEG == 0) ? __fmaf_rn((float)i, H.a_corr, e.t) : e.t;
                float phi = horner<DEG>(tab + tab_poly(e.sg, i), ti);
                if (DEG == 0 && e.tie) phi = 0.5f * phi;
                int node = vert ? r * g.nx + q : q * g.nx + r;
                op(node, phi);
            }
        }
        if (DEG == 0 && e.tie) {
            // the run also starts at u = 0: midpoint value on that edge too
            int q = e.q0 - sgn;
            if ((unsigned)q < (unsigned)Nq) {
                int node = vert ? r * g.nx + q : q * g.nx + r;
                op(node, 0.5f * inv_a);
            }
        }
    }
}

// Is candidate i of a row in the support (u_0 + i a < 2w; <= for ties)?
template <int DEG>
__device__ __forceinline__ bool candidate_in(const LineHdr &H, const float *s, const RowEval &e, int i,
                                             float bf)
{
    if constexpr (DEG == 0) {
        // u_0 + i|kappa| - (a + b) with u_0 = uhi + ulo and |kappa| = a + a_corr:
        // (uhi - (1-i) a) is exact when it is small, the rest are small terms.
        float d = __fadd_rn(__fsub_rn(e.uhi, (float)(1 - i) * H.a),
                            __fsub_rn(__fmaf_rn((float)i, H.a_corr, e.ulo), bf));
        return (H.flags & kDeg0Axis) ? d <= 0.f : d < 0.f;
    } else {
        float u0 = (e.sg ? s[e.sg - 1] : 0.f) + e.t;
        return __fmaf_rn((float)i, H.a, u0) < H.two_w;
    }
}

template <int DEG>
__global__ void __launch_bounds__(256) fwd_kernel(GridDev g, const LineHdr *__restrict__ hdr,
                                                  const float *__restrict__ tabs, int64_t M,
                                                  const float *__restrict__ coef,
                                                  float *__restrict__ sino)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); line < M;
         line += nw) {
        const LineHdr H = hdr[line];
        float acc = 0.f;
        if (!(H.flags & kEmpty)) {
            const float *tab = tabs + (int64_t)H.tab * kTabFloats;
            walk_line<DEG>(H, tab, g, lane, [&](int node, float phi) {
                acc = __fmaf_rn(__ldg(coef + node), phi, acc);
            });
        }
        acc = warp_sum(acc);
        if (lane == 0) sino[line] = g.h * acc;
    }
}

template <int DEG>
__global__ void __launch_bounds__(256) adj_kernel(GridDev g, const LineHdr *__restrict__ hdr,
                                                  const float *__restrict__ tabs, int64_t M,
                                                  const float *__restrict__ sino,
                                                  float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); line < M;
         line += nw) {
        const LineHdr H = hdr[line];
        if (H.flags & kEmpty) continue;
        const float hp = g.h * __ldg(sino + line);
        if (hp == 0.f) continue;
        const float *tab = tabs + (int64_t)H.tab * kTabFloats;
        walk_line<DEG>(H, tab, g, lane, [&](int node, float phi) {
            atomicAdd(out + node, hp * phi);
        });
    }
}

template <int DEG>
__global__ void visited_kernel(GridDev g, const LineHdr *__restrict__ hdr,
                               const float *__restrict__ tabs, int64_t M, int32_t *counts,
                               const int64_t *offsets, int32_t *nodes)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); line < M;
         line += nw) {
        const LineHdr H = hdr[line];
        int total = 0;
        if (!(H.flags & kEmpty)) {
            const float *tab = tabs + (int64_t)H.tab * kTabFloats;
            const bool vert = H.flags & kVert;
            const int sgn = (H.flags & kKapNeg) ? -1 : 1;
            const int Nq = vert ? g.nx : g.ny;
            const float inv_a = 1.0f / H.a;
            // b of the table: 2w = m (a + b)
            const float bf = tab[kTabB];   // b the table was built with
            float s[DEG + 1];
#pragma unroll
            for (int q = 0; q <= DEG; ++q) s[q] = tab[q];
            const int64_t base = offsets ? offsets[line] : 0;
            // rows in rounds of 32 so that every lane's writes have a place
            for (int r0 = H.r_begin; r0 < H.r_end; r0 += 32) {
                const int r = r0 + lane;
                int cnt = 0;
                RowEval e{0, 0, 0.f, false, 0.f, 0.f};
                if (r < H.r_end) {
                    e = row_eval<DEG>(H, s, inv_a, sgn, r);
                    for (int i = 0; i < H.K; ++i) {
                        int q = e.q0 + sgn * i;
                        if ((unsigned)q < (unsigned)Nq && candidate_in<DEG>(H, s, e, i, bf)) ++cnt;
                    }
                    if (e.tie && (unsigned)(e.q0 - sgn) < (unsigned)Nq) ++cnt;
                }
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int excl = incl - cnt;
                const int round_total = __shfl_sync(0xffffffffu, incl, 31);
                if (nodes && offsets && cnt > 0) {
                    int64_t pos = base + total + excl;
                    for (int i = 0; i < H.K; ++i) {
                        int q = e.q0 + sgn * i;
                        if ((unsigned)q < (unsigned)Nq && candidate_in<DEG>(H, s, e, i, bf))
                            nodes[pos++] = vert ? r * g.nx + q : q * g.nx + r;
                    }
                    if (e.tie && (unsigned)(e.q0 - sgn) < (unsigned)Nq) {
                        int q = e.q0 - sgn;
                        nodes[pos++] = vert ? r * g.nx + q : q * g.nx + r;
                    }
                }
                total += round_total;
            }
        }
        if (lane == 0) counts[line] = total;
    }
}

__global__ void expand_kernel(LinesDev L, int64_t M, float *theta_out, float *y_out)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    if (L.kind == SP_LINES_THETA_Y) {
        if (theta_out) theta_out[r] = L.theta[r];
        if (y_out) y_out[r] = L.y[r];
        return;
    }
    double dx, dy, px, py;
    line_geometry(L, r, dx, dy, px, py);
    if (theta_out) theta_out[r] = (float)atan2(dy, dx);
    if (y_out) y_out[r] = (float)(px * dy - py * dx);
}

template <int DEG>
__device__ float footprint_from_table(const float *tab, float a, float b, int mode, float yt)
{
    // The offset is split in double so that the probe measures the table only.
    float two_w;
    double w;
    int K;
    support_params(DEG, a, b, mode, two_w, w, K);
    const double u = (double)yt + w;
    const bool ties = (DEG == 0) && (b == 0.f);
    const double tw = 2.0 * w;
    if (ties) {
        if (u < 0.0 || u > tw) return 0.f;
        if (u == 0.0 || u == tw) return 0.5f / a;
    } else if (u <= 0.0 || u >= tw) {
        return 0.f;
    }
    int i = (int)ceil(u / (double)a) - 1;
    double u0d = u - (double)i * (double)a;
    if (u0d <= 0.0) { i -= 1; u0d += (double)a; }
    else if (u0d > (double)a) { i += 1; u0d -= (double)a; }
    if (i < 0 || i >= K) return 0.f;
    float s_lo;
    const float u0 = (float)u0d;
    int sg = sigma_of<DEG>(tab, u0, s_lo);
    return horner<DEG>(tab + tab_poly(sg, i), (float)(u0d - (double)s_lo));
}

template <int DEG>
__global__ void footprint_eval_kernel(int64_t count, const float *theta, const float *yt, float *out, int basis)
{
    __shared__ __align__(16) float scratch[kTabWarps][kBuildScratch];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * kTabWarps + warp;
    if (r >= count) return;
    double s, c;
    sincos((double)theta[r], &s, &c);
    float af, bf;
    footprint_ab(DEG, c, s, af, bf);
    const int mode = footprint_mode(basis, c, s);
    if (DEG == 2 && mode != kModeBspline) build_table_box(af, bf, mode, nullptr, scratch[warp], lane);
    else if (lane < 16) build_table_half<DEG>(af, bf, nullptr, scratch[warp], lane, 0x0000FFFFu);
    __syncwarp();
    if (lane == 0) out[r] = footprint_from_table<DEG>(scratch[warp], af, bf, mode, yt[r]);
}

inline unsigned blocks_for(int64_t n, int per)
{
    int64_t b = (n + per - 1) / per;
    return (unsigned)(b < 1 ? 1 : b);
}

inline unsigned warp_blocks(int64_t lines)
{
    // 8 warps per block, grid-stride; enough blocks for several waves on 152 SMs
    int64_t b = (lines + 7) / 8;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

#define SPX_DISPATCH(DEGVAR, KERNEL, GRID, BLOCK, STREAM, ...)                          \
    switch (DEGVAR) {                                                                     \
    case 0: KERNEL<0><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                    \
    case 1: KERNEL<1><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                    \
    case 2: KERNEL<2><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                    \
    default: KERNEL<3><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                   \
    }

cudaError_t launch_setup(const GridDev &g, const LinesDev &L, LineHdr *hdr, float *tabs, cudaStream_t s)
{
    if (L.m <= 0) return cudaSuccess;
    setup_kernel<<<blocks_for(L.m, kSetupThreads), kSetupThreads, 0, s>>>(g, L, hdr, tabs, L.m);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const GridDev &g, const LinesDev &L, LineHdr *hdr, float *tabs, int64_t n_tab,
                           cudaStream_t s)
{
    if (L.m <= 0) return cudaSuccess;
    // one table per line: setup and tables in one kernel, where there are
    // enough lines for warps at the FP64 stage and warps at the table stage to
    // coexist (at least two waves of four 256-line blocks per SM; with fewer,
    // all warps pass through both stages together and two kernels are faster)
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t wave = (int64_t)sms * 4 * kTabWarps * 32;
    if (g.basis == SP_BASIS_BSPLINE && L.kind != SP_LINES_PARALLEL && L.m >= 2 * wave) {
        SPX_DISPATCH(g.kdeg, setup_tables_kernel, blocks_for(L.m, kTabWarps * 32), kTabWarps * 32, s, g, L, hdr, tabs,
                     L.m);
        return cudaGetLastError();
    }
    e = launch_setup(g, L, hdr, tabs, s);
    if (e == cudaSuccess) e = launch_tables(g, L, tabs, n_tab, s);
    return e;
}

cudaError_t launch_tables(const GridDev &g, const LinesDev &L, float *tabs, int64_t n_tab,
                          cudaStream_t s)
{
    (void)L;
    if (n_tab <= 0) return cudaSuccess;
    SPX_DISPATCH(g.kdeg, tables_kernel, blocks_for(n_tab, 2 * kTabWarps), kTabWarps * 32, s, tabs, n_tab);
    return cudaGetLastError();
}

cudaError_t launch_fwd(const GridDev &g, const LineHdr *hdr, const float *tabs, int64_t m,
                       const float *coef, float *sino, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    SPX_DISPATCH(g.kdeg, fwd_kernel, warp_blocks(m), 256, s, g, hdr, tabs, m, coef, sino);
    return cudaGetLastError();
}

cudaError_t launch_adj(const GridDev &g, const LineHdr *hdr, const float *tabs, int64_t m,
                       const float *sino, float *coef_out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(coef_out, 0, sizeof(float) * (size_t)g.nx * (size_t)g.ny, s);
    if (e != cudaSuccess || m <= 0) return e;
    SPX_DISPATCH(g.kdeg, adj_kernel, warp_blocks(m), 256, s, g, hdr, tabs, m, sino, coef_out);
    return cudaGetLastError();
}

cudaError_t launch_visited(const GridDev &g, const LineHdr *hdr, const float *tabs, int64_t m,
                           int32_t *counts, const int64_t *offsets, int32_t *nodes,
                           cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    SPX_DISPATCH(g.kdeg, visited_kernel, warp_blocks(m), 256, s, g, hdr, tabs, m, counts,
                 offsets, nodes);
    return cudaGetLastError();
}

cudaError_t launch_expand(const LinesDev &L, float *theta_out, float *y_out, cudaStream_t s)
{
    if (L.m <= 0) return cudaSuccess;
    expand_kernel<<<blocks_for(L.m, 256), 256, 0, s>>>(L, L.m, theta_out, y_out);
    return cudaGetLastError();
}

cudaError_t launch_footprint_eval(const GridDev &g, int64_t count, const float *theta, const float *yt,
                                  float *out, float *scratch, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    (void)scratch;
    SPX_DISPATCH(g.kdeg, footprint_eval_kernel, blocks_for(count, kTabWarps), kTabWarps * 32, s, count, theta, yt,
                 out, g.basis);
    return cudaGetLastError();
}

}  // namespace spx
