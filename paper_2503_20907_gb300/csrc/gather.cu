// Pixel-driven adjoint (a gather): c'_k = h sum_m p_m phi_theta_m(y~_{m,k})
// evaluated node by node, for parallel and fan beams of degree >= 1.  It is
// the exact transpose of the forward projection (same pairs, same footprint
// tables, Sec. II.B), computed without atomics: each thread owns one node
// and writes it once.
//
// A block owns a tile of kTile x kTile nodes and walks the views.  For one
// view the lines that can touch the tile form one range of consecutive bins
// (the lines of a view do not cross inside the grid); the block stages their
// records (LineHdr), the heads of their footprint tables (the interval ends
// s_q) and their sinogram values in shared memory.  Each thread then finds
// the bin whose line passes closest to its node and walks outward in both
// directions while the node stays inside the footprint's support: per pair,
// u (the offset from the support's start) from the line's stepping constants,
// the candidate index i and u_0 = u - i a, the interval sigma of u_0, and one
// Horner scheme of T[sigma][i] read from the line's table in device memory.
//
// Versus the strip scatter: no strip staging, no reductions, no flush; but a
// pair costs its own polynomial (eight coefficients fetched per pair, where
// the scatter fetches them once per interval and line) and its own interval
// search.  spline_plan_autotune times both and keeps the faster.
#include <cfloat>
#include <climits>

#include "common.cuh"

namespace spx {
namespace {

constexpr int kTile = 16;                  // nodes per tile side; one thread per node
constexpr int kThreads = kTile * kTile;
constexpr int kMaxLines = 384;             // bins of one view staged per pass

struct ViewGeom {
    float sb, cb;   // view angle: sin, cos
};

// Detector offset (the bin coordinate times ddet, plus det0) of the line of
// view (sb, cb) through the point (x, y), in grid world units.
__device__ __forceinline__ float view_offset(const LinesDev &L, float sb, float cb, float x, float y)
{
    if (L.kind == SP_LINES_PARALLEL) {
        // line j: direction (c, s) through y_j (s, -c); a point X lies on the
        // line of offset X . (s, -c)
        return x * sb - y * cb;
    }
    // fan: source S = dso (cb, sb); detector through -dod (cb, sb) along
    // (-sb, cb); the ray from S through X meets it at offset
    // (dso + dod) across / along
    const float dx = x - L.dso * cb, dy = y - L.dso * sb;
    const float along = -(dx * cb + dy * sb);
    const float across = -dx * sb + dy * cb;
    return (L.dso + L.dod) * across / along;
}

template <int DEG>
__global__ void __launch_bounds__(kThreads) gather_adj_kernel(GridDev g, LinesDev L, const LineHdr *__restrict__ hdr,
                                                              const float *__restrict__ tabs,
                                                              const float *__restrict__ sino, float *__restrict__ out)
{
    __shared__ LineHdr hs[kMaxLines];
    __shared__ float4 heads[kMaxLines];   // s_0..s_3 of each staged line's table
    __shared__ float ps[kMaxLines];
    __shared__ int range[2];

    const int ix = blockIdx.x * kTile + (threadIdx.x % kTile);
    const int iy = blockIdx.y * kTile + (threadIdx.x / kTile);
    const bool node_in = ix < g.nx && iy < g.ny;
    const float ic = 0.5f * (g.nx - 1), jc = 0.5f * (g.ny - 1);
    const float x = g.cx + ((float)ix - ic) * g.h, y = g.cy + ((float)iy - jc) * g.h;
    // tile corners, widened by the largest support half-width (n+1)/sqrt(2)
    // nodes and one node
    const float marg = ((float)(g.kdeg + 1) * 0.7072f + 1.0f) * g.h;
    const float x0 = g.cx + ((float)(blockIdx.x * kTile) - ic) * g.h - marg;
    const float x1 = g.cx + ((float)(blockIdx.x * kTile + kTile - 1) - ic) * g.h + marg;
    const float y0 = g.cy + ((float)(blockIdx.y * kTile) - jc) * g.h - marg;
    const float y1 = g.cy + ((float)(blockIdx.y * kTile + kTile - 1) - jc) * g.h + marg;

    float acc = 0.f;
    for (int v = 0; v < L.n_view; ++v) {
        float sb, cb;
        sincosf(L.view[v], &sb, &cb);
        // bins whose lines can touch the tile: the offsets of the widened
        // tile's corners (lines of a view are ordered by offset and do not
        // cross inside the grid), one bin of margin
        if (threadIdx.x == 0) {
            float omin = FLT_MAX, omax = -FLT_MAX;
            const float xs[2] = {x0, x1}, ys[2] = {y0, y1};
            bool ok = true;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    const float o = view_offset(L, sb, cb, xs[a], ys[b]);
                    if (!isfinite(o)) ok = false;
                    omin = fminf(omin, o);
                    omax = fmaxf(omax, o);
                }
            int jl = 0, jh = L.n_det - 1;
            if (ok) {
                const float f0 = (omin - L.det0) / L.ddet, f1 = (omax - L.det0) / L.ddet;
                const float lo = fminf(f0, f1) - 1.0f, hi = fmaxf(f0, f1) + 1.0f;
                jl = lo < 0.f ? 0 : (lo > (float)(L.n_det - 1) ? L.n_det : (int)floorf(lo));
                jh = hi < 0.f ? -1 : (hi > (float)(L.n_det - 1) ? L.n_det - 1 : (int)ceilf(hi));
            }
            range[0] = jl;
            range[1] = jh;
        }
        __syncthreads();
        const int jl = range[0], jh = range[1];
        // passes of at most kMaxLines bins (one pass on the usual geometries)
        for (int jp = jl; jp <= jh; jp += kMaxLines) {
            const int nj = min(kMaxLines, jh - jp + 1);
            __syncthreads();
            const int64_t m0 = (int64_t)v * L.n_det + jp;
            for (int i = threadIdx.x; i < nj * 4; i += kThreads)
                reinterpret_cast<int4 *>(hs)[i] = __ldg(reinterpret_cast<const int4 *>(hdr + m0) + i);
            __syncthreads();
            for (int i = threadIdx.x; i < nj; i += kThreads) {
                ps[i] = sino[m0 + i];
                heads[i] = __ldg(reinterpret_cast<const float4 *>(tabs + (int64_t)hs[i].tab * kTabFloats));
            }
            __syncthreads();
            if (!node_in) continue;
            // the staged bin nearest to this node's own offset, then outward
            const float o = view_offset(L, sb, cb, x, y);
            int jn = isfinite(o) ? (int)floorf((o - L.det0) / L.ddet + 0.5f) - jp : 0;
            jn = max(0, min(nj - 1, jn));
            for (int dir = 0; dir < 2; ++dir) {
                const int step = dir ? -1 : 1;
                int misses = 0;
                for (int jj = dir ? jn - 1 : jn; jj >= 0 && jj < nj; jj += step) {
                    const LineHdr &H = hs[jj];
                    const float p = ps[jj];
                    bool hit = false;
                    if (!(H.flags & kEmpty)) {
                        const bool vert = H.flags & kVert;
                        const int r = vert ? iy : ix, q = vert ? ix : iy;
                        // u = U0 + (r - r_ref) rho + (q - q_ref) kappa, kappa = +-a:
                        // the stepping of the strip kernels (row_u0) with the
                        // step count k = -+(q - q_ref), hi products exact
                        const float fr = (float)(r - H.r_ref);
                        const float fk = (float)((H.flags & kKapNeg) ? (q - H.q_ref) : (H.q_ref - q));
                        const float big = __fsub_rn(__fmul_rn(fr, H.rho_hi), __fmul_rn(fk, H.a_hi));
                        const float small = __fmaf_rn(fr, H.rho_lo, __fmul_rn(-fk, H.a_lo));
                        const float u = __fadd_rn(__fadd_rn(H.U0, small), big);
                        if (u > 0.f && u < H.two_w) {
                            hit = true;
                            int i = (int)ceilf(u / H.a) - 1;
                            float u0 = u - (float)i * H.a;
                            if (u0 <= 0.f) { i -= 1; u0 += H.a; }
                            else if (u0 > H.a) { i += 1; u0 -= H.a; }
                            if (i >= 0 && i < H.K && p != 0.f) {
                                const float4 hd = heads[jj];
                                const float sq[4] = {hd.x, hd.y, hd.z, hd.w};
                                float s_lo;
                                const int sg = sigma_of<DEG>(sq, u0, s_lo);
                                const float4 *T4 = reinterpret_cast<const float4 *>(
                                    tabs + (int64_t)H.tab * kTabFloats + tab_poly(sg, i));
                                const float4 c0 = __ldg(T4), c1 = __ldg(T4 + 1);
                                const float c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
                                constexpr int NC = 2 * DEG + 2;
                                const float t = u0 - s_lo;
                                float ph = c[NC - 1];
#pragma unroll
                                for (int d = NC - 2; d >= 0; --d) ph = __fmaf_rn(ph, t, c[d]);
                                acc = __fmaf_rn(p, ph, acc);
                            }
                        }
                    }
                    // the node leaves the support for good once two lines in a
                    // row miss it (the offsets move monotonically with the bin)
                    misses = hit ? 0 : misses + 1;
                    if (misses >= 2) break;
                }
            }
        }
        __syncthreads();
    }
    if (node_in) out[(size_t)iy * g.nx + ix] = g.h * acc;
}

}  // namespace

bool gather_supported(const GridDev &g, const LinesDev &L)
{
    return (L.kind == SP_LINES_PARALLEL || L.kind == SP_LINES_FAN) && g.kdeg >= 1 && g.basis == SP_BASIS_BSPLINE;
}

cudaError_t launch_adj_gather(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                              const float *sino, float *coef_out, cudaStream_t s)
{
    const dim3 grid((g.nx + kTile - 1) / kTile, (g.ny + kTile - 1) / kTile);
    switch (g.kdeg) {
    case 1: gather_adj_kernel<1><<<grid, kThreads, 0, s>>>(g, L, hdr, tabs, sino, coef_out); break;
    case 2: gather_adj_kernel<2><<<grid, kThreads, 0, s>>>(g, L, hdr, tabs, sino, coef_out); break;
    default: gather_adj_kernel<3><<<grid, kThreads, 0, s>>>(g, L, hdr, tabs, sino, coef_out); break;
    }
    return cudaGetLastError();
}

}  // namespace spx
