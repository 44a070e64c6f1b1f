// Forward projection and adjoint for structured geometries (parallel and fan
// beams) with coefficient strips in shared memory.
//
// One CTA takes a chunk of up to kChunk neighbouring lines of one view
// (consecutive detector bins).  Such lines are nearly parallel and adjacent,
// so in every major-axis row their runs of nonzero nodes fall inside a short
// window; the CTA keeps those windows (a skewed strip, one row per major-axis
// row) in shared memory: staged from the coefficients for the forward
// projection, accumulated and then added to the output for the adjoint.
// Lines whose major axis is x1 use transposed images so that strip rows stay
// contiguous in global memory.
//
// Per line (one warp), a lane takes one major-axis row at a time and all of
// its candidates, two at a time with packed FP32 FMAs (fma.rn.f32x2): the
// Horner schemes of a candidate pair advance in one instruction.  The line's
// footprint table sits in the warp's shared memory; its 16-byte loads are
// broadcasts, since the lanes of a warp touch at most n+2 of its intervals.
#include <climits>

#include "common.cuh"

namespace spx {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kChunk = 32;          // lines per chunk
constexpr int kPitch = 41;          // strip row length (floats); odd, so consecutive rows hit different banks
constexpr int kSlabRows = 512;      // strip rows held at once

constexpr size_t kStripBytes = sizeof(float) * ((kSlabRows * kPitch + 3) & ~3);
constexpr size_t kCloBytes = sizeof(int) * kSlabRows;
// Each warp's copy of its current table, interval blocks padded from 64 to 68
// floats so that the blocks of different intervals start on different banks.
constexpr int kSigStrideS = kSigStride + 4;
constexpr int kTabFloatsS = kTabHead + kMaxSig * kSigStrideS;
constexpr size_t kTabWarpBytes = sizeof(float) * kWarps * kTabFloatsS;
constexpr size_t kAccBytes = sizeof(float) * kChunk;
constexpr size_t kMiscBytes = 32 + 4 * 64;
constexpr size_t kHdrBytes = sizeof(LineHdr) * kChunk;
constexpr size_t kSmemBytes = kStripBytes + kCloBytes + kTabWarpBytes + kAccBytes + kMiscBytes + kHdrBytes;

// ------------------------------------------------------------------ packed FP32
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2pack(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void f2unpack(f2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ void red_shared(float *p, float v)
{
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "f"(v)
                 : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

constexpr int kTabLines = (kTabFloats * 4 + 127) / 128;   // 128-byte lines of one table

// First and last column of the run of line H in row r, for a run of K nodes.
__device__ __forceinline__ void run_columns(const LineHdr &H, float inv_a, int r, int &lo, int &hi)
{
    int k;
    row_start(H, inv_a, r, k);
    const int sgn = (H.flags & kKapNeg) ? -1 : 1;
    const int q0 = H.q_ref - sgn * k;
    const int q1 = q0 + sgn * (H.K - 1);
    lo = min(q0, q1);
    hi = max(q0, q1);
}

// One line over the strip rows [S0, S1).  Forward (ADJ false): returns
// sum_k c_k phi (no factor h).  Adjoint: adds hp * phi into the strip.
//
// Lane l takes rows S0' + l, S0' + l + 32, ...  The line's footprint table
// has been copied to this warp's shared memory (tabw); a row in interval
// sigma evaluates candidate pair p with the packed polynomials at
// tab_poly(sigma, 2p).  Lanes of one warp touch at most n+2 different
// intervals, so each 16-byte table load is a broadcast of few addresses.
template <int DEG, bool ADJ>
__device__ float strip_line(const LineHdr &H, const float *tabw, const float *__restrict__ tab, float *strip,
                            const int *clo, int S0, int S1, int lane, const float *__restrict__ src,
                            float *dst, int Nq, int *err, float hp)
{
    constexpr int NC = 2 * DEG + 2;
    const int sgn = (H.flags & kKapNeg) ? -1 : 1;
    const float inv_a = 1.0f / H.a;
    float s[DEG + 1];
#pragma unroll
    for (int q = 0; q <= DEG; ++q) s[q] = tabw[q];
    const int K = H.K;
    const int np = (K + 1) >> 1;
    const bool odd = K & 1;
    f2 acc2 = 0ull, acc2b = 0ull;
    float acc_slow = 0.f;

    const int rb = max(H.r_begin, S0), re = min(H.r_end, S1);
    for (int r = rb + lane; r < re; r += 32) {
        const RowEval e = row_eval<DEG>(H, s, inv_a, sgn, r);
        const int rr = r - S0;
        const int oq = e.q0 - clo[rr];
        const int lo = sgn > 0 ? oq : oq - (K - 1);
        const int hi = sgn > 0 ? oq + (K - 1) : oq;
        if (lo >= 0 && hi < kPitch) {
            const float *row = strip + rr * kPitch + oq;
            const f2 tt = f2pack(e.t, e.t);
            const float *T = tabw + kTabHead + e.sg * kSigStrideS;
            for (int p = 0; p < np; ++p) {
                const ulonglong2 *tp = reinterpret_cast<const ulonglong2 *>(T + p * 2 * kNC);
                f2 Tp[NC];
#pragma unroll
                for (int v = 0; v < NC / 2; ++v) {
                    const ulonglong2 x = tp[v];
                    Tp[2 * v] = x.x;
                    Tp[2 * v + 1] = x.y;
                }
                f2 ph = Tp[NC - 1];
#pragma unroll
                for (int d = NC - 2; d >= 0; --d) ph = f2fma(ph, tt, Tp[d]);
                const bool has_b = !(odd && p == np - 1);
                const int ia = sgn * 2 * p;
                if constexpr (ADJ) {
                    float pa, pb;
                    f2unpack(ph, pa, pb);
                    red_shared(const_cast<float *>(row) + ia, hp * pa);
                    if (has_b) red_shared(const_cast<float *>(row) + ia + sgn, hp * pb);
                } else {
                    const float ca = row[ia];
                    const float cb = has_b ? row[ia + sgn] : 0.f;
                    if (p & 1) acc2b = f2fma(f2pack(ca, cb), ph, acc2b);
                    else acc2 = f2fma(f2pack(ca, cb), ph, acc2);
                }
            }
        } else {
            // run outside the staged window: straight from or to global memory
            atomicAdd(err, 1);
            for (int i = 0; i < K; ++i) {
                const int q = e.q0 + sgn * i;
                if ((unsigned)q < (unsigned)Nq) {
                    const float phi = horner<DEG>(tab + tab_poly(e.sg, i), e.t);
                    if constexpr (ADJ) atomicAdd(dst + (size_t)r * Nq + q, hp * phi);
                    else acc_slow = __fmaf_rn(__ldg(src + (size_t)r * Nq + q), phi, acc_slow);
                }
            }
        }
    }
    if constexpr (ADJ) {
        return 0.f;
    } else {
        float a0, a1, b0, b1;
        f2unpack(acc2, a0, a1);
        f2unpack(acc2b, b0, b1);
        return warp_sum((a0 + a1) + (b0 + b1) + acc_slow);
    }
}

// Forward (ADJ false): sino[line] = h sum c phi.  Adjoint (ADJ true): adds
// h sino[line] phi to out (vertical lines) or outT (horizontal lines, the
// transposed image).
template <int DEG, bool ADJ>
__global__ void __launch_bounds__(kThreads, 2)
strip_kernel(GridDev g, LinesDev L, const LineHdr *__restrict__ hdr, const float *__restrict__ tabs,
             const float *__restrict__ coef, const float *__restrict__ coefT, float *__restrict__ sino,
             float *__restrict__ out, float *__restrict__ outT, int chunks_per_view, int *err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *strip = reinterpret_cast<float *>(smem);
    size_t o = kStripBytes;
    int *clo = reinterpret_cast<int *>(smem + o);
    o += kCloBytes;
    float *tabw_all = reinterpret_cast<float *>(smem + o);
    o += kTabWarpBytes;
    float *line_acc = reinterpret_cast<float *>(smem + o);
    o += kAccBytes;
    int *misc = reinterpret_cast<int *>(smem + o);
    o += kMiscBytes;
    int *gstack = misc + 8;   // pending line groups, (first | last << 8)
    LineHdr *hdr_s = reinterpret_cast<LineHdr *>(smem + o);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *tabw = tabw_all + warp * kTabFloatsS;
    const int v = blockIdx.x / chunks_per_view, cb = blockIdx.x - v * chunks_per_view;
    const int j0 = cb * kChunk;
    const int nl = min(kChunk, L.n_det - j0);
    const int64_t line0 = (int64_t)v * L.n_det + j0;

    if (!ADJ && threadIdx.x < kChunk) line_acc[threadIdx.x] = 0.f;
    // the chunk's line records into shared memory, its tables towards L2
    for (int i = threadIdx.x; i < nl * 4; i += kThreads)
        reinterpret_cast<int4 *>(hdr_s)[i] = __ldg(reinterpret_cast<const int4 *>(hdr + line0) + i);
    if (L.kind != SP_LINES_PARALLEL)
        for (int i = threadIdx.x; i < nl * kTabLines; i += kThreads)
            prefetch_l2(tabs + (line0 + i / kTabLines) * (int64_t)kTabFloats + (i % kTabLines) * 32);

    for (int axis = 0; axis < 2; ++axis) {
        __syncthreads();
        if (warp == 0) {
            bool mine = false;
            if (lane < nl) {
                const LineHdr &H = hdr_s[lane];
                mine = !(H.flags & kEmpty) && (((H.flags & kVert) != 0) == (axis == 0)) && H.r_end > H.r_begin;
                if (ADJ && mine) mine = sino[line0 + lane] != 0.f;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, mine);
            if (lane == 0) {
                misc[0] = (int)mask;
                if (mask) { gstack[0] = (__ffs(mask) - 1) | ((31 - __clz(mask)) << 8); misc[3] = 1; }
                else misc[3] = 0;
            }
        }
        __syncthreads();
        const unsigned mask = (unsigned)misc[0];
        if (mask == 0u) continue;
        const bool vert = (axis == 0);
        const int Nq = vert ? g.nx : g.ny;
        const float *src = vert ? coef : coefT;
        float *dst = vert ? out : outT;
        // Groups of lines whose runs fit the pitch; a group that is too wide
        // (lines fanning out) is split in halves.
        for (;;) {
            __syncthreads();
            const int sp = misc[3];
            if (sp == 0) break;
            const int top = gstack[sp - 1];
            const int ga = top & 255, gb = top >> 8;
            const unsigned span = (gb >= 31 ? 0xffffffffu : ((1u << (gb + 1)) - 1u)) & ~((1u << ga) - 1u);
            const unsigned gmask = mask & span;
            __syncthreads();
            if (threadIdx.x == 0) { misc[3] = sp - 1; misc[4] = 0; }
            if (gmask == 0u) continue;
            const int first = __ffs(gmask) - 1, last = 31 - __clz(gmask);
            const LineHdr Hf = hdr_s[first], Hl = hdr_s[last];
            const float inv_af = 1.0f / Hf.a, inv_al = 1.0f / Hl.a;
            // row range of the group (lane = line), and the widest window:
            // the outermost runs move linearly with the row, so it is at an end
            int R0 = INT_MAX, R1 = INT_MIN;
            if ((gmask >> lane) & 1u) { R0 = hdr_s[lane].r_begin; R1 = hdr_s[lane].r_end; }
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                R0 = min(R0, __shfl_xor_sync(0xffffffffu, R0, o2));
                R1 = max(R1, __shfl_xor_sync(0xffffffffu, R1, o2));
            }
            int wmax = 0;
            {
                int lo1, hi1, lo2, hi2;
                run_columns(Hf, inv_af, R0, lo1, hi1);
                run_columns(Hl, inv_al, R0, lo2, hi2);
                wmax = max(hi1, hi2) - min(lo1, lo2) + 5;
                run_columns(Hf, inv_af, R1 - 1, lo1, hi1);
                run_columns(Hl, inv_al, R1 - 1, lo2, hi2);
                wmax = max(wmax, max(hi1, hi2) - min(lo1, lo2) + 5);
            }
            __syncthreads();
            if (wmax > kPitch && first < last) {
                if (threadIdx.x == 0) {
                    const int mid = (first + last) >> 1;
                    const int s2 = misc[3];
                    gstack[s2] = first | (mid << 8);
                    gstack[s2 + 1] = (mid + 1) | (last << 8);
                    misc[3] = s2 + 2;
                }
                continue;
            }
            for (int S0 = R0; S0 < R1; S0 += kSlabRows) {
                const int S1 = min(S0 + kSlabRows, R1);
                const int nrows = S1 - S0;
                __syncthreads();
                // window of each strip row from the two outermost lines of the
                // group (lines of a view do not cross inside the grid), margin 2
                for (int rr = threadIdx.x; rr < nrows; rr += kThreads) {
                    int lo1, hi1, lo2, hi2;
                    run_columns(Hf, inv_af, S0 + rr, lo1, hi1);
                    run_columns(Hl, inv_al, S0 + rr, lo2, hi2);
                    const int lo = min(lo1, lo2) - 2, hi = max(hi1, hi2) + 2;
                    clo[rr] = lo - max(0, (kPitch - (hi - lo + 1)) / 2);
                }
                __syncthreads();
                if constexpr (ADJ) {
                    for (int i = threadIdx.x; i < nrows * kPitch; i += kThreads) strip[i] = 0.f;
                } else {
                    // asynchronous copies, zero-filled outside the grid; one wait
                    for (int rr = warp; rr < nrows; rr += kWarps) {
                        const int c0 = clo[rr];
                        const float *row = src + (size_t)(S0 + rr) * Nq;
                        for (int cc = lane; cc < kPitch; cc += 32) {
                            const int q = c0 + cc;
                            const bool in = (unsigned)q < (unsigned)Nq;
                            const unsigned dsts = (unsigned)__cvta_generic_to_shared(strip + rr * kPitch + cc);
                            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dsts),
                                         "l"(in ? row + q : src), "r"(in ? 4 : 0)
                                         : "memory");
                        }
                    }
                    asm volatile("cp.async.wait_all;" ::: "memory");
                }
                __syncthreads();
                for (int li = first + warp; li <= last; li += kWarps) {
                    if (!((gmask >> li) & 1u)) continue;
                    const LineHdr H = hdr_s[li];
                    const float *tab = tabs + (int64_t)H.tab * kTabFloats;
                    const float hp = ADJ ? g.h * sino[line0 + li] : 0.f;
                    __syncwarp();
                    for (int i = lane; i < kTabFloats / 4; i += 32) {
                        // head (2 float4), then 16 float4 per interval block
                        const int blk = i < 2 ? -1 : (i - 2) >> 4;
                        const int dst4 = i < 2 ? i : 2 + blk * (kSigStrideS / 4) + ((i - 2) & 15);
                        reinterpret_cast<float4 *>(tabw)[dst4] = __ldg(reinterpret_cast<const float4 *>(tab) + i);
                    }
                    __syncwarp();
                    const float sum = strip_line<DEG, ADJ>(H, tabw, tab, strip, clo, S0, S1, lane, src, dst, Nq,
                                                           err, hp);
                    if (!ADJ && lane == 0) line_acc[li] += sum;
                }
                if constexpr (ADJ) {
                    __syncthreads();
                    // add the accumulated strip into the image, row by row
                    for (int rr = warp; rr < nrows; rr += kWarps) {
                        const int c0 = clo[rr];
                        float *row = dst + (size_t)(S0 + rr) * Nq;
                        for (int cc = lane; cc < kPitch; cc += 32) {
                            const int q = c0 + cc;
                            const float val = strip[rr * kPitch + cc];
                            if ((unsigned)q < (unsigned)Nq && val != 0.f) atomicAdd(row + q, val);
                        }
                    }
                }
            }
        }
    }
    if constexpr (!ADJ) {
        __syncthreads();
        if (threadIdx.x < nl) sino[line0 + threadIdx.x] = g.h * line_acc[threadIdx.x];
    }
}

__global__ void transpose_kernel(const float *__restrict__ in, float *__restrict__ out, int nx, int ny)
{
    __shared__ float tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int i = bx + threadIdx.x, j = by + y;
        if (i < nx && j < ny) tile[y][threadIdx.x] = in[(size_t)j * nx + i];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int j = by + threadIdx.x, i = bx + y;
        if (i < nx && j < ny) out[(size_t)i * ny + j] = tile[threadIdx.x][y];
    }
}

// out[j][i] += inT[i][j]
__global__ void add_transposed_kernel(const float *__restrict__ inT, float *__restrict__ out, int nx, int ny)
{
    __shared__ float tile[32][33];
    const int bi = blockIdx.x * 32, bj = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int i = bi + y, j = bj + threadIdx.x;
        if (i < nx && j < ny) tile[y][threadIdx.x] = inT[(size_t)i * ny + j];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int j = bj + y, i = bi + threadIdx.x;
        if (i < nx && j < ny) out[(size_t)j * nx + i] += tile[threadIdx.x][y];
    }
}

template <int DEG, bool ADJ>
cudaError_t launch_strip_t(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                           const float *coef, float *imgT, float *sino, float *out, int *err, cudaStream_t s)
{
    const dim3 tb(32, 8), tg((g.nx + 31) / 32, (g.ny + 31) / 32);
    cudaError_t e;
    if (!ADJ) {
        transpose_kernel<<<tg, tb, 0, s>>>(coef, imgT, g.nx, g.ny);
    } else {
        e = cudaMemsetAsync(out, 0, sizeof(float) * (size_t)g.nx * g.ny, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(imgT, 0, sizeof(float) * (size_t)g.nx * g.ny, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(strip_kernel<DEG, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    const int cpv = (L.n_det + kChunk - 1) / kChunk;
    const unsigned grid = (unsigned)(L.n_view * cpv);
    strip_kernel<DEG, ADJ><<<grid, kThreads, kSmemBytes, s>>>(g, L, hdr, tabs, coef, imgT,
                                                              const_cast<float *>(sino), out, imgT, cpv, err);
    e = cudaGetLastError();
    if (e == cudaSuccess && ADJ) {
        add_transposed_kernel<<<tg, tb, 0, s>>>(imgT, out, g.nx, g.ny);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

bool strip_supported(const GridDev &g, const LinesDev &L)
{
    return (L.kind == SP_LINES_PARALLEL || L.kind == SP_LINES_FAN) && g.degree >= 1;
}

size_t strip_scratch_bytes(const GridDev &g) { return sizeof(float) * (size_t)g.nx * g.ny + 256; }

cudaError_t launch_fwd_strip(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                             const float *coef, void *scratch, float *sino, int *err, cudaStream_t s)
{
    float *coefT = static_cast<float *>(scratch);
    switch (g.degree) {
    case 1: return launch_strip_t<1, false>(g, L, hdr, tabs, coef, coefT, sino, nullptr, err, s);
    case 2: return launch_strip_t<2, false>(g, L, hdr, tabs, coef, coefT, sino, nullptr, err, s);
    default: return launch_strip_t<3, false>(g, L, hdr, tabs, coef, coefT, sino, nullptr, err, s);
    }
}

cudaError_t launch_adj_strip(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                             const float *sino, void *scratch, float *coef_out, int *err, cudaStream_t s)
{
    float *outT = static_cast<float *>(scratch);
    float *p = const_cast<float *>(sino);
    switch (g.degree) {
    case 1: return launch_strip_t<1, true>(g, L, hdr, tabs, nullptr, outT, p, coef_out, err, s);
    case 2: return launch_strip_t<2, true>(g, L, hdr, tabs, nullptr, outT, p, coef_out, err, s);
    default: return launch_strip_t<3, true>(g, L, hdr, tabs, nullptr, outT, p, coef_out, err, s);
    }
}

}  // namespace spx
