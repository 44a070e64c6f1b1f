// Chunk order of a free line list (THETA_Y or POINTS) for the strip kernels.
//
// The strip kernels stage, for a chunk of 32 lines, the short window of
// coefficient rows that the lines' runs cover (Alg. 2 restricted to one
// major-axis row, Lemma 1).  Parallel and fan beams get such chunks for free
// (neighbouring bins of one view); a free list is first sorted so that 32
// consecutive lines of the order are nearly parallel neighbours:
//
//   key = axis (1 bit) | direction bucket (10 bits) | offset (16 bits),
//
// with the direction the slope dq/dr of the line's run (|slope| <= 1 along
// the major axis) cut into D buckets, and the offset the run's centre column
// at the grid's middle row.  D balances the two ways a chunk widens: with m
// lines, a bucket holds ~m/D lines spread over the grid's width, so 32 of them
// span ~32 sqrt(2) N D / m columns, while the slopes within a bucket differ by
// up to 2/D, i.e. N/D columns over half the grid; the sum is smallest at
// D = sqrt(m / (32 sqrt(2))).  Empty lines sort last.
//
// The sort is a stable LSD radix sort of (key, line index) with 8-bit digits
// in four passes (count per block, one exclusive scan, stable scatter with
// warp-level matching), so the order (and with it every projection's
// summation order) is deterministic.
#include <cmath>

#include "common.cuh"

namespace spx {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kPerThread = 8;
constexpr int kTile = kSortThreads * kPerThread;   // keys per block and pass
constexpr int kDigits = 256;
constexpr int kScanThreads = 1024;

size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

__global__ void order_keys_kernel(GridDev g, const LineHdr *__restrict__ hdr, int m, int D,
                                  unsigned *__restrict__ keys, int *__restrict__ vals)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const LineHdr H = hdr[i];
    unsigned key = 0xffffffffu;
    if (!(H.flags & kEmpty) && H.r_end > H.r_begin) {
        const bool vert = (H.flags & kVert) != 0;
        const int Nr = vert ? g.ny : g.nx, Nq = vert ? g.nx : g.ny;
        const float sgn = (H.flags & kKapNeg) ? -1.f : 1.f;
        // column where u(r, q) = U0 + (r - r_ref) rho + (q - q_ref) kappa
        // reaches the support's centre w, kappa = sgn a: the run's centre
        const float rho = H.rho_hi + H.rho_lo;
        const float w = 0.5f * H.two_w;
        auto centre = [&](float r) { return (float)H.q_ref + sgn * (w - H.U0 - (r - (float)H.r_ref) * rho) / H.a; };
        const float qa = centre(0.f), qb = centre((float)(Nr - 1));
        const float slope = Nr > 1 ? (qb - qa) / (float)(Nr - 1) : 0.f;
        const float c = 0.5f * (qa + qb);
        const float fd = floorf((slope + 1.f) * 0.5f * (float)D);
        const int db = (int)fminf(fmaxf(fd, 0.f), (float)(D - 1));
        const float fo = floorf((c + (float)Nq) / (3.f * (float)Nq) * 65536.f);
        const int ob = (int)fminf(fmaxf(fo, 0.f), 65535.f);
        key = ((vert ? 1u : 0u) << 26) | ((unsigned)db << 16) | (unsigned)ob;
    }
    keys[i] = key;
    vals[i] = i;
}

// counts[d * nb + b] = keys of block b whose digit is d.
__global__ void __launch_bounds__(kSortThreads) radix_count_kernel(const unsigned *__restrict__ keys, int m,
                                                                   int shift, int *__restrict__ counts, int nb)
{
    __shared__ int hist[kDigits];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kTile;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const long long i = base + j * kSortThreads + threadIdx.x;
        if (i < m) atomicAdd(&hist[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * nb + blockIdx.x] = hist[threadIdx.x];
}

// Exclusive prefix sum of counts[0..n) in place, one block.
__global__ void __launch_bounds__(kScanThreads) radix_scan_kernel(int *__restrict__ counts, int n)
{
    __shared__ int wsum[kScanThreads / 32];
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += counts[i];
    // block-wide exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
        int vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        wsum[lane] = vi - v;
    }
    __syncthreads();
    int run = wsum[warp] + inc - s;
    for (int i = lo; i < hi; ++i) {
        const int c = counts[i];
        counts[i] = run;
        run += c;
    }
}

// Stable scatter of one block's keys by the digit at `shift`: warp w owns
// positions [w 256, w 256 + 256) of the block's tile, taken in 8 rounds of 32
// consecutive keys; a key's place among equal digits is (earlier blocks, from
// the scanned counts) + (earlier warps of the block) + (earlier rounds of its
// warp) + (lower lanes of its round).
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const unsigned *__restrict__ kin,
                                                                     const int *__restrict__ vin,
                                                                     unsigned *__restrict__ kout,
                                                                     int *__restrict__ vout, int m, int shift,
                                                                     const int *__restrict__ counts, int nb)
{
    __shared__ int wcnt[kSortWarps][kDigits];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kDigits; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kTile + warp * (32 * kPerThread);
    unsigned key[kPerThread];
    int val[kPerThread], dig[kPerThread];
    unsigned peers[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const long long i = base + j * 32 + lane;
        const bool ok = i < m;
        key[j] = ok ? kin[i] : 0u;
        val[j] = ok ? vin[i] : 0;
        dig[j] = ok ? (int)((key[j] >> shift) & 255u) : kDigits;   // kDigits: no key
        peers[j] = __match_any_sync(0xffffffffu, dig[j]);
        if (dig[j] < kDigits && lane == __ffs(peers[j]) - 1) wcnt[warp][dig[j]] += __popc(peers[j]);
        __syncwarp();
    }
    __syncthreads();
    {
        // per digit: the block's global start, then each warp's start
        const int d = threadIdx.x;
        int run = counts[(size_t)d * nb + blockIdx.x];
        for (int w = 0; w < kSortWarps; ++w) {
            const int c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const bool ok = dig[j] < kDigits;
        int pos = 0;
        if (ok) pos = wcnt[warp][dig[j]] + __popc(peers[j] & lt);
        __syncwarp();
        if (ok) {
            kout[pos] = key[j];
            vout[pos] = val[j];
            if (lane == __ffs(peers[j]) - 1) wcnt[warp][dig[j]] += __popc(peers[j]);
        }
        __syncwarp();
    }
}

struct OrderArea {
    int *order;        // the result (values of the last pass)
    unsigned *keysA, *keysB;
    int *valsB;
    int *counts;
};

OrderArea carve(void *area, int64_t m)
{
    char *p = static_cast<char *>(area);
    const size_t a = al(sizeof(int) * (size_t)m);
    OrderArea o;
    o.order = reinterpret_cast<int *>(p);
    o.keysA = reinterpret_cast<unsigned *>(p + a);
    o.keysB = reinterpret_cast<unsigned *>(p + 2 * a);
    o.valsB = reinterpret_cast<int *>(p + 3 * a);
    o.counts = reinterpret_cast<int *>(p + 4 * a);
    return o;
}

}  // namespace

size_t line_order_bytes(int64_t m)
{
    const size_t nb = (size_t)((m + kTile - 1) / kTile);
    return 4 * al(sizeof(int) * (size_t)m) + al(sizeof(int) * kDigits * nb);
}

cudaError_t launch_line_order(const GridDev &g, const LinesDev &L, const LineHdr *hdr, void *area, cudaStream_t s)
{
    const int64_t m = L.m;
    if (m <= 0) return cudaSuccess;
    if (m > 0x7fffffffLL || !area) return cudaErrorInvalidValue;
    const int mi = (int)m;
    const int nb = (int)((m + kTile - 1) / kTile);
    int D = (int)std::lround(std::sqrt((double)m / (32.0 * std::sqrt(2.0))));
    D = D < 1 ? 1 : (D > 1023 ? 1023 : D);
    OrderArea o = carve(area, m);
    order_keys_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(g, hdr, mi, D, o.keysA, o.order);
    cudaError_t e = cudaGetLastError();
    // four 8-bit passes, A -> B -> A -> B -> A: the order ends in o.order
    unsigned *ka = o.keysA, *kb = o.keysB;
    int *va = o.order, *vb = o.valsB;
    for (int pass = 0; pass < 4 && e == cudaSuccess; ++pass) {
        const int shift = 8 * pass;
        radix_count_kernel<<<nb, kSortThreads, 0, s>>>(ka, mi, shift, o.counts, nb);
        radix_scan_kernel<<<1, kScanThreads, 0, s>>>(o.counts, kDigits * nb);
        radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(ka, va, kb, vb, mi, shift, o.counts, nb);
        e = cudaGetLastError();
        unsigned *tk = ka; ka = kb; kb = tk;
        int *tv = va; va = vb; vb = tv;
    }
    return e;
}

}  // namespace spx
