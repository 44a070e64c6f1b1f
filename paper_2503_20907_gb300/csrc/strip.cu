// Forward projection and adjoint with coefficient strips in shared memory,
// for parallel and fan beams and for free line lists sorted into the same
// kind of chunks (order.cu).
//
// One CTA takes a chunk of up to kChunk neighbouring lines of one view
// (consecutive detector bins, or consecutive lines of a sorted free list).
// Such lines are nearly parallel and adjacent,
// so in every major-axis row their runs of nonzero nodes fall inside a short
// window; the CTA keeps those windows (a skewed strip, one row per major-axis
// row) in shared memory: staged from the coefficients for the forward
// projection, accumulated and then added to the output for the adjoint.
// Lines whose major axis is x1 use transposed images so that strip rows stay
// contiguous in global memory.
//
// One warp takes one line at a time, in batches of up to kBatch rows:
//   A. lane per row: u_0 (stepped from row to row in 64-bit fixed point),
//      its interval sigma, t = u_0 - s_sigma and the strip offset of the
//      row's first candidate; the rows are then ordered by sigma (counting
//      sort, in the warp's shared memory);
//   B. lane per (candidate i, row slot): for each interval sigma the lane
//      holds the polynomial T[sigma][i] in registers and runs it over the
//      rows of that interval, two rows per packed FP32 FMA (fma.rn.f32x2).
// Polynomial coefficients are then read once per interval and batch instead
// of once per row, which keeps shared-memory traffic to the row records and
// the coefficients (or strip accumulators) themselves.
//
// The adjoint accumulates its strip in 32-bit fixed point: a shared-memory
// integer reduction costs about what a plain shared store does on this GPU,
// a float one four to six times more.  Each chunk takes the power of two S
// that puts its largest contribution h |p| phi (phi <= sqrt(2) < 1.5 for
// every basis here) at 2^21 or less; a pair then adds round(S h p phi) to its
// node, at most 2^26 in magnitude after 32 lines, and the flush adds the
// sums times 1/S (exact) to the image.  The rounding rides on the last FMA
// of the Horner scheme: its constant term carries M = 1.5 2^23, so the
// result lies in [2^23, 2^24) where floats are the integers, and its bits
// minus M's bits are round(S h p phi).  Per pair that is an error of at most
// one unit, 1/S <= 1.5 h max|p| 2^-21 = 7e-7 h max|p|.
#include <climits>

#include "common.cuh"

namespace spx {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kChunk = 32;          // lines per chunk
constexpr int kPitch = 44;          // strip row length (floats), whole 16-byte chunks
constexpr int kWin = kPitch - 3;    // window width that fits once its start is rounded down to 4 columns
constexpr int kSlabRows = 360;      // strip rows held at once (one sorting batch per line and slab)
constexpr int kDummy = 16;          // zero floats after the strip: target of padding records
constexpr int kBatch = 384;         // rows of one line per sorting batch (12 per lane), >= kSlabRows
constexpr int kRowsPerLane = kBatch / 32;
constexpr int kEntCap = kBatch + 4 * kMaxSig;   // sorted row records, segments padded to multiples of 4

constexpr size_t kStripBytes = sizeof(float) * (kSlabRows * kPitch + kDummy);
constexpr size_t kCloBytes = sizeof(int) * kSlabRows;
// Per warp: two table buffers (current line and the next one, loaded
// asynchronously) and the sorted row records of one batch.
constexpr size_t kTabBufBytes = sizeof(float) * kTabFloats;
constexpr size_t kWarpBytes = 2 * kTabBufBytes + 2 * sizeof(float) * kEntCap;   // + t[] and offset[]
constexpr size_t kAccBytes = sizeof(float) * kChunk;
constexpr size_t kMiscBytes = 32 + 4 * 64;
constexpr size_t kHdrBytes = sizeof(LineHdr) * kChunk;
constexpr size_t kRecOffBytes = sizeof(int) * kChunk;
constexpr size_t kSmemBytes =
    kStripBytes + kCloBytes + kWarps * kWarpBytes + kAccBytes + kMiscBytes + kHdrBytes + kRecOffBytes;
static_assert(kTabBufBytes % 16 == 0 && kWarpBytes % 16 == 0 && kStripBytes % 16 == 0 && kCloBytes % 16 == 0,
              "16-byte alignment of the shared-memory regions");
static_assert(kSmemBytes <= 115712, "two CTAs per SM");
static_assert(kPitch % 4 == 0, "strip rows of whole 16-byte chunks");
static_assert(kSlabRows * kPitch + kDummy < (1 << 16), "strip offsets fit 16 bits (phase A packs sigma above them)");
static_assert(kBatch >= kSlabRows && kEntCap < 512, "one batch per line and slab; 9-bit counters of the sort");

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

// No "memory" clobber: the strip is read only after the block's barrier
// before its flush, so the reductions need not order the row-record and table
// loads of the next groups, which the compiler may then issue early.
__device__ __forceinline__ void red_shared_u32(int *p, int v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v));
}

// Fixed-point rounding constant M = 1.5 * 2^23 (see the top of the file).
constexpr float kFixMagic = 12582912.0f;
constexpr int kFixMagicBits = 0x4B400000;
// Largest contribution of a chunk after scaling, and the bound on phi used
// to choose the scale.
constexpr float kFixMax = 2097152.0f;   // 2^21
constexpr float kPhiBound = 1.5f;

// Row records kept by a plan (see spline_plan_prepare): kRecWrite runs the
// traversal (line groups, strip slabs, row batches, phase A and the sort) and
// stores each batch's sorted records instead of projecting; kRecRead loads
// them in the same order and runs phase B only.  Per line a region of
// strip_rec_line_bytes(); per batch a 16-byte header (padded segment lengths,
// and a flag for batches with runs outside the staged window, which the
// replay recomputes), then t[R] and the strip offsets[R].
enum RecMode { kRecNone = 0, kRecWrite = 1, kRecRead = 2 };
// Which chunks an adjoint call runs (strip_chunk's FM).
enum FixMode { kFmAll = 0, kFmFixed = 1, kFmFloat = 2 };
constexpr unsigned long long kRecSlowBit = 1ull << 63;

template <int NS>
__device__ __forceinline__ int4 rec_pack(const int (&segn)[NS], bool slow)
{
    int n[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < NS; ++q) n[q] = segn[q];
    return make_int4(n[0] | (n[1] << 16), n[2] | (n[3] << 16), n[4], slow ? (1 << 16) : 0);
}

template <int NS>
__device__ __forceinline__ int rec_unpack(int4 hd, int (&segb)[NS], int (&segn)[NS])
{
    const int n[5] = {hd.x & 0xffff, hd.x >> 16, hd.y & 0xffff, hd.y >> 16, hd.z & 0xffff};
    int b = 0;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        segb[q] = b;
        segn[q] = n[q];
        b += n[q];
    }
    return b;
}

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

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

// Copy the first n16 16-byte chunks of a footprint table (all kTabFloats / 4
// of them, or its head alone) to shared memory.
__device__ __forceinline__ void table_copy_async(float *dst, const float *src, int lane, int n16 = kTabFloats / 4)
{
    for (int i = lane; i < n16; i += 32) cp_async16(dst + 4 * i, src + 4 * i);
}

// floor(a / b) for b > 0.
__device__ __forceinline__ long long floor_div(long long a, long long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Prefetch `bytes` from p towards L2 (one 128-byte line per lane and pass).
__device__ __forceinline__ void prefetch_span_l2(const unsigned char *p, int bytes, int lane)
{
    for (int o = lane * 128; o < bytes; o += 32 * 128) prefetch_l2(p + o);
}

// Phase B helpers of strip_line.  load_poly: the packed coefficients of
// T[q][ci] (times hp for the adjoint; degree 0 with candidate ci's argument
// shift ci (|kappa| - a) folded into the constant term).
template <int DEG, bool ADJ, bool FIX = false>
__device__ __forceinline__ void load_poly(const float *tabw, int q, int ci, float hp, float a_corr,
                                          f2 (&C)[2 * DEG + 2])
{
    constexpr int NC = 2 * DEG + 2;
    // T[sigma][ci]: 32-byte aligned (table buffers and entries are)
    const float4 *Tq4 = reinterpret_cast<const float4 *>(tabw + tab_poly(q, ci));
    float cq[NC];
#pragma unroll
    for (int d4 = 0; d4 < (NC + 3) / 4; ++d4) {
        const float4 w = Tq4[d4];
        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (4 * d4 + u < NC) cq[4 * d4 + u] = wv[u];
    }
    if constexpr (DEG == 0) cq[0] = __fmaf_rn(cq[1], (float)ci * a_corr, cq[0]);
#pragma unroll
    for (int d = 0; d < NC; ++d) {
        float c = ADJ ? cq[d] * hp : cq[d];
        if (FIX && d == 0) c += kFixMagic;   // hp carries the chunk's scale S
        C[d] = f2pack(c, c);
    }
}

// run_group: the 4 sorted row records at e (one interval), two rows per packed
// Horner chain; forward: acc2 += c phi from the strip; adjoint: reductions of
// phi into the strip.
template <int DEG, bool ADJ, bool FIX = false>
__device__ __forceinline__ void run_group(const f2 (&C)[2 * DEG + 2], const float *ent_t, const int *ent_p, int e,
                                          float *strip, int coloff, f2 &acc2)
{
    constexpr int NC = 2 * DEG + 2;
    const ulonglong2 tt = *reinterpret_cast<const ulonglong2 *>(ent_t + e);
    const int4 P = *reinterpret_cast<const int4 *>(ent_p + e);
    f2 pa = C[NC - 1], pb = C[NC - 1];
#pragma unroll
    for (int d = NC - 2; d >= 0; --d) {
        pa = f2fma(pa, tt.x, C[d]);
        pb = f2fma(pb, tt.y, C[d]);
    }
    if constexpr (ADJ && FIX) {
        float f0, f1, f2_, f3;
        f2unpack(pa, f0, f1);
        f2unpack(pb, f2_, f3);
        int *istrip = reinterpret_cast<int *>(strip);
        red_shared_u32(istrip + P.x + coloff, __float_as_int(f0) - kFixMagicBits);
        red_shared_u32(istrip + P.y + coloff, __float_as_int(f1) - kFixMagicBits);
        red_shared_u32(istrip + P.z + coloff, __float_as_int(f2_) - kFixMagicBits);
        red_shared_u32(istrip + P.w + coloff, __float_as_int(f3) - kFixMagicBits);
    } else if constexpr (ADJ) {
        float f0, f1, f2_, f3;
        f2unpack(pa, f0, f1);
        f2unpack(pb, f2_, f3);
        red_shared(strip + P.x + coloff, f0);
        red_shared(strip + P.y + coloff, f1);
        red_shared(strip + P.z + coloff, f2_);
        red_shared(strip + P.w + coloff, f3);
    } else {
        acc2 = f2fma(f2pack(strip[P.x + coloff], strip[P.y + coloff]), pa, acc2);
        acc2 = f2fma(f2pack(strip[P.z + coloff], strip[P.w + coloff]), pb, acc2);
    }
}

// Degree 0 exactly along an axis (kDeg0Axis): the footprint is a rectangle
// whose edges fall on nodes, each taking the midpoint value on both sides, so
// a row has one more candidate.  Such lines run lane per row straight from or
// to global memory (as the general kernels do); they occur only at views
// exactly along an axis.
__device__ float strip_tie_line(const LineHdr &H, const float *tabw, int S0, int S1, int lane,
                                const float *__restrict__ src, float *dst, int Nq, float hp, bool adj)
{
    const int sgn = (H.flags & kKapNeg) ? -1 : 1;
    const float inv_a = 1.0f / H.a;
    float s0[1] = {tabw[0]};
    float acc = 0.f;
    const int rb = max(H.r_begin, S0), re = min(H.r_end, S1);
    for (int r = rb + lane; r < re; r += 32) {
        const RowEval e = row_eval<0>(H, s0, inv_a, sgn, r);
        for (int i = -1; i < H.K; ++i) {
            const int q = e.q0 + sgn * i;
            if ((unsigned)q >= (unsigned)Nq) continue;
            float phi;
            if (i < 0) {
                if (!e.tie) continue;
                phi = 0.5f * inv_a;   // the run also starts at u = 0
            } else {
                phi = horner<0>(tabw + tab_poly(e.sg, i), __fmaf_rn((float)i, H.a_corr, e.t));
                if (e.tie) phi = 0.5f * phi;
            }
            if (adj) atomicAdd(dst + (size_t)r * Nq + q, hp * phi);
            else acc = __fmaf_rn(__ldg(src + (size_t)r * Nq + q), phi, acc);
        }
    }
    return acc;
}

// One line over the strip rows [S0, S1).  Forward (ADJ false): returns this
// lane's part of sum_k c_k phi (no factor h).  Adjoint: adds hp * phi into the
// strip.  tabw is the line's table in shared memory; ent_t / ent_p hold the
// warp's sorted row records (t, strip offset of candidate 0).  FIX: the
// adjoint's fixed-point strip (hpS = hp S); RM: the row-record mode.
// A row whose run fell outside the staged window: its candidates straight
// from (forward; returns the partial sum) or to (adjoint) global memory, and
// counted.  Kept out of line: it runs only on geometries the windows do not
// anticipate, and inlined into every unrolled row of phase A it only
// lengthened the kernel.
template <int DEG, bool ADJ>
__device__ __noinline__ float strip_slow_row(const float *tabw, int sg, float t, int q0, int sgn, int K, float a_corr,
                                             int r, int Nq, const float *__restrict__ src, float *dst, float hp,
                                             int *err)
{
    atomicAdd(err, 1);
    const float *T0 = tabw + tab_poly(sg, 0);
    float acc = 0.f;
    for (int i = 0; i < K; ++i) {
        const int q = q0 + sgn * i;
        if ((unsigned)q < (unsigned)Nq) {
            const float ti = (DEG == 0) ? __fmaf_rn((float)i, a_corr, t) : t;
            const float phi = horner<DEG>(T0 + i * kNC, ti);
            if constexpr (ADJ) atomicAdd(dst + (size_t)r * Nq + q, hp * phi);
            else acc = __fmaf_rn(__ldg(src + (size_t)r * Nq + q), phi, acc);
        }
    }
    return acc;
}

template <int DEG, bool ADJ, bool FIX = false, int RM = kRecNone>
__device__ float strip_line(const LineHdr &H, const float *tabw, float *ent_t, int *ent_p, float *strip, const int *clo,
                            int S0, int S1, int lane, const float *__restrict__ src, float *dst, int Nq,
                            int *err, float hp, float hpS, unsigned char *&rp, const unsigned char *rend)
{
    constexpr int rmode = RM;
    constexpr int NC = 2 * DEG + 2;
    constexpr int NS = DEG + 2;       // intervals sigma
    if constexpr (DEG == 0)
        if (H.flags & kDeg0Axis) return strip_tie_line(H, tabw, S0, S1, lane, src, dst, Nq, hp, ADJ);
    const int sgn = (H.flags & kKapNeg) ? -1 : 1;
    const float inv_a = 1.0f / H.a;
    float s[DEG + 1];
#pragma unroll
    for (int q = 0; q <= DEG; ++q) s[q] = tabw[q];
    const int K = H.K;
    // phase B lane roles: candidate ci of row slot sl (nsl slots of K lanes)
    const int rk = (int)ceilf(256.0f * __frcp_rn((float)K));   // ceil(256 / K): (l * rk) >> 8 == l / K for l < 32, K <= 8
    const int nsl = (32 * rk) >> 8;
    const int sl = (lane * rk) >> 8;
    const int ci = lane - sl * K;
    const bool lane_on = sl < nsl;
    const int coloff = sgn * ci;
    f2 acc2 = 0ull;
    float acc_slow = 0.f;
    // a run fits the strip row iff its first column oq satisfies
    // oq_lo <= oq <= oq_lo + kPitch - K (the run spans oq .. oq + sgn (K - 1))
    const int oq_lo = sgn > 0 ? 0 : K - 1;
    const unsigned oq_span = (unsigned)(kPitch - K);
    // Row stepping in fixed point (degree >= 1): W(r) = 2^32 u(r)/a - 1 as a
    // 64-bit integer, u(r) = U0 + (r - r_ref) rho the offset of row r at
    // column q_ref.  Its high word is the row's step count k (u_0 = u - k a
    // in (0, a]) and u_0 = (low word + 1) a 2^-32.  rho/a and U0/a enter as
    // float pairs (one correction step of the float quotient), rounded to 32
    // fractional bits: over 2^11 rows that is within 2^-21 a of the exact u_0.
    long long Wstep = 0, Wbase = 0;
    float ua = 0.f;
    if constexpr (DEG >= 1) {
        auto fix_quot = [&](float xh, float xl) {
            const float q1 = xh * inv_a;
            const float r = __fmaf_rn(-q1, H.a_lo, __fmaf_rn(-q1, H.a_hi, xh) + xl);
            const float q2 = r * inv_a;
            return __float2ll_rn(q1 * 4294967296.f) + __float2ll_rn(q2 * 4294967296.f);
        };
        Wstep = fix_quot(H.rho_hi, H.rho_lo);
        Wbase = fix_quot(H.U0, H.U0_lo) - 1 - (long long)H.r_ref * Wstep;
        ua = H.a * 2.3283064365386963e-10f;   // a 2^-32
    }

    const int dummy_pos = kSlabRows * kPitch + kDummy / 2;
    const int rb = max(H.r_begin, S0), re = min(H.r_end, S1);
    for (int r0 = rb; r0 < re; r0 += kBatch) {
        int segb[NS], segn[NS];   // segment start and padded length (a multiple of 4)
        bool ready = false;
        if (rmode == kRecRead && rp + 16 <= rend) {
            // the batch as the record pass left it: header, then its t and offsets
            const int4 hd = __ldg(reinterpret_cast<const int4 *>(rp));
            const int R = rec_unpack(hd, segb, segn);
            const bool slow = (hd.w >> 16) != 0;
            if (!slow) {
                const float4 *gt = reinterpret_cast<const float4 *>(rp + 16);
                const int4 *gp = reinterpret_cast<const int4 *>(rp + 16 + 4 * R);
                for (int i = lane; i < R / 4; i += 32) {
                    reinterpret_cast<float4 *>(ent_t)[i] = __ldg(gt + i);
                    reinterpret_cast<int4 *>(ent_p)[i] = __ldg(gp + i);
                }
                __syncwarp();
                ready = true;
            }
            rp += 16 + 8 * (slow ? 0 : R);   // a flagged batch was stored without records
        }
        if (!ready) {
        // ---- A: lane per row
        float tv[kRowsPerLane];
        int pv[kRowsPerLane];
        unsigned long long own = 0ull;
        long long W = Wbase + (long long)(r0 + lane) * Wstep;   // W of this lane's first row
#pragma unroll
        for (int j = 0; j < kRowsPerLane; ++j) {
            const int r = r0 + j * 32 + lane;
            const long long Wr = W;
            W += 32 * Wstep;
            tv[j] = 0.f;
            pv[j] = -1;
            if (r < re) {
                RowEval e;
                if constexpr (DEG == 0) {
                    e = row_eval<0>(H, s, inv_a, sgn, r);
                } else {
                    const int k = (int)(Wr >> 32);
                    const float u0 = __fmaf_rn((float)(unsigned)Wr, ua, ua);
                    float s_lo;
                    e.sg = sigma_of<DEG>(s, u0, s_lo);
                    e.t = u0 - s_lo;
                    e.q0 = H.q_ref - sgn * k;
                }
                const int rr = r - S0;
                const int oq = e.q0 - clo[rr];
                if ((unsigned)(oq - oq_lo) <= oq_span) {
                    tv[j] = e.t;
                    pv[j] = (rr * kPitch + oq) | (e.sg << 16);
                    own += 1ull << (9 * e.sg);
                } else if (rmode == kRecWrite) {
                    // the replay recomputes this batch (and reaches global memory then)
                    own |= kRecSlowBit;
                } else {
                    // run outside the staged window: straight from or to global memory
                    acc_slow += strip_slow_row<DEG, ADJ>(tabw, e.sg, e.t, e.q0, sgn, K, H.a_corr, r, Nq, src, dst,
                                                         hp, err);
                }
            }
        }
        // counting sort by sigma: 9-bit counters per interval, packed
        const bool slow_batch = rmode == kRecWrite && __any_sync(0xffffffffu, (own & kRecSlowBit) != 0ull);
        own &= ~kRecSlowBit;
        unsigned long long inc = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const unsigned long long tot = __shfl_sync(0xffffffffu, inc, 31);
        unsigned long long basep = 0ull;
        {
            int b = 0;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int c = (int)((tot >> (9 * q)) & 511ull);
                const int cp = (c + 3) & ~3;
                segb[q] = b;
                segn[q] = cp;
                basep |= (unsigned long long)b << (9 * q);
                // padding records (t = 0, zero target) complete the segment
                if (lane < cp - c) { ent_t[b + c + lane] = 0.f; ent_p[b + c + lane] = dummy_pos; }
                b += cp;
            }
        }
        unsigned long long cur = basep + (inc - own);
#pragma unroll
        for (int j = 0; j < kRowsPerLane; ++j) {
            if (pv[j] >= 0) {
                const int sh = 9 * (pv[j] >> 16);
                const int idx = (int)((cur >> sh) & 511ull);
                cur += 1ull << sh;
                ent_t[idx] = tv[j];
                ent_p[idx] = pv[j] & 0xffff;
            }
        }
        __syncwarp();
        if (rmode == kRecWrite) {
            // store the batch for the replays: header, t[R], offsets[R] (a
            // batch that would not fit the line's region is stored flagged,
            // without records; past its end nothing is stored, and the
            // replay, reading the same positions, recomputes those batches)
            if (rp + 16 > rend) continue;
            int R = 0;
#pragma unroll
            for (int q = 0; q < NS; ++q) R += segn[q];
            const bool flag = slow_batch || rp + 16 + 8 * R > rend;
            if (flag) R = 0;
            if (lane == 0) *reinterpret_cast<int4 *>(rp) = rec_pack(segn, flag);
            float4 *gt = reinterpret_cast<float4 *>(rp + 16);
            int4 *gp = reinterpret_cast<int4 *>(rp + 16 + 4 * R);
            for (int i = lane; i < R / 4; i += 32) {
                gt[i] = reinterpret_cast<const float4 *>(ent_t)[i];
                gp[i] = reinterpret_cast<const int4 *>(ent_p)[i];
            }
            rp += 16 + 8 * R;
            __syncwarp();
            continue;
        }
        }   // !ready
        // ---- B: lane per (candidate, row slot), four rows per step
        if (lane_on) {
            f2 C[NC];
            // one interval at a time (an interval's last step may leave some
            // row slots idle; walking the concatenated intervals instead costs
            // a segment test per step and was slower in both directions once
            // the adjoint's reductions became integer ones)
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int n = segn[q];
                if (n == 0) continue;
                load_poly<DEG, ADJ, FIX>(tabw, q, ci, FIX ? hpS : hp, H.a_corr, C);
                const int end = segb[q] + n;
                for (int e = segb[q] + 4 * sl; e < end; e += 4 * nsl)
                    run_group<DEG, ADJ, FIX>(C, ent_t, ent_p, e, strip, coloff, acc2);
            }
        }
        __syncwarp();
    }
    if constexpr (ADJ) {
        return 0.f;
    } else {
        float a0, a1;
        f2unpack(acc2, a0, a1);
        return (a0 + a1) + acc_slow;
    }
}

// Forward (ADJ false): sino[line] = h sum c phi.  Adjoint (ADJ true): adds
// h sino[line] phi to out (vertical lines) or outT (horizontal lines, the
// transposed image).
// One chunk (view v, bins j0..j0+31) of one instance; smem is the CTA's
// dynamic shared memory (kSmemBytes).
// FM (adjoint only) picks the chunks a call runs: kFmFixed only those that
// accumulate in fixed point, kFmFloat only the others (non-finite values, or
// a scale outside the safe range; see the top of the file), with float
// strips.  A launch of each covers every chunk, and the fixed-point kernel
// carries no second copy of the line code (a second inlined copy, or a call
// anywhere in the kernel, made the fixed-point adjoint about a tenth
// slower).  The forward takes kFmAll.
template <int DEG, bool ADJ, int RM = kRecNone, int FM = kFmAll>
__device__ __forceinline__ bool strip_chunk(unsigned char *smem, const GridDev g, const LinesDev L,
                                            const LineHdr *__restrict__ hdr, const float *__restrict__ tabs,
                                            const float *__restrict__ coef, const float *__restrict__ coefT,
                                            float *__restrict__ sino, float *__restrict__ out,
                                            float *__restrict__ outT, int chunks_per_view, int vec, int *err,
                                            int chunk, unsigned char *rec = nullptr, long long rec_cap = 0)
{
    constexpr int rmode = RM;
    float *strip = reinterpret_cast<float *>(smem);
    size_t o = kStripBytes;
    int *clo = reinterpret_cast<int *>(smem + o);
    o += kCloBytes;
    unsigned char *warp_area = smem + o;
    o += kWarps * kWarpBytes;
    float *line_acc = reinterpret_cast<float *>(smem + o);
    o += kAccBytes;
    int *misc = reinterpret_cast<int *>(smem + o);
    o += kMiscBytes;
    int *gstack = misc + 8;   // pending line groups, (first | last << 8)
    LineHdr *hdr_s = reinterpret_cast<LineHdr *>(smem + o);
    o += kHdrBytes;
    int *rec_off = reinterpret_cast<int *>(smem + o);   // per line: bytes of its records used so far

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *tabbuf = reinterpret_cast<float *>(warp_area + warp * kWarpBytes);   // [2][kTabFloats]
    float *ent_t = reinterpret_cast<float *>(warp_area + warp * kWarpBytes + 2 * kTabBufBytes);
    int *ent_p = reinterpret_cast<int *>(ent_t + kEntCap);
    const int v = chunk / chunks_per_view, cb = chunk - v * chunks_per_view;
    const int j0 = cb * kChunk;
    const int64_t nd = chunk_bins(L);
    const int nl = (int)min((int64_t)kChunk, nd - j0);
    // position of the chunk's first line (in the sorted order for free lists;
    // records are kept by position), and lane l's line index in every warp
    const int64_t line0 = (int64_t)v * nd + j0;
    const int my_line = lane < nl ? (L.order ? __ldg(L.order + line0 + lane) : (int)(line0 + lane)) : 0;

    if constexpr (ADJ) {
        // The chunk's fixed-point scale S (a power of two; see the top of the
        // file): misc[5] = 1 if the strip accumulates in fixed point, misc[6]
        // and misc[7] the bits of S and 1/S.  Non-finite values, or values so
        // large or small that S leaves a safe exponent range, keep the float
        // reductions.
        if (warp == 0) {
            const float pv = lane < nl ? sino[my_line] : 0.f;
            const bool bad = !isfinite(pv);
            float pm = fabsf(pv);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pm = fmaxf(pm, __shfl_xor_sync(0xffffffffu, pm, o));
            const float top = kPhiBound * g.h * pm;   // largest |h p phi| of the chunk
            // (an all-zero chunk counts as fixed point: its lines are skipped)
            const bool fix = !__any_sync(0xffffffffu, bad) && (top == 0.f || (top >= 1e-20f && top <= 1e20f));
            if (lane == 0) {
                int e = 0;
                if (fix && top > 0.f) {
                    frexpf(kFixMax / top, &e);   // kFixMax / top in [2^(e-1), 2^e)
                    e -= 1;                      // S = 2^e <= kFixMax / top
                }
                misc[5] = fix ? 1 : 0;
                misc[6] = __float_as_int(ldexpf(1.f, e));
                misc[7] = __float_as_int(ldexpf(1.f, -e));
            }
        }
        __syncthreads();
        const bool fx = misc[5] != 0;
        static_assert(!ADJ || FM != kFmAll, "the adjoint runs as fixed-point and float launches");
        if constexpr (FM == kFmFixed) {
            if (!fx) return false;   // left to the float launch
        } else if constexpr (FM == kFmFloat) {
            if (fx) return false;    // done by the fixed-point launch
        }
    }

    if (!ADJ && threadIdx.x < kChunk) line_acc[threadIdx.x] = 0.f;
    if (threadIdx.x < kChunk) rec_off[threadIdx.x] = 0;
    if (!ADJ && threadIdx.x < kDummy) strip[kSlabRows * kPitch + threadIdx.x] = 0.f;
    // the chunk's line records into shared memory, its tables towards L2
    // (lines other than parallel beams have one table each, indexed by line)
    static_assert(kChunk * 4 <= kThreads, "one pass over the chunk's line records");
    {
        const int src = __shfl_sync(0xffffffffu, my_line, (threadIdx.x >> 2) & 31);
        if ((int)threadIdx.x < nl * 4)
            reinterpret_cast<int4 *>(hdr_s)[threadIdx.x] =
                __ldg(reinterpret_cast<const int4 *>(hdr + src) + (threadIdx.x & 3));
    }
    if (L.kind != SP_LINES_PARALLEL)
        for (int i0 = 0; i0 < kChunk * kTabLines; i0 += kThreads) {
            const int i = i0 + threadIdx.x;
            const int src = __shfl_sync(0xffffffffu, my_line, min(i / kTabLines, kChunk - 1));
            if (i < nl * kTabLines) prefetch_l2(tabs + (int64_t)src * kTabFloats + (i % kTabLines) * 32);
        }
    bool fixed = false;
    float fscale = 1.f, finv = 1.f;
    for (int axis = 0; axis < 2; ++axis) {
        __syncthreads();
        if (ADJ && axis == 0) {
            fixed = FM != kFmFloat && misc[5] != 0;
            fscale = __int_as_float(misc[6]);
            finv = __int_as_float(misc[7]);
        }
        if (warp == 0) {
            bool mine = false;
            if (lane < nl) {
                const LineHdr &H = hdr_s[lane];
                mine = !(H.flags & kEmpty) && (((H.flags & kVert) != 0) == (axis == 0)) && H.r_end > H.r_begin;
                // (with kept records the groups must be those of the record pass,
                // so lines with p = 0 stay in them and are skipped below)
                if (ADJ && mine && rmode == kRecNone) mine = sino[my_line] != 0.f;
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
            // free lists: the extreme run columns over all lines of the group
            // at the first and the last row (la..ha, lb..hb); between them the
            // window follows the chords, which bound the runs: each run moves
            // linearly with the row, so the lowest start is concave in the row
            // and the highest end convex
            int la = 0, ha = 0, lb = 0, hb = 0;
            if (L.order) {
                la = lb = INT_MAX;
                ha = hb = INT_MIN;
                if ((gmask >> lane) & 1u) {
                    const LineHdr &Hx = hdr_s[lane];
                    const float ia = 1.0f / Hx.a;
                    run_columns(Hx, ia, R0, la, ha);
                    run_columns(Hx, ia, R1 - 1, lb, hb);
                }
#pragma unroll
                for (int o2 = 16; o2 > 0; o2 >>= 1) {
                    la = min(la, __shfl_xor_sync(0xffffffffu, la, o2));
                    ha = max(ha, __shfl_xor_sync(0xffffffffu, ha, o2));
                    lb = min(lb, __shfl_xor_sync(0xffffffffu, lb, o2));
                    hb = max(hb, __shfl_xor_sync(0xffffffffu, hb, o2));
                }
                wmax = max(ha - la, hb - lb) + 7;
            } else {
                int lo1, hi1, lo2, hi2;
                run_columns(Hf, inv_af, R0, lo1, hi1);
                run_columns(Hl, inv_al, R0, lo2, hi2);
                wmax = max(hi1, hi2) - min(lo1, lo2) + 5;
                run_columns(Hf, inv_af, R1 - 1, lo1, hi1);
                run_columns(Hl, inv_al, R1 - 1, lo2, hi2);
                wmax = max(wmax, max(hi1, hi2) - min(lo1, lo2) + 5);
            }
            __syncthreads();
            if (wmax > kWin && first < last) {
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
                    int lo, hi;
                    if (L.order) {
                        // the chords, rounded outwards, margin 3 (a run lies
                        // within one column of its line)
                        const long long span = max(R1 - 1 - R0, 1), dr = S0 + rr - R0;
                        lo = la + (int)floor_div((long long)(lb - la) * dr, span) - 3;
                        hi = ha - (int)floor_div(-(long long)(hb - ha) * dr, span) + 3;
                    } else {
                        int lo1, hi1, lo2, hi2;
                        run_columns(Hf, inv_af, S0 + rr, lo1, hi1);
                        run_columns(Hl, inv_al, S0 + rr, lo2, hi2);
                        lo = min(lo1, lo2) - 2;
                        hi = max(hi1, hi2) + 2;
                    }
                    // centred in the usable width, start rounded down to a 16-byte chunk
                    clo[rr] = (lo - max(0, (kWin - (hi - lo + 1)) / 2)) & ~3;
                }
                __syncthreads();
                constexpr int kCh = kPitch / 4;   // 16-byte chunks per strip row
                if (rmode == kRecWrite) {
                    // the record pass projects nothing: no strip
                } else if constexpr (ADJ) {
                    float4 *s4 = reinterpret_cast<float4 *>(strip);
                    for (int i = threadIdx.x; i < nrows * kCh; i += kThreads) s4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                } else if (vec) {
                    // asynchronous 16-byte copies; chunks are wholly inside or
                    // outside the grid (Nq and chunk starts are multiples of 4)
                    for (int i = threadIdx.x; i < nrows * kCh; i += kThreads) {
                        const int rr = i / kCh, cc = i - rr * kCh;
                        const int q = clo[rr] + 4 * cc;
                        const bool in = (unsigned)q < (unsigned)Nq;
                        const float *gp = in ? src + (size_t)(S0 + rr) * Nq + q : src;
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                                         (unsigned)__cvta_generic_to_shared(strip + 4 * i)),
                                     "l"(gp), "r"(in ? 16 : 0)
                                     : "memory");
                    }
                    asm volatile("cp.async.wait_all;" ::: "memory");
                } else {
                    // 4-byte copies, zero-filled outside the grid
                    for (int i = threadIdx.x; i < nrows * kPitch; i += kThreads) {
                        const int rr = i / kPitch, cc = i - rr * kPitch;
                        const int q = clo[rr] + cc;
                        const bool in = (unsigned)q < (unsigned)Nq;
                        const float *gp = in ? src + (size_t)(S0 + rr) * Nq + q : src;
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                                         (unsigned)__cvta_generic_to_shared(strip + i)),
                                     "l"(gp), "r"(in ? 4 : 0)
                                     : "memory");
                    }
                    asm volatile("cp.async.wait_all;" ::: "memory");
                }
                __syncthreads();
                // this warp's lines of the group: li = first + warp + k kWarps in
                // wmask (gmask less, in the adjoint with kept records, lines with
                // p = 0); the table of the next one is loaded while the current
                // one runs.  The record pass needs only each table's head (the
                // interval ends s_q); replays prefetch a line's records one line
                // ahead.
                unsigned wmask = gmask;
                if (ADJ && rmode == kRecRead) {
                    const bool nz = lane < nl && sino[my_line] != 0.f;
                    wmask &= __ballot_sync(0xffffffffu, nz);
                }
                int li = first + warp;
                while (li <= last && !((wmask >> li) & 1u)) li += kWarps;
                int buf = 0;
                const int tab16 = rmode == kRecWrite ? kTabHead / 4 : kTabFloats / 4;
                constexpr int kRecAhead = 4096;
                if (li <= last) {
                    table_copy_async(tabbuf, tabs + (int64_t)hdr_s[li].tab * kTabFloats, lane, tab16);
                    cp_async_commit();
                    if (rmode == kRecRead)
                        prefetch_span_l2(rec + (line0 + li) * rec_cap + rec_off[li],
                                         (int)min((long long)kRecAhead, rec_cap - rec_off[li]), lane);
                }
                while (li <= last) {
                    int ln = li + kWarps;
                    while (ln <= last && !((wmask >> ln) & 1u)) ln += kWarps;
                    if (ln <= last) {
                        table_copy_async(tabbuf + (buf ^ 1) * kTabFloats,
                                         tabs + (int64_t)hdr_s[ln].tab * kTabFloats, lane, tab16);
                        if (rmode == kRecRead)
                            prefetch_span_l2(rec + (line0 + ln) * rec_cap + rec_off[ln],
                                             (int)min((long long)kRecAhead, rec_cap - rec_off[ln]), lane);
                    }
                    cp_async_commit();
                    cp_async_wait<1>();
                    __syncwarp();
                    const LineHdr H = hdr_s[li];
                    const float hp = ADJ ? g.h * sino[__shfl_sync(0xffffffffu, my_line, li)] : 0.f;
                    unsigned char *lrec = rec ? rec + (line0 + li) * rec_cap : nullptr;
                    unsigned char *rp = lrec ? lrec + rec_off[li] : nullptr;
                    const unsigned char *rend = lrec ? lrec + rec_cap : nullptr;
                    float part;
                    if constexpr (ADJ) {
                        part = strip_line<DEG, true, FM != kFmFloat, RM>(H, tabbuf + buf * kTabFloats, ent_t, ent_p,
                                                                         strip, clo, S0, S1, lane, src, dst, Nq, err,
                                                                         hp, FM != kFmFloat ? hp * fscale : 0.f, rp,
                                                                         rend);
                    } else {
                        part = strip_line<DEG, false, false, RM>(H, tabbuf + buf * kTabFloats, ent_t, ent_p, strip,
                                                                 clo, S0, S1, lane, src, dst, Nq, err, hp, 0.f, rp,
                                                                 rend);
                    }
                    if (!ADJ && rmode != kRecWrite) {
                        const float sum = warp_sum(part);
                        if (lane == 0) line_acc[li] += sum;
                    }
                    if (lrec && lane == 0) rec_off[li] = (int)(rp - lrec);
                    __syncwarp();
                    li = ln;
                    buf ^= 1;
                }
                cp_async_wait<0>();
                if (ADJ && rmode != kRecWrite) {
                    __syncthreads();
                    // add the accumulated strip into the image
                    if (vec) {
                        const float4 *s4 = reinterpret_cast<const float4 *>(strip);
                        const int4 *i4 = reinterpret_cast<const int4 *>(strip);
                        for (int i = threadIdx.x; i < nrows * kCh; i += kThreads) {
                            const int rr = i / kCh, cc = i - rr * kCh;
                            const int q = clo[rr] + 4 * cc;
                            float4 v4;
                            if (fixed) {
                                const int4 n4 = i4[i];
                                v4 = make_float4((float)n4.x * finv, (float)n4.y * finv, (float)n4.z * finv,
                                                 (float)n4.w * finv);
                            } else {
                                v4 = s4[i];
                            }
                            if ((unsigned)q < (unsigned)Nq &&
                                (v4.x != 0.f || v4.y != 0.f || v4.z != 0.f || v4.w != 0.f))
                                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(
                                                 dst + (size_t)(S0 + rr) * Nq + q),
                                             "f"(v4.x), "f"(v4.y), "f"(v4.z), "f"(v4.w)
                                             : "memory");
                        }
                    } else {
                        for (int i = threadIdx.x; i < nrows * kPitch; i += kThreads) {
                            const int rr = i / kPitch, cc = i - rr * kPitch;
                            const int q = clo[rr] + cc;
                            const float val = fixed ? (float)reinterpret_cast<const int *>(strip)[i] * finv : strip[i];
                            if ((unsigned)q < (unsigned)Nq && val != 0.f)
                                atomicAdd(dst + (size_t)(S0 + rr) * Nq + q, val);
                        }
                    }
                }
            }
        }
    }
    if (!ADJ && rmode != kRecWrite) {
        __syncthreads();
        if ((int)threadIdx.x < nl) sino[my_line] = g.h * line_acc[threadIdx.x];   // warp 0: lane = line
    }
    return true;
}

// One CTA per chunk.  The adjoint runs the fixed-point chunks (FM kFmFixed:
// nearly all) and appends the others to defer[2..] (count defer[0]) for
// strip_float_kernel.
template <int DEG, bool ADJ, int RM, int FM = kFmAll>
__global__ void __launch_bounds__(kThreads, 2)
strip_kernel(GridDev g, LinesDev L, const LineHdr *__restrict__ hdr, const float *__restrict__ tabs,
             const float *__restrict__ coef, const float *__restrict__ coefT, float *__restrict__ sino,
             float *__restrict__ out, float *__restrict__ outT, int chunks_per_view, int vec, int *err,
             unsigned char *rec, long long rec_cap, unsigned *defer)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const bool ran = strip_chunk<DEG, ADJ, RM, FM>(smem, g, L, hdr, tabs, coef, coefT, sino, out, outT,
                                                   chunks_per_view, vec, err, (int)blockIdx.x, rec, rec_cap);
    if (FM == kFmFixed && !ran && threadIdx.x == 0) defer[2 + atomicAdd(defer, 1u)] = blockIdx.x;
}

// The deferred adjoint chunks (float strip accumulators): a small persistent
// grid over defer[2 .. 2 + defer[0]), defer[1] its counter.
template <int DEG, int RM>
__global__ void __launch_bounds__(kThreads, 2)
strip_float_kernel(GridDev g, LinesDev L, const LineHdr *__restrict__ hdr, const float *__restrict__ tabs,
                   float *__restrict__ sino, float *__restrict__ out, float *__restrict__ outT, int chunks_per_view,
                   int vec, int *err, unsigned char *rec, long long rec_cap, unsigned *defer)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned cur;
    const unsigned n = defer[0];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(defer + 1, 1u);
        __syncthreads();
        if (cur >= n) break;
        strip_chunk<DEG, true, RM, kFmFloat>(smem, g, L, hdr, tabs, nullptr, nullptr, sino, out, outT,
                                             chunks_per_view, vec, err, (int)defer[2 + cur], rec, rec_cap);
    }
}

// Persistent kernel over the chunks of several instances of one degree: each
// CTA takes the next chunk from one counter (atomicAdd; no CTA waits on
// another) and runs it with its instance's parameters, until every chunk is
// taken.  Instance k owns chunks [jobs[k].chunk0, jobs[k + 1].chunk0).  The
// adjoint runs the fixed-point chunks and appends the others to defer[]
// (count *defer_n) for strip_queue_float_kernel, as the per-instance adjoint
// does with its second launch.  (One kernel per degree: a kernel holding all
// three degrees spilled over a hundred bytes per thread.)
__device__ __forceinline__ const StripJob *queue_job(const StripJob *__restrict__ jobs, int njobs, long long c)
{
    int lo = 0, hi = njobs - 1;   // last job whose first chunk is <= c
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].chunk0 <= c) lo = mid;
        else hi = mid - 1;
    }
    return jobs + lo;
}

template <int DEG, bool ADJ>
__global__ void __launch_bounds__(kThreads, 2)
strip_queue_kernel(const StripJob *__restrict__ jobs, int njobs, long long total, unsigned long long *counter,
                   long long *defer, unsigned long long *defer_n)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long cur;
    for (;;) {
        __syncthreads();   // the previous chunk's last readers of shared memory are done
        if (threadIdx.x == 0) cur = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long c = cur;
        if (c >= total) break;
        const StripJob *J = queue_job(jobs, njobs, c);
        const bool ran = strip_chunk<DEG, ADJ, kRecNone, ADJ ? kFmFixed : kFmAll>(
            smem, J->g, J->L, J->hdr, J->tabs, J->coef, J->coefT, J->sino, J->out, J->outT, J->cpv, J->vec, J->err,
            (int)(c - J->chunk0));
        if (ADJ && !ran && threadIdx.x == 0) defer[atomicAdd(defer_n, 1ull)] = c;
    }
}

// The deferred adjoint chunks (float strip accumulators), persistent likewise.
template <int DEG>
__global__ void __launch_bounds__(kThreads, 2)
strip_queue_float_kernel(const StripJob *__restrict__ jobs, int njobs, const long long *__restrict__ defer,
                         const unsigned long long *__restrict__ defer_n, unsigned long long *counter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long cur;
    const unsigned long long n = *defer_n;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) cur = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long k = cur;
        if (k >= (long long)n) break;
        const long long c = defer[k];
        const StripJob *J = queue_job(jobs, njobs, c);
        strip_chunk<DEG, true, kRecNone, kFmFloat>(smem, J->g, J->L, J->hdr, J->tabs, J->coef, J->coefT, J->sino,
                                                   J->out, J->outT, J->cpv, J->vec, J->err, (int)(c - J->chunk0));
    }
}

template <int DEG>
cudaError_t launch_queue_t(bool adj, const StripJob *jobs, int njobs, int64_t total, unsigned long long *counter,
                           long long *defer, int64_t grid, int sms, cudaStream_t s)
{
    cudaError_t e;
    if (adj) {
        e = cudaFuncSetAttribute(strip_queue_kernel<DEG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(strip_queue_float_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        strip_queue_kernel<DEG, true><<<(unsigned)grid, kThreads, kSmemBytes, s>>>(jobs, njobs, (long long)total,
                                                                                  counter, defer, counter + 1);
        e = cudaGetLastError();
        // the deferred chunks are few (non-finite or extreme sinogram values): a small grid
        if (e == cudaSuccess)
            strip_queue_float_kernel<DEG><<<(unsigned)(grid < sms ? grid : sms), kThreads, kSmemBytes, s>>>(
                jobs, njobs, defer, counter + 1, counter + 2);
        return e == cudaSuccess ? cudaGetLastError() : e;
    }
    e = cudaFuncSetAttribute(strip_queue_kernel<DEG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    strip_queue_kernel<DEG, false><<<(unsigned)grid, kThreads, kSmemBytes, s>>>(jobs, njobs, (long long)total, counter,
                                                                               nullptr, nullptr);
    return cudaGetLastError();
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
                           const float *coef, float *imgT, float *sino, float *out, int *err, cudaStream_t s,
                           const StripRec *rec = nullptr, int rmode = kRecNone, unsigned *defer = nullptr)
{
    const dim3 tb(32, 8), tg((g.nx + 31) / 32, (g.ny + 31) / 32);
    cudaError_t e;
    unsigned char *rb = (rec && rmode != kRecNone) ? rec->base : nullptr;
    const long long rcap = rb ? rec->line_bytes : 0;
    if (!rb) rmode = kRecNone;
    if (ADJ && !defer) return cudaErrorInvalidValue;
    if (rmode == kRecWrite) {
        // records only: no image in or out
    } else if (!ADJ) {
        transpose_kernel<<<tg, tb, 0, s>>>(coef, imgT, g.nx, g.ny);
    } else {
        e = cudaMemsetAsync(out, 0, sizeof(float) * (size_t)g.nx * g.ny, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(imgT, 0, sizeof(float) * (size_t)g.nx * g.ny, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(defer, 0, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    // the adjoint: fixed-point chunks, then (a small second launch) the
    // chunks they deferred to float strips
    constexpr int FM1 = ADJ ? kFmFixed : kFmAll;
    auto kern = rmode == kRecRead ? strip_kernel<DEG, ADJ, kRecRead, FM1>
                : rmode == kRecWrite ? strip_kernel<DEG, ADJ, (ADJ ? kRecNone : kRecWrite), FM1>
                                     : strip_kernel<DEG, ADJ, kRecNone, FM1>;
    auto kern2 = rmode == kRecRead ? strip_float_kernel<DEG, kRecRead> : strip_float_kernel<DEG, kRecNone>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess && ADJ)
        e = cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    if (strip_needs_order(L) && !L.order) return cudaErrorInvalidValue;   // free lists need their order
    const int cpv = (int)((chunk_bins(L) + kChunk - 1) / kChunk);
    const unsigned grid = (unsigned)(chunk_views(L) * cpv);
    // 16-byte staging and flushing: image rows (nx and ny floats) and bases aligned
    const float *img = ADJ ? out : coef;
    const int vec = (g.nx % 4 == 0) && (g.ny % 4 == 0) && ((reinterpret_cast<uintptr_t>(img) & 15) == 0) &&
                    ((reinterpret_cast<uintptr_t>(imgT) & 15) == 0);
    kern<<<grid, kThreads, kSmemBytes, s>>>(g, L, hdr, tabs, coef, imgT, const_cast<float *>(sino), out, imgT, cpv,
                                            vec, err, rb, rcap, defer);
    e = cudaGetLastError();
    if (e == cudaSuccess && ADJ) {
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned g2 = grid < (unsigned)sms ? grid : (unsigned)sms;
        if (e == cudaSuccess)
            kern2<<<g2, kThreads, kSmemBytes, s>>>(g, L, hdr, tabs, const_cast<float *>(sino), out, imgT, cpv, vec,
                                                   err, rb, rcap, defer);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess && ADJ && rmode != kRecWrite) {
        add_transposed_kernel<<<tg, tb, 0, s>>>(imgT, out, g.nx, g.ny);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

StripJob make_strip_job(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs, bool adj,
                        const float *img_in, float *sino, float *img_out, void *scratch, int *err)
{
    StripJob J;
    J.g = g;
    J.L = L;
    J.hdr = hdr;
    J.tabs = tabs;
    J.coef = adj ? nullptr : img_in;
    J.coefT = static_cast<float *>(scratch);
    J.sino = sino;
    J.out = adj ? img_out : nullptr;
    J.outT = static_cast<float *>(scratch);
    J.err = err;
    J.cpv = (int)((chunk_bins(L) + kChunk - 1) / kChunk);
    const void *img = adj ? static_cast<const void *>(img_out) : static_cast<const void *>(img_in);
    J.vec = (g.nx % 4 == 0) && (g.ny % 4 == 0) && ((reinterpret_cast<uintptr_t>(img) & 15) == 0) &&
            ((reinterpret_cast<uintptr_t>(scratch) & 15) == 0);
    J.chunk0 = 0;
    return J;
}

int64_t strip_job_chunks(const StripJob &J) { return chunk_views(J.L) * J.cpv; }

cudaError_t launch_strip_pre(const StripJob &J, bool adj, cudaStream_t s)
{
    const dim3 tb(32, 8), tg((J.g.nx + 31) / 32, (J.g.ny + 31) / 32);
    if (!adj) {
        transpose_kernel<<<tg, tb, 0, s>>>(J.coef, J.coefT, J.g.nx, J.g.ny);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(J.out, 0, sizeof(float) * (size_t)J.g.nx * J.g.ny, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(J.outT, 0, sizeof(float) * (size_t)J.g.nx * J.g.ny, s);
    return e;
}

cudaError_t launch_strip_post(const StripJob &J, bool adj, cudaStream_t s)
{
    if (!adj) return cudaSuccess;
    const dim3 tb(32, 8), tg((J.g.nx + 31) / 32, (J.g.ny + 31) / 32);
    add_transposed_kernel<<<tg, tb, 0, s>>>(J.outT, J.out, J.g.nx, J.g.ny);
    return cudaGetLastError();
}

cudaError_t launch_strip_queue(int deg, bool adj, const StripJob *jobs, int njobs, int64_t total,
                               unsigned long long *counter, long long *defer, cudaStream_t s)
{
    if (njobs <= 0 || total <= 0) return cudaSuccess;
    if (deg < 0 || deg > 3 || (adj && !defer)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int64_t grid = 2 * (int64_t)sms;   // two CTAs per SM, resident at once
    if (grid > total) grid = total;
    switch (deg) {
    case 0: return launch_queue_t<0>(adj, jobs, njobs, total, counter, defer, grid, sms, s);
    case 1: return launch_queue_t<1>(adj, jobs, njobs, total, counter, defer, grid, sms, s);
    case 2: return launch_queue_t<2>(adj, jobs, njobs, total, counter, defer, grid, sms, s);
    default: return launch_queue_t<3>(adj, jobs, njobs, total, counter, defer, grid, sms, s);
    }
}

bool strip_supported(const GridDev &g, const LinesDev &L)
{
    return (L.kind == SP_LINES_PARALLEL || L.kind == SP_LINES_FAN || strip_needs_order(L)) && g.kdeg >= 0;
}

size_t strip_scratch_bytes(const GridDev &g) { return sizeof(float) * (size_t)g.nx * g.ny + 256; }

long long strip_rec_line_bytes(const GridDev &g)
{
    // A line's rows lie in [0, Nr) (Nr the grid's extent along its major
    // axis) and are split into strip slabs of kSlabRows, each into batches of
    // kBatch: at most nb = 2 ceil(Nr / kSlabRows) batches, hence at most
    // Nr + nb 3 (n + 2) records (each interval segment padded by at most 3),
    // 8 bytes each, and a 16-byte header per batch.
    const long long nr = g.nx > g.ny ? g.nx : g.ny;
    const long long nb = 2 * ((nr + kSlabRows - 1) / kSlabRows) + 2;
    const long long bytes = nb * 16 + 8 * (nr + nb * 3 * (g.kdeg + 2));
    return (bytes + 15) & ~15LL;
}

cudaError_t launch_fwd_strip(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                             const float *coef, void *scratch, float *sino, int *err, cudaStream_t s,
                             const StripRec *rec)
{
    float *coefT = static_cast<float *>(scratch);
    const int rm = rec ? kRecRead : kRecNone;
    switch (g.kdeg) {
    case 0: return launch_strip_t<0, false>(g, L, hdr, tabs, coef, coefT, sino, nullptr, err, s, rec, rm);
    case 1: return launch_strip_t<1, false>(g, L, hdr, tabs, coef, coefT, sino, nullptr, err, s, rec, rm);
    case 2: return launch_strip_t<2, false>(g, L, hdr, tabs, coef, coefT, sino, nullptr, err, s, rec, rm);
    default: return launch_strip_t<3, false>(g, L, hdr, tabs, coef, coefT, sino, nullptr, err, s, rec, rm);
    }
}

int64_t strip_chunk_count(const LinesDev &L) { return chunk_views(L) * ((chunk_bins(L) + kChunk - 1) / kChunk); }

cudaError_t launch_adj_strip(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                             const float *sino, void *scratch, float *coef_out, int *err, cudaStream_t s,
                             const StripRec *rec, unsigned *defer)
{
    float *outT = static_cast<float *>(scratch);
    float *p = const_cast<float *>(sino);
    const int rm = rec ? kRecRead : kRecNone;
    switch (g.kdeg) {
    case 0: return launch_strip_t<0, true>(g, L, hdr, tabs, nullptr, outT, p, coef_out, err, s, rec, rm, defer);
    case 1: return launch_strip_t<1, true>(g, L, hdr, tabs, nullptr, outT, p, coef_out, err, s, rec, rm, defer);
    case 2: return launch_strip_t<2, true>(g, L, hdr, tabs, nullptr, outT, p, coef_out, err, s, rec, rm, defer);
    default: return launch_strip_t<3, true>(g, L, hdr, tabs, nullptr, outT, p, coef_out, err, s, rec, rm, defer);
    }
}

cudaError_t launch_strip_record(const GridDev &g, const LinesDev &L, const LineHdr *hdr, const float *tabs,
                                const StripRec &rec, cudaStream_t s)
{
    switch (g.kdeg) {
    case 0: return launch_strip_t<0, false>(g, L, hdr, tabs, nullptr, nullptr, nullptr, nullptr, nullptr, s, &rec, kRecWrite);
    case 1: return launch_strip_t<1, false>(g, L, hdr, tabs, nullptr, nullptr, nullptr, nullptr, nullptr, s, &rec, kRecWrite);
    case 2: return launch_strip_t<2, false>(g, L, hdr, tabs, nullptr, nullptr, nullptr, nullptr, nullptr, s, &rec, kRecWrite);
    default: return launch_strip_t<3, false>(g, L, hdr, tabs, nullptr, nullptr, nullptr, nullptr, nullptr, s, &rec, kRecWrite);
    }
}

}  // namespace spx
