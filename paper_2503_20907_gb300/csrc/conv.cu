// 3x3 convolution layers of the warm-start network (no paper counterpart):
// stride 1, zero padding 1, NHWC, BF16 activations and weights, FP32
// accumulation.
//
// Taps may be dilated (offsets -d, 0, d).
//
//   forward, 32 -> 32 channels: implicit GEMM on the fifth-generation
//     tensor cores (conv32_tc05_kernel: tcgen05.mma, BF16 in, FP32
//     accumulators in tensor memory, read back with tcgen05.ld).  A CTA
//     takes 128 pixels of one image row; the three input rows it needs and
//     the weights are staged in shared memory in the canonical K-major
//     layout, so each tap's operand is the staged rows read from another
//     start address.  Epilogue: bias, optional ReLU, BF16 store.
//   forward, 1 -> 32 and 32 -> 1: CUDA cores, thread per pixel.
//   gradients of the 32 -> 32 layers (training), on the tensor cores too:
//     the input gradient is the same tcgen05 kernel run on the incoming
//     gradient g (rounded to BF16 while it is staged) with the weights
//     flipped while they are staged (W'[i, 8 - tap, o] = W[o, tap, i]), FP32
//     output gated by the ReLU of the layer below; the weight gradient
//     (conv32_wgrad_tc05_kernel) is a tcgen05 GEMM over the pixels (M = 4
//     taps x 32 input channels per tile, N = 32 output channels, K = pixels)
//     with g and the nine shifted inputs staged transposed, one partial sum
//     per block added to the result.
//   gradients of the 1 -> 32 and 32 -> 1 layers: CUDA cores in FP32.
#include <cuda_bf16.h>

#include <cstdint>
#include <string>

#include "common.cuh"
#include "../../include/warmstart_conv.h"

namespace spx {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kC = 32;              // channels of the inner layers
constexpr int kMaxDil = 16;         // largest dilation of the taps

__device__ __forceinline__ float ld_act(const bf16 *p) { return __bfloat162float(*p); }

// Forward on CUDA cores for cin = 1 (y bf16 [.., 32]) or cout = 1 (y float [..]).
__global__ void conv_edge_fwd_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ w,
                                     const float *__restrict__ bias, void *y, int B, int H, int W, int cin,
                                     int cout, int relu, int dil)
{
    __shared__ float wsh[9 * kC];
    for (int i = threadIdx.x; i < 9 * kC; i += blockDim.x) wsh[i] = __bfloat162float(w[i]);
    __syncthreads();
    const int64_t n = (int64_t)B * H * W;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int ww = (int)(p % W), hh = (int)((p / W) % H);
        const int64_t bb = p / ((int64_t)W * H);
        if (cin == 1) {
            float acc[kC];
#pragma unroll
            for (int o = 0; o < kC; ++o) acc[o] = bias ? bias[o] : 0.f;
            for (int tap = 0; tap < 9; ++tap) {
                const int y0 = hh + (tap / 3 - 1) * dil, x0 = ww + (tap % 3 - 1) * dil;
                if (y0 < 0 || y0 >= H || x0 < 0 || x0 >= W) continue;
                const float v = ld_act(x + (bb * H + y0) * W + x0);
#pragma unroll
                for (int o = 0; o < kC; ++o) acc[o] = __fmaf_rn(v, wsh[o * 9 + tap], acc[o]);
            }
            bf16 *out = static_cast<bf16 *>(y) + p * kC;
#pragma unroll
            for (int o = 0; o < kC; o += 2) {
                float v0 = acc[o], v1 = acc[o + 1];
                if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                *reinterpret_cast<__nv_bfloat162 *>(out + o) = __floats2bfloat162_rn(v0, v1);
            }
        } else {
            float acc = bias ? bias[0] : 0.f;
            for (int tap = 0; tap < 9; ++tap) {
                const int y0 = hh + (tap / 3 - 1) * dil, x0 = ww + (tap % 3 - 1) * dil;
                if (y0 < 0 || y0 >= H || x0 < 0 || x0 >= W) continue;
                const bf16 *xp = x + ((bb * H + y0) * W + x0) * kC;
#pragma unroll
                for (int i = 0; i < kC; ++i) acc = __fmaf_rn(ld_act(xp + i), wsh[tap * kC + i], acc);
            }
            if (relu) acc = fmaxf(acc, 0.f);
            static_cast<float *>(y)[p] = acc;
        }
    }
}

// dx[p, i] = sum_{tap, o} g[p - off(tap), o] W[o, tap, i], gated by x_gate[p, i] > 0.
template <int CIN, int COUT>
__global__ void conv_dgrad_kernel(const float *__restrict__ g, const bf16 *__restrict__ w,
                                  const bf16 *__restrict__ gate, float *__restrict__ dx, int B, int H, int W, int dil)
{
    __shared__ float wsh[COUT * 9 * CIN];
    for (int i = threadIdx.x; i < COUT * 9 * CIN; i += blockDim.x) wsh[i] = __bfloat162float(w[i]);
    __syncthreads();
    const int64_t n = (int64_t)B * H * W;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int ww = (int)(p % W), hh = (int)((p / W) % H);
        const int64_t bb = p / ((int64_t)W * H);
        float acc[CIN];
#pragma unroll
        for (int i = 0; i < CIN; ++i) acc[i] = 0.f;
        for (int tap = 0; tap < 9; ++tap) {
            const int y0 = hh - (tap / 3 - 1) * dil, x0 = ww - (tap % 3 - 1) * dil;
            if (y0 < 0 || y0 >= H || x0 < 0 || x0 >= W) continue;
            const float *gp = g + ((bb * H + y0) * W + x0) * COUT;
#pragma unroll 4
            for (int o = 0; o < COUT; ++o) {
                const float gv = gp[o];
                const float *wr = wsh + (o * 9 + tap) * CIN;
#pragma unroll
                for (int i = 0; i < CIN; ++i) acc[i] = __fmaf_rn(gv, wr[i], acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < CIN; ++i) {
            float v = acc[i];
            if (gate && !(__bfloat162float(gate[p * CIN + i]) > 0.f)) v = 0.f;
            dx[p * CIN + i] = v;
        }
    }
}

// dW[o, tap, i] += sum_p g[p, o] x[p + off(tap), i]; dbias[o] += sum_p g[p, o].
// A CTA takes `rows` image rows (over B*H) one at a time, with the row of g
// (FP32) and the three rows of x it meets (BF16) staged in shared memory.
// Each thread owns a block of OB x IB outputs of one tap (OB = min(cout, 4),
// IB = min(cin, 4)); the bias gradient is taken by extra threads.
__global__ void conv_wgrad_kernel(const bf16 *__restrict__ x, const float *__restrict__ g, float *__restrict__ dw,
                                  float *__restrict__ db, int B, int H, int W, int cin, int cout, int rows, int dil)
{
    extern __shared__ __align__(16) unsigned char smw[];
    float *gs = reinterpret_cast<float *>(smw);                           // [W][cout]
    bf16 *xs = reinterpret_cast<bf16 *>(gs + (size_t)W * cout);           // [3][W + 2 dil][cin]
    const int WP = W + 2 * dil;
    const int OB = cout < 4 ? cout : 4, IB = cin < 4 ? cin : 4;
    const int nob = cout / OB, nib = cin / IB;
    const int nblk = 9 * nob * nib;
    const int j = threadIdx.x;
    int tap = 0, ob = 0, ib = 0;
    if (j < nblk) { tap = j / (nob * nib); ob = (j / nib) % nob; ib = j % nib; }
    const int dxo = tap % 3 - 1, dyr = tap / 3;   // staged row dyr = input row h + tap/3 - 1
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
    float bacc = 0.f;
    const int r0 = blockIdx.x * rows, r1 = min(r0 + rows, B * H);
    for (int r = r0; r < r1; ++r) {
        const int bb = r / H, hh = r - bb * H;
        __syncthreads();
        for (int k = threadIdx.x; k < W * cout; k += blockDim.x) gs[k] = g[(size_t)r * W * cout + k];
        for (int k = threadIdx.x; k < 3 * WP * cin; k += blockDim.x) {
            const int rr = k / (WP * cin), rem = k - rr * WP * cin;
            const int p = rem / cin, i = rem - p * cin;
            const int y0 = hh + (rr - 1) * dil, x0 = p - dil;
            xs[k] = (y0 >= 0 && y0 < H && x0 >= 0 && x0 < W) ? x[(((size_t)bb * H + y0) * W + x0) * cin + i]
                                                          : __float2bfloat16(0.f);
        }
        __syncthreads();
        if (j < nblk) {
            const bf16 *xr = xs + ((size_t)dyr * WP + dil + dxo * dil) * cin + ib * IB;
            const float *gr = gs + ob * OB;
            for (int w = 0; w < W; ++w) {
                float gv[4], xv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) gv[a] = a < OB ? gr[(size_t)w * cout + a] : 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) xv[c] = c < IB ? __bfloat162float(xr[(size_t)w * cin + c]) : 0.f;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] = __fmaf_rn(gv[a], xv[c], acc[a][c]);
            }
        } else if (j < nblk + cout) {
            const int o = j - nblk;
            for (int w = 0; w < W; ++w) bacc += gs[(size_t)w * cout + o];
        }
    }
    if (j < nblk) {
        for (int a = 0; a < OB; ++a)
            for (int c = 0; c < IB; ++c)
                atomicAdd(dw + ((size_t)(ob * OB + a) * 9 + tap) * cin + ib * IB + c, acc[a][c]);
    } else if (j < nblk + cout) {
        atomicAdd(db + (j - nblk), bacc);
    }
}

// W'[i, 2-ky, 2-kx, o] = W[o, ky, kx, i] (the input gradient as a forward convolution)
__global__ void flip_weights_kernel(const bf16 *__restrict__ w, bf16 *__restrict__ wf, int cin, int cout)
{
    const int n = cout * 9 * cin;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int o = j / (9 * cin), rem = j - o * 9 * cin, tap = rem / cin, i = rem - tap * cin;
        wf[((size_t)i * 9 + (8 - tap)) * cout + o] = w[j];
    }
}

// ------------------------------------------------------------------ tcgen05
// The 32 -> 32 forward on the fifth-generation tensor cores: one CTA of 4
// warps computes 128 output pixels of one image row as D[128 x 32] =
// sum over the 18 K-steps (9 taps x 2 halves of 16 input channels) of
// A_s[128 x 16] B_s[16 x 32]^T, one tcgen05.mma (kind::f16, BF16 in, FP32
// accumulators in tensor memory) per step, issued by one thread.
//
// Shared-memory operands use the canonical no-swizzle K-major layout: core
// matrices of 8 rows x 16 bytes stored contiguously (128 bytes), LBO the
// byte distance between core matrices along K, SBO along M (or N).
//   input  xs[cg][row][pixel][8]: channel group cg (8 channels) of the three
//          rows h - d, h, h + d and pixels w0 - d .. w0 + 127 + d.  A tap's
//          A operand is the same array read from another start address:
//          LBO = one channel group (kXRows5 * kXPix5 * 16 B), SBO = 128 B
//          (8 pixels of 16 B).
//   weights wb[kc][n][8]: K = tap 32 + input channel in groups kc of 8,
//          n the output channel; LBO = 32 * 16 B, SBO = 128 B.
constexpr int kTile5 = 128;                  // output pixels of one CTA (M)
constexpr int kXPix5 = kTile5 + 2 * kMaxDil;  // staged pixels per row
constexpr int kXRows5 = 3;
constexpr int kXBytes5 = 4 * kXRows5 * kXPix5 * 16;   // 30,720
constexpr int kWBytes5 = 36 * kC * 16;                // 18,432
constexpr int kSmem5 = kXBytes5 + kWBytes5 + 16;      // + mbarrier and TMEM address
constexpr uint32_t kTmemCols5 = 32;                   // FP32 accumulators: N = 32 columns

__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte
// units, the descriptor version of this architecture (bits 46-47 = 1), no
// swizzle (layout type 0), base offset 0.
__host__ __device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit
// 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(uint32_t M, uint32_t N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// y = conv(x) + bias (ReLU optional), 32 -> 32 channels, taps dil apart, on
// tcgen05.  128 threads; warp w reads the accumulators of pixels 32w..32w+31
// (tensor-memory lanes 32w..).  Every wait is bounded; a CTA whose MMAs did
// not complete writes NaN and still frees its tensor memory.
// GRAD: the input gradient instead: x is the FP32 gradient g of the layer's
// output (rounded to BF16 while staged), the weights are flipped while staged
// (W'[i][8 - tap][o] = W[o][tap][i]), y is the FP32 gradient of the layer's
// input, zeroed where gate <= 0 (gate may be NULL).
template <bool GRAD>
__global__ void __launch_bounds__(128) conv32_tc05_kernel(const void *__restrict__ xv, const bf16 *__restrict__ w,
                                                          const float *__restrict__ bias, void *__restrict__ yv,
                                                          int B, int H, int W, int relu, int dil,
                                                          const bf16 *__restrict__ gate)
{
    extern __shared__ __align__(128) unsigned char sm5[];
    unsigned char *xs = sm5;
    unsigned char *wsb = sm5 + kXBytes5;
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(sm5 + kXBytes5 + kWBytes5);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_w = (W + kTile5 - 1) / kTile5;
    const int tw = blockIdx.x % tiles_w;
    const int h = (blockIdx.x / tiles_w) % H;
    const int b = blockIdx.x / (tiles_w * H);
    const int w0 = tw * kTile5;

    // tensor memory (warp 0) and the MMA completion barrier (thread 0)
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(tslot)),
                     "r"(kTmemCols5)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights: wb[kc][n][8] = W[n][kc 8 .. kc 8 + 7] (W is [n][tap][i], K = tap 32 + i);
    // flipped for the input gradient: n = i, K = tap' 32 + o, W[o][8 - tap'][i]
    for (int i = threadIdx.x; i < 36 * kC; i += 128) {
        const int kc = i / kC, n = i - kc * kC;
        if constexpr (GRAD) {
            const int tp = kc >> 2, o0 = (kc & 3) * 8;
            __align__(16) bf16 e[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) e[j] = w[((size_t)(o0 + j) * 9 + (8 - tp)) * kC + n];
            *reinterpret_cast<uint4 *>(wsb + (kc * kC + n) * 16) = *reinterpret_cast<const uint4 *>(e);
        } else {
            *reinterpret_cast<uint4 *>(wsb + (kc * kC + n) * 16) =
                *reinterpret_cast<const uint4 *>(w + (size_t)n * 9 * kC + kc * 8);
        }
    }
    // input rows h - d, h, h + d; pixels w0 - d .. w0 + 127 + d; zero outside
    const int tw2 = kTile5 + 2 * dil;
    for (int i = threadIdx.x; i < kXRows5 * tw2 * 4; i += 128) {
        const int r = i / (tw2 * 4), rem = i - r * tw2 * 4;
        const int p = rem >> 2, cg = rem & 3;
        const int hh = h + (r - 1) * dil, ww = w0 + p - dil;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (hh >= 0 && hh < H && ww >= 0 && ww < W) {
            const size_t off = (((size_t)b * H + hh) * W + ww) * kC + cg * 8;
            if constexpr (GRAD) {
                const float4 f0 = *reinterpret_cast<const float4 *>(static_cast<const float *>(xv) + off);
                const float4 f1 = *reinterpret_cast<const float4 *>(static_cast<const float *>(xv) + off + 4);
                __nv_bfloat162 q[4] = {__floats2bfloat162_rn(f0.x, f0.y), __floats2bfloat162_rn(f0.z, f0.w),
                                       __floats2bfloat162_rn(f1.x, f1.y), __floats2bfloat162_rn(f1.z, f1.w)};
                v = *reinterpret_cast<const uint4 *>(q);
            } else {
                v = *reinterpret_cast<const uint4 *>(static_cast<const bf16 *>(xv) + off);
            }
        }
        *reinterpret_cast<uint4 *>(xs + ((cg * kXRows5 + r) * kXPix5 + p) * 16) = v;
    }
    // generic-proxy shared stores visible to the tensor cores, then sync
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = *tslot;

    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = umma_idesc_bf16(kTile5, kC);
        const uint32_t xbase = s_u32(xs), wbase = s_u32(wsb);
        constexpr uint32_t kGroup = kXRows5 * kXPix5 * 16;   // A: LBO (next 8 channels)
#pragma unroll 1
        for (int s = 0; s < 18; ++s) {
            const int tap = s >> 1, half = s & 1;
            const int ky = tap / 3, kx = tap - 3 * ky;
            const uint32_t a_addr = xbase + (uint32_t)(2 * half) * kGroup + (uint32_t)(ky * kXPix5 * 16) +
                                    (uint32_t)(kx * dil) * 16u;
            const uint64_t adesc = umma_smem_desc(a_addr, kGroup, 128);
            const uint64_t bdesc = umma_smem_desc(wbase + (uint32_t)s * 2u * kC * 16u, kC * 16, 128);
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                         "l"(adesc), "l"(bdesc), "r"(idesc), "r"(s)
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         s_u32(mbar))
                     : "memory");
    }
    // wait (bounded) for the MMAs
    bool done = false;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(s_u32(mbar))
                     : "memory");
        done = ok != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // accumulators of this warp's 32 pixels: 32 columns (output channels)
    uint32_t acc[kC];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                 "[%32];"
                 : "=r"(acc[0]), "=r"(acc[1]), "=r"(acc[2]), "=r"(acc[3]), "=r"(acc[4]), "=r"(acc[5]),
                   "=r"(acc[6]), "=r"(acc[7]), "=r"(acc[8]), "=r"(acc[9]), "=r"(acc[10]), "=r"(acc[11]),
                   "=r"(acc[12]), "=r"(acc[13]), "=r"(acc[14]), "=r"(acc[15]), "=r"(acc[16]), "=r"(acc[17]),
                   "=r"(acc[18]), "=r"(acc[19]), "=r"(acc[20]), "=r"(acc[21]), "=r"(acc[22]), "=r"(acc[23]),
                   "=r"(acc[24]), "=r"(acc[25]), "=r"(acc[26]), "=r"(acc[27]), "=r"(acc[28]), "=r"(acc[29]),
                   "=r"(acc[30]), "=r"(acc[31])
                 : "r"(taddr + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // epilogue: pixel w0 + 32 warp + lane, 32 channels = 64 bytes
    const int ww = w0 + warp * 32 + lane;
    if (GRAD && ww < W) {
        const size_t off = (((size_t)b * H + h) * W + ww) * kC;
        float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(yv) + off);
        uint4 gt[4];
        if (gate) {
            const uint4 *gp = reinterpret_cast<const uint4 *>(gate + off);
#pragma unroll
            for (int k = 0; k < 4; ++k) gt[k] = gp[k];
        }
        const bf16 *ge = reinterpret_cast<const bf16 *>(gt);
#pragma unroll
        for (int o = 0; o < kC; o += 4) {
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                v[j] = done ? __uint_as_float(acc[o + j]) : __int_as_float(0x7fc00000);
                if (gate && !(__bfloat162float(ge[o + j]) > 0.f)) v[j] = 0.f;
            }
            dst[o >> 2] = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
    if (!GRAD && ww < W) {
        uint4 out[4];
        __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(out);
#pragma unroll
        for (int o = 0; o < kC; o += 2) {
            float v0 = done ? __uint_as_float(acc[o]) : __int_as_float(0x7fc00000);
            float v1 = done ? __uint_as_float(acc[o + 1]) : __int_as_float(0x7fc00000);
            if (bias) { v0 += bias[o]; v1 += bias[o + 1]; }
            if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
            o2[o >> 1] = __floats2bfloat162_rn(v0, v1);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<bf16 *>(yv) + (((size_t)b * H + h) * W + ww) * kC);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = out[k];
    }
    // free the tensor memory once every warp's loads are done
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols5)
                     : "memory");
    }
}

// The 32 -> 32 weight gradient on tcgen05:
//   dW[o, tap, i] = sum_p g[p, o] x[p + off(tap), i],  dbias[o] = sum_p g[p, o]
// taken as D[(tap, i)][o] = sum over pixels p of A[(tap, i)][p] B[o][p]: M =
// 4 taps x 32 input channels per MMA tile (three tiles; tap slots 9..11 are
// zero), N = the 32 output channels, K = pixels, 16 per MMA.  A block takes
// `rows` image rows (over B*H), each in segments of 128 pixels, thread p
// staging pixel p of the segment: for A, per 8-pixel block, the nine
// shifted inputs as [tap slot][i][8 pixels] (K-major core matrices: LBO one
// pixel block, SBO 8 rows); for B, g rounded to BF16 as [o][8 pixels] (LBO
// 32 x 16 B, SBO 8 rows).  One thread issues the segment's 8 K-steps x 3
// tiles into 96 tensor-memory columns, and the block waits for them
// (bounded) before it stages the next segment.  At the end warp w reads the
// accumulators of taps 4t + w and the block adds them, and its FP32 sums of
// g, to dw and dbias with one atomic per entry; a block whose MMAs did not
// complete adds NaN.
constexpr int kWgSlots5 = 12;                          // tap slots: 9 taps, 3 zero
constexpr int kWgBlockA5 = kWgSlots5 * kC * 16;        // A bytes per 8-pixel block (6,144)
constexpr int kWgABytes5 = (kTile5 / 8) * kWgBlockA5;  // 98,304
constexpr int kWgBBytes5 = (kTile5 / 8) * kC * 16;     // 8,192
constexpr int kWgSmem5 = kWgABytes5 + kWgBBytes5 + 16; // + mbarrier and TMEM address
constexpr uint32_t kWgCols5 = 128;                     // 3 tiles x 32 columns, as a power of two

// Writes the 32 channels of one pixel, v[k] = channels 8k..8k+7 as BF16
// pairs, into the rows c = 0..31 (16-byte pitch) of its column `col` of a
// staged [channel][8 pixels] block.  The four 8-pixel blocks of a warp
// write with their word order rotated by rot = 0..3, so that a store
// instruction of the warp meets 16 distinct banks.
__device__ __forceinline__ void stage_column(unsigned short *col, const uint4 (&v)[4], int rot)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t a0 = v[k].x, a1 = v[k].y, a2 = v[k].z, a3 = v[k].w;
        if (rot & 1) { const uint32_t t = a0; a0 = a1; a1 = a2; a2 = a3; a3 = t; }
        if (rot & 2) { uint32_t t = a0; a0 = a2; a2 = t; t = a1; a1 = a3; a3 = t; }
        const uint32_t q[4] = {a0, a1, a2, a3};   // q[m] = channels 8k + 2((m + rot) & 3) (+1)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int c = 8 * k + 2 * ((m + rot) & 3);
            col[c * 8] = (unsigned short)(q[m] & 0xFFFFu);
            col[(c + 1) * 8] = (unsigned short)(q[m] >> 16);
        }
    }
}

__global__ void __launch_bounds__(128) conv32_wgrad_tc05_kernel(const bf16 *__restrict__ x,
                                                                const float *__restrict__ g, float *__restrict__ dw,
                                                                float *__restrict__ db, int B, int H, int W,
                                                                int rows, int dil)
{
    extern __shared__ __align__(128) unsigned char smw[];
    unsigned char *as = smw;
    unsigned char *bs = smw + kWgABytes5;
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(smw + kWgABytes5 + kWgBBytes5);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pb = threadIdx.x >> 3, pc = threadIdx.x & 7;   // this thread's pixel: block, column
    const int rot = pb & 3;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(tslot)),
                     "r"(kWgCols5)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // tap slots 9..11 of every pixel block stay zero
    for (int k = threadIdx.x; k < (kTile5 / 8) * (kWgSlots5 - 9) * kC; k += 128) {
        const int blk = k / ((kWgSlots5 - 9) * kC), rem = k - blk * (kWgSlots5 - 9) * kC;
        *reinterpret_cast<uint4 *>(as + blk * kWgBlockA5 + (9 * kC + rem) * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = *tslot;

    float gsum[kC];   // FP32 sums of g over this thread's pixels (bias gradient)
#pragma unroll
    for (int o = 0; o < kC; ++o) gsum[o] = 0.f;
    const int r0 = blockIdx.x * rows, r1 = min(r0 + rows, B * H);
    const int segs = (W + kTile5 - 1) / kTile5;
    bool done = true;
    uint32_t nseg = 0;
    for (int r = r0; r < r1 && done; ++r) {
        const int b = r / H, h = r - b * H;
        for (int sg = 0; sg < segs && done; ++sg, ++nseg) {
            const int ww = sg * kTile5 + threadIdx.x;
            // B: g of this pixel in BF16 (zero past the row)
            {
                uint4 v[4] = {};
                if (ww < W) {
                    const float4 *gp = reinterpret_cast<const float4 *>(g + (((size_t)b * H + h) * W + ww) * kC);
                    uint32_t *vw = reinterpret_cast<uint32_t *>(v);
#pragma unroll
                    for (int k = 0; k < kC / 4; ++k) {
                        const float4 f = gp[k];
                        gsum[4 * k] += f.x; gsum[4 * k + 1] += f.y; gsum[4 * k + 2] += f.z; gsum[4 * k + 3] += f.w;
                        const __nv_bfloat162 lo = __floats2bfloat162_rn(f.x, f.y), hi = __floats2bfloat162_rn(f.z, f.w);
                        vw[2 * k] = *reinterpret_cast<const uint32_t *>(&lo);
                        vw[2 * k + 1] = *reinterpret_cast<const uint32_t *>(&hi);
                    }
                }
                stage_column(reinterpret_cast<unsigned short *>(bs + pb * kC * 16) + pc, v, rot);
            }
            // A: the nine shifted inputs of this pixel (zero outside the image)
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap - 3 * ky;
                const int hh = h + (ky - 1) * dil, wx = ww + (kx - 1) * dil;
                uint4 v[4] = {};
                if (ww < W && hh >= 0 && hh < H && wx >= 0 && wx < W) {
                    const uint4 *xp = reinterpret_cast<const uint4 *>(x + (((size_t)b * H + hh) * W + wx) * kC);
#pragma unroll
                    for (int k = 0; k < 4; ++k) v[k] = xp[k];
                }
                stage_column(reinterpret_cast<unsigned short *>(as + pb * kWgBlockA5 + tap * kC * 16) + pc, v, rot);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                constexpr uint32_t idesc = umma_idesc_bf16(kTile5, kC);
                const uint32_t abase = s_u32(as), bbase = s_u32(bs);
#pragma unroll 1
                for (int k = 0; k < kTile5 / 16; ++k) {
                    const uint64_t bdesc = umma_smem_desc(bbase + (uint32_t)(2 * k * kC * 16), kC * 16, 128);
#pragma unroll 1
                    for (int t = 0; t < 3; ++t) {
                        const uint64_t adesc =
                            umma_smem_desc(abase + (uint32_t)(2 * k * kWgBlockA5 + 4 * t * kC * 16), kWgBlockA5, 128);
                        const uint32_t accumulate = (nseg > 0 || k > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                         taddr + (uint32_t)(t * kC)),
                                     "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                                     : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 s_u32(mbar))
                             : "memory");
            }
            // bounded wait for the segment's MMAs before its operands are overwritten
            bool ok_seg = false;
            for (int it = 0; it < (1 << 24) && !ok_seg; ++it) {
                uint32_t ok;
                asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                             "selp.u32 %0, 1, 0, p;\n\t}"
                             : "=r"(ok)
                             : "r"(s_u32(mbar)), "r"(nseg & 1u)
                             : "memory");
                ok_seg = ok != 0;
            }
            done = __syncthreads_and(ok_seg) != 0;   // block-uniform: stop at the first failure
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
    }
    const float bad = __int_as_float(0x7fc00000);
    // bias gradient: the warp's sums, one atomic per channel and warp
#pragma unroll
    for (int o = 0; o < kC; ++o) {
        float v = gsum[o];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) atomicAdd(db + o, done ? v : bad);
    }
    // weight gradient: warp w holds the rows (tap 4t + w, i = lane) of tile t
#pragma unroll 1
    for (int t = 0; t < 3; ++t) {
        uint32_t acc[kC];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                     "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, "
                     "%31}, [%32];"
                     : "=r"(acc[0]), "=r"(acc[1]), "=r"(acc[2]), "=r"(acc[3]), "=r"(acc[4]), "=r"(acc[5]),
                       "=r"(acc[6]), "=r"(acc[7]), "=r"(acc[8]), "=r"(acc[9]), "=r"(acc[10]), "=r"(acc[11]),
                       "=r"(acc[12]), "=r"(acc[13]), "=r"(acc[14]), "=r"(acc[15]), "=r"(acc[16]), "=r"(acc[17]),
                       "=r"(acc[18]), "=r"(acc[19]), "=r"(acc[20]), "=r"(acc[21]), "=r"(acc[22]), "=r"(acc[23]),
                       "=r"(acc[24]), "=r"(acc[25]), "=r"(acc[26]), "=r"(acc[27]), "=r"(acc[28]), "=r"(acc[29]),
                       "=r"(acc[30]), "=r"(acc[31])
                     : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * kC)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int tap = 4 * t + warp;
        if (tap < 9 && nseg > 0) {
#pragma unroll
            for (int o = 0; o < kC; ++o)
                atomicAdd(dw + ((size_t)o * 9 + tap) * kC + lane, done ? __uint_as_float(acc[o]) : bad);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kWgCols5)
                     : "memory");
    }
}

}  // namespace
}  // namespace spx

extern "C" {

sp_status sp_conv3x3_fwd(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dilation,
                         const void *x, const void *w, const float *bias, int32_t relu, void *y, void *stream)
{
    spx::clear_error();
    if (B < 1 || H < 1 || W < 1) return spx::record_error(SP_EINVAL, "B, H, W must be >= 1");
    if (dilation < 1 || dilation > spx::kMaxDil) return spx::record_error(SP_EINVAL, "dilation must be 1..16");
    const bool inner = cin == 32 && cout == 32, edge = (cin == 1 && cout == 32) || (cin == 32 && cout == 1);
    if (!inner && !edge) return spx::record_error(SP_EINVAL, "supported channels: 1->32, 32->32, 32->1");
    if (!x || !w || !y) return spx::record_error(SP_EINVAL, "NULL pointer");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(y)) & 15)
        return spx::record_error(SP_EINVAL, "x, w, y must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const spx::bf16 *xb = static_cast<const spx::bf16 *>(x), *wb = static_cast<const spx::bf16 *>(w);
    if (inner) {
        // tcgen05 (tensor memory accumulators), 128 pixels of a row per CTA
        const int tiles = (W + spx::kTile5 - 1) / spx::kTile5;
        const int64_t grid = (int64_t)B * H * tiles;
        if (grid > 0x7fffffff) return spx::record_error(SP_EINVAL, "too many tiles");
        cudaError_t ea = cudaFuncSetAttribute(spx::conv32_tc05_kernel<false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, spx::kSmem5);
        if (ea != cudaSuccess) return spx::record_error(SP_ECUDA, cudaGetErrorString(ea));
        spx::conv32_tc05_kernel<false><<<(unsigned)grid, 128, spx::kSmem5, s>>>(xb, wb, bias, y, B, H, W, relu,
                                                                                dilation, nullptr);
    } else {
        const int64_t n = (int64_t)B * H * W;
        int64_t blocks = (n + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        spx::conv_edge_fwd_kernel<<<(unsigned)blocks, 256, 0, s>>>(xb, wb, bias, y, B, H, W, cin, cout, relu,
                                                                   dilation);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SP_OK : spx::record_error(SP_ECUDA, cudaGetErrorString(e));
}

sp_status sp_conv3x3_bwd_data(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dilation,
                              const float *g, const void *w, const void *gate, float *dx, void *stream)
{
    spx::clear_error();
    if (B < 1 || H < 1 || W < 1) return spx::record_error(SP_EINVAL, "B, H, W must be >= 1");
    if (dilation < 1 || dilation > spx::kMaxDil) return spx::record_error(SP_EINVAL, "dilation must be 1..16");
    if (!((cin == 32 && (cout == 32 || cout == 1)) || (cin == 1 && cout == 32)))
        return spx::record_error(SP_EINVAL, "supported channels: 1->32, 32->32, 32->1");
    if (!g || !w || !dx) return spx::record_error(SP_EINVAL, "NULL pointer");
    const int64_t n = (int64_t)B * H * W;
    int64_t blocks = (n + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const spx::bf16 *wb = static_cast<const spx::bf16 *>(w), *gb = static_cast<const spx::bf16 *>(gate);
    if (cin == 32 && cout == 32) {
        if ((reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(dx)) & 15)
            return spx::record_error(SP_EINVAL, "g, w, dx must be 16-byte aligned");
        const int tiles = (W + spx::kTile5 - 1) / spx::kTile5;
        const int64_t grid = (int64_t)B * H * tiles;
        if (grid > 0x7fffffff) return spx::record_error(SP_EINVAL, "too many tiles");
        if (gate && (reinterpret_cast<uintptr_t>(gate) & 15))
            return spx::record_error(SP_EINVAL, "gate must be 16-byte aligned");
        cudaError_t ea = cudaFuncSetAttribute(spx::conv32_tc05_kernel<true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, spx::kSmem5);
        if (ea != cudaSuccess) return spx::record_error(SP_ECUDA, cudaGetErrorString(ea));
        spx::conv32_tc05_kernel<true><<<(unsigned)grid, 128, spx::kSmem5, s>>>(g, wb, nullptr, dx, B, H, W, 0,
                                                                               dilation, gb);
    } else if (cin == 32)
        spx::conv_dgrad_kernel<32, 1><<<(unsigned)blocks, 128, 0, s>>>(g, wb, gb, dx, B, H, W, dilation);
    else
        spx::conv_dgrad_kernel<1, 32><<<(unsigned)blocks, 128, 0, s>>>(g, wb, gb, dx, B, H, W, dilation);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SP_OK : spx::record_error(SP_ECUDA, cudaGetErrorString(e));
}

sp_status sp_conv3x3_bwd_weight(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dilation,
                                const void *x, const float *g, float *dw, float *dbias, void *stream)
{
    spx::clear_error();
    if (B < 1 || H < 1 || W < 1) return spx::record_error(SP_EINVAL, "B, H, W must be >= 1");
    if (dilation < 1 || dilation > spx::kMaxDil) return spx::record_error(SP_EINVAL, "dilation must be 1..16");
    if (!((cin == 32 && (cout == 32 || cout == 1)) || (cin == 1 && cout == 32)))
        return spx::record_error(SP_EINVAL, "supported channels: 1->32, 32->32, 32->1");
    if (!x || !g || !dw || !dbias) return spx::record_error(SP_EINVAL, "NULL pointer");
    if (cin == 32 && cout == 32 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(g)) & 15))
        return spx::record_error(SP_EINVAL, "x, g must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(dw, 0, sizeof(float) * (size_t)cout * 9 * cin, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dbias, 0, sizeof(float) * (size_t)cout, s);
    if (cin == 32 && cout == 32) {
        // about two blocks per SM (each holds 104 KB of shared memory), every
        // block at least one image row
        int dev = 0, sms = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(spx::conv32_wgrad_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     spx::kWgSmem5);
        if (e == cudaSuccess) {
            const int64_t nrows = (int64_t)B * H, target = 2 * (int64_t)(sms > 0 ? sms : 1);
            const int rows = (int)((nrows + target - 1) / target);
            const int blocks = (int)((nrows + rows - 1) / rows);
            spx::conv32_wgrad_tc05_kernel<<<blocks, 128, spx::kWgSmem5, s>>>(static_cast<const spx::bf16 *>(x), g, dw,
                                                                             dbias, B, H, W, rows, dilation);
            e = cudaGetLastError();
        }
        return e == cudaSuccess ? SP_OK : spx::record_error(SP_ECUDA, cudaGetErrorString(e));
    }
    const size_t sh = sizeof(float) * (size_t)W * cout + sizeof(spx::bf16) * 3 * (size_t)(W + 2 * dilation) * cin;
    if (sh > 200 * 1024) return spx::record_error(SP_EINVAL, "image too wide for the weight-gradient kernel");
    const int OB = cout < 4 ? cout : 4, IB = cin < 4 ? cin : 4;
    int threads = 9 * (cout / OB) * (cin / IB) + cout;
    threads = (threads + 31) / 32 * 32;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spx::conv_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e == cudaSuccess) {
        const int rows = 16;
        const int blocks = (B * H + rows - 1) / rows;
        spx::conv_wgrad_kernel<<<blocks, threads, sh, s>>>(static_cast<const spx::bf16 *>(x), g, dw, dbias, B, H, W,
                                                           cin, cout, rows, dilation);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? SP_OK : spx::record_error(SP_ECUDA, cudaGetErrorString(e));
}

sp_status sp_conv3x3_flip_weights(int32_t cin, int32_t cout, const void *w, void *wf, void *stream)
{
    spx::clear_error();
    if (cin < 1 || cout < 1 || !w || !wf) return spx::record_error(SP_EINVAL, "bad arguments");
    const int n = cout * 9 * cin;
    spx::flip_weights_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const spx::bf16 *>(w), static_cast<spx::bf16 *>(wf), cin, cout);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SP_OK : spx::record_error(SP_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
