// Conjugate gradients on the normal equations (CGLS) with the plan's
// projector: the reconstruction step of Sec. V, where the linear system
// A^T A x = A^T y is solved by conjugate gradients.
//
// Vector work per iteration is three kernels besides the two projections:
// a dot product whose last block also forms the step length, a fused update
// of the iterate and the residual, and a fused direction update.  Scalars
// stay on the device, so an iteration never waits for the host.
#include <cstdint>

#include "common.cuh"

namespace spx {
namespace {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 2 * 152;   // partial sums, reduced in a fixed order

// Scalars of one CGLS run (device memory).
struct CgScalars {
    double gamma;     // <s, s> of the current residual of the normal equations
    double alpha;     // step length gamma / <q, q>
    double beta;      // gamma_new / gamma
    unsigned int ticket;
};

enum DotRole { kDotAlpha = 0, kDotGamma0 = 1, kDotGammaNext = 2 };

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < kDotThreads / 32) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;   // valid in thread 0
}

// <a, a> in FP64 (partial sums per block, then the last block to finish adds
// them in block order and updates the CG scalars according to `role`).
__global__ void __launch_bounds__(kDotThreads) dot_kernel(const float *__restrict__ a, int64_t n,
                                                          double *__restrict__ partial, CgScalars *sc,
                                                          int role, double *hist, int k)
{
    __shared__ double sh[kDotThreads / 32];
    __shared__ bool last;
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads) {
        const double x = (double)a[i];
        v = fma(x, x, v);
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = v;
        __threadfence();
        last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kDotThreads) t += __ldcg(partial + b);
    // fixed order: per-thread strided sums, then the tree of block_sum
    __syncthreads();
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        sc->ticket = 0u;
        if (role == kDotAlpha) {
            sc->alpha = (t > 0.0) ? sc->gamma / t : 0.0;
        } else if (role == kDotGamma0) {
            sc->gamma = t;
            sc->beta = 0.0;
            if (hist) hist[0] = t;
        } else {
            sc->beta = (sc->gamma > 0.0) ? t / sc->gamma : 0.0;
            sc->gamma = t;
            if (hist) hist[k] = t;
        }
    }
}

// r = b - q
__global__ void residual_kernel(const float *__restrict__ b, const float *__restrict__ q, float *__restrict__ r,
                                int64_t m)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - q[i];
}

// x += alpha p (n values), r -= alpha q (m values)
__global__ void update_xr_kernel(float *__restrict__ x, const float *__restrict__ p, int64_t n,
                                 float *__restrict__ r, const float *__restrict__ q, int64_t m,
                                 const CgScalars *__restrict__ sc)
{
    const float alpha = (float)sc->alpha;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n || i < m; i += stride) {
        if (i < n) x[i] = __fmaf_rn(alpha, p[i], x[i]);
        if (i < m) r[i] = __fmaf_rn(-alpha, q[i], r[i]);
    }
}

// p = s + beta p
__global__ void update_p_kernel(float *__restrict__ p, const float *__restrict__ s, int64_t n,
                                const CgScalars *__restrict__ sc)
{
    const float beta = (float)sc->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = __fmaf_rn(beta, p[i], s[i]);
}

inline unsigned vec_blocks(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

size_t cg_workspace_bytes(int64_t n, int64_t m)
{
    // r, q [m]; s, p [n]; partial sums; scalars
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    return al(sizeof(float) * (size_t)m) * 2 + al(sizeof(float) * (size_t)n) * 2 + al(sizeof(double) * kDotBlocks) +
           al(sizeof(CgScalars));
}

cudaError_t run_cgls(const CgOps &ops, int64_t n, int64_t m, const float *b, float *x, int iters, double *hist,
                     void *ws, cudaStream_t s)
{
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    char *w = static_cast<char *>(ws);
    float *r = reinterpret_cast<float *>(w);
    w += al(sizeof(float) * (size_t)m);
    float *q = reinterpret_cast<float *>(w);
    w += al(sizeof(float) * (size_t)m);
    float *sv = reinterpret_cast<float *>(w);
    w += al(sizeof(float) * (size_t)n);
    float *p = reinterpret_cast<float *>(w);
    w += al(sizeof(float) * (size_t)n);
    double *partial = reinterpret_cast<double *>(w);
    w += al(sizeof(double) * kDotBlocks);
    CgScalars *sc = reinterpret_cast<CgScalars *>(w);

    cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(CgScalars), s);
    if (e != cudaSuccess) return e;
    // r = b - A x0; s = A^T r; p = s; gamma = <s, s>
    if ((e = ops.fwd(ops.ctx, x, q, s)) != cudaSuccess) return e;
    residual_kernel<<<vec_blocks(m), 256, 0, s>>>(b, q, r, m);
    if ((e = ops.adj(ops.ctx, r, sv, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(p, sv, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    dot_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(sv, n, partial, sc, kDotGamma0, hist, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int k = 1; k <= iters; ++k) {
        if ((e = ops.fwd(ops.ctx, p, q, s)) != cudaSuccess) return e;
        dot_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(q, m, partial, sc, kDotAlpha, nullptr, k);
        update_xr_kernel<<<vec_blocks(n > m ? n : m), 256, 0, s>>>(x, p, n, r, q, m, sc);
        if ((e = ops.adj(ops.ctx, r, sv, s)) != cudaSuccess) return e;
        dot_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(sv, n, partial, sc, kDotGammaNext, hist, k);
        update_p_kernel<<<vec_blocks(n), 256, 0, s>>>(p, sv, n, sc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace spx
