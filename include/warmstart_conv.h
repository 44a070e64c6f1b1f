/*
 * warmstart_conv.h -- 3x3 convolution layers of the learned warm start for
 * the conjugate-gradient reconstruction (part of libspline_project.so).
 *
 * No counterpart in the paper: the network maps the backprojection A^T y to
 * an initial guess of the coefficients (it does not change the projector).
 *
 * All layers: 3x3 cross-correlation with taps d = dilation (1..16) apart,
 * stride 1, zero padding d, NHWC tensors [B][H][W][C] with B, H, W >= 1,
 * channels (cin, cout) in {(1, 32), (32, 32), (32, 1)}:
 *   y[b,h,w,o] = bias[o] + sum_{ky,kx,i} x[b,h+(ky-1)d,w+(kx-1)d,i] W[o,ky,kx,i].
 * Weights W are BF16 [cout][3][3][cin]; bias FP32 [cout] (NULL = 0).
 * Activations x are BF16; products accumulate in FP32.  All pointers are
 * device pointers, 16-byte aligned; work is enqueued on `stream`.  Host
 * argument errors return SP_EINVAL (message in sp_last_error()).
 */
#ifndef WARMSTART_CONV_H
#define WARMSTART_CONV_H

#include "spline_project.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Forward: y BF16 [B][H][W][cout] (FP32 [B][H][W] when cout = 1); relu != 0
 * clamps at 0 after the bias.  32 -> 32 runs on the fifth-generation tensor
 * cores (tcgen05.mma, BF16 inputs, FP32 accumulators in tensor memory; 128
 * pixels of a row per CTA); 1 -> 32 and 32 -> 1 on the CUDA cores. */
sp_status sp_conv3x3_fwd(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                         int32_t dilation, const void *x, const void *w, const float *bias, int32_t relu,
                         void *y, void *stream);

/* Input gradient: dx[b,h,w,i] = sum_{ky,kx,o} g[b,h-(ky-1)d,w-(kx-1)d,o] W[o,ky,kx,i]
 * with g FP32 [B][H][W][cout] and dx FP32 [B][H][W][cin]; if gate != NULL
 * (BF16 [B][H][W][cin]) dx is zeroed where gate <= 0 (ReLU of the layer
 * below).  32 -> 32 runs on the tcgen05 tensor cores (g rounded to BF16,
 * FP32 accumulation in tensor memory; g, w, dx and gate 16-byte aligned);
 * the others on the CUDA cores in FP32. */
sp_status sp_conv3x3_bwd_data(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                              int32_t dilation, const float *g, const void *w, const void *gate, float *dx,
                              void *stream);

/* Weight gradient: dw[o,ky,kx,i] = sum_{b,h,w} g[b,h,w,o] x[b,h+(ky-1)d,w+(kx-1)d,i]
 * (FP32 [cout][3][3][cin], overwritten) and dbias[o] = sum g[b,h,w,o]
 * (FP32 [cout], overwritten).  x BF16 [B][H][W][cin], g FP32.  32 -> 32 runs
 * on the tcgen05 tensor cores (g rounded to BF16 in dw, FP32 accumulation in
 * tensor memory, one atomic add per entry and block, so the order of the
 * blocks' partial sums may vary between runs; dbias from g in FP32); the
 * others on the CUDA cores in FP32.  Returns SP_EINVAL for unsupported
 * channels, a dilation outside 1..16, NULL pointers, or (32 -> 32) x or g
 * not 16-byte aligned. */
sp_status sp_conv3x3_bwd_weight(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                                int32_t dilation, const void *x, const float *g, float *dw, float *dbias,
                                void *stream);

/* wf[i][2-ky][2-kx][o] = w[o][ky][kx][i] (BF16): the input gradient written
 * as a forward convolution with cin and cout exchanged. */
sp_status sp_conv3x3_flip_weights(int32_t cin, int32_t cout, const void *w, void *wf,
                                  void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WARMSTART_CONV_H */
