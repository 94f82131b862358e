/*
 * tsurr.h -- C ABI of the learned surface surrogate (part of libtsim.so).
 *
 * Not a part of the paper's method: a project addition.  A convolutional
 * encoder-decoder maps the indenter heightmap and the pose/material scalars
 * of a contact (broadcast as image channels) to the gel surface
 * displacement field that the IMPM simulator produces (tsim_read_displacement),
 * plus one channel that predicts the per-pixel error of that prediction (the
 * residual indicator used to fall back to the simulator).  Training and
 * inference run in hand-written BF16-input / FP32-accumulate tensor-core
 * kernels; the master parameters, gradients and Adam state are FP32.
 *
 * Architecture (fixed; every convolution 3x3, padding 1, NHWC):
 *   L0  in 12 (padded to 16) -> 32,  stride 1, ReLU            a0  (H,   W)
 *   L1  a0  32 -> 64,  stride 2, ReLU                          a1  (H/2, W/2)
 *   L2  a1  64 -> 128, stride 2, ReLU                          a2  (H/4, W/4)
 *   L3  a2 128 -> 256, stride 2, ReLU                          a3  (H/8, W/8)
 *   L4  a3 256 -> 256, stride 1, ReLU                          a4  (H/8, W/8)
 *   L5  up2(a4) 256 -> 128, ReLU(conv + bias + a2)             a5  (H/4, W/4)
 *   L6  up2(a5) 128 -> 64,  ReLU(conv + bias + a1)             a6  (H/2, W/2)
 *   L7  up2(a6)  64 -> 32,  ReLU(conv + bias + a0)             a7  (H,   W)
 *   L8  a7  32 -> 4 (stored as 16 with 12 zero rows), no ReLU  y   (H,   W)
 * up2 = nearest-neighbour upsampling by 2.  Parameters are flattened layer
 * by layer as W[cout][3][3][cin] then b[cout] (FP32).
 *
 * Loss of a batch (x, target t, mask m), with e = |y[0:3] - t| per pixel
 * treated as a constant:
 *   L = sum_p m_p (|y_p[0:3] - t_p|^2 + (y_p[3] - e_p)^2) / sum_p m_p.
 *
 * Conventions as in tsim.h: int status codes (TSIM_*), tsim_last_error()
 * for the reason, the caller's stream, no allocation after tsurr_create.
 *
 * Kernels: the forward, data-gradient and weight-gradient convolutions run
 * on the tcgen05 tensor cores (accumulators in tensor memory; UMMA M = 128
 * pixels x N = cout forward, N = cin for the data gradient, M = cout x
 * N = cin over the pixels for the weight gradient); the weight gradient of
 * a layer whose output width is not a multiple of 16 runs on mma.sync
 * m16n8k16.
 */
#ifndef TSURR_H
#define TSURR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsurr_net tsurr_net;

#define TSURR_CIN 12
#define TSURR_COUT 4

/* Network for batches of up to max_batch images of height x width pixels
 * (multiples of 8, at most 512); allocates parameters, gradients, Adam
 * state, activations and their FP32 gradients, and the channel-major copies
 * of the weight-gradient operands (the output gradient, and three
 * column-shifted copies of the largest layer input), all sized for
 * max_batch: about 1.3 KB of device memory per pixel of max_batch x height
 * x width (5.2 GB at 256 x 128 x 128).  TSIM_ERR_OOM if that does not fit. */
int tsurr_create(int max_batch, int height, int width, void *stream, tsurr_net **out);

/* Number of FP32 parameters (layout above). */
int64_t tsurr_num_params(const tsurr_net *net);

/* Copy the FP32 parameters in (also refreshes the BF16 copies) or out. */
int tsurr_set_params(tsurr_net *net, const float *p, int64_t n, int on_device);
int tsurr_get_params(tsurr_net *net, float *p, int64_t n, int on_device);

/* Gradients of the loss from the last tsurr_backward (FP32, same layout). */
int tsurr_get_grads(tsurr_net *net, float *g, int64_t n, int on_device);

/* y[B,H,W,4] = net(x[B,H,W,12]), FP32 in and out; 1 <= batch <= max_batch. */
int tsurr_forward(tsurr_net *net, const float *x, int batch, float *y, int on_device);

/* Forward and backward of the loss for x[B,H,W,12], target[B,H,W,3],
 * mask[B,H,W]; gradients go to the internal buffer; *loss (host) = L. */
int tsurr_backward(tsurr_net *net, const float *x, const float *target, const float *mask, int batch,
                   double *loss, int on_device);

/* Wait for the network's work on its stream; returns TSIM_ERR_TIMEOUT if a
 * bounded pipeline wait inside a kernel gave up (latched until destroy).
 * tsurr_forward with device pointers does not wait: call this to see such
 * errors; host-pointer calls and tsurr_backward check them themselves. */
int tsurr_sync(tsurr_net *net);

/* One Adam step (bias-corrected, step t >= 1) on all parameters. */
int tsurr_adam(tsurr_net *net, float lr, float beta1, float beta2, float eps, int t);

void tsurr_destroy(tsurr_net *net);

/* Serving helpers (device arrays, the caller's stream, no allocation; they
 * need no network object).  tsurr_features assembles the network input
 * x[B,H,W,12] = [height, px, py, scalars[b][0..8]] from the indenter height
 * maps height[B,H,W] (mm) and the per-frame scalars[B,9], with px = (x + 0.5)
 * / W * 2 - 1 and py = (y + 0.5) / H * 2 - 1; x must be 16-byte aligned.
 * tsurr_indicator reduces the indicator channel of y[B,H,W,4] to the
 * predicted error per frame, out[b] = sqrt(mean over pixels of y[b,:,:,3]^2)
 * / press[b], the quantity the fallback rule compares with its threshold.
 * TSIM_ERR_INVALID_ARG on NULL pointers, non-positive sizes or a misaligned
 * x. */
int tsurr_features(const float *height, const float *scalars, int batch, int height_px, int width_px, float *x,
                   void *stream);
int tsurr_indicator(const float *y, const float *press, int batch, int height_px, int width_px, float *out,
                    void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TSURR_H */
