/*
 * osog_cnn.h - C ABI of libosog's convolution kernels for the learned warm
 * start of inverse rendering: a small BF16 convolutional network with FP32
 * accumulation, trained on images the renderer produces, that predicts the
 * optics and per-particle starting values (no counterpart in the paper's
 * method; it extends the paper's differentiable calibration, Sec. IV.B).
 *
 * Layouts (all device memory owned by the caller):
 *   activations  bf16 NHWC [N][H][W][C], C a multiple of 8
 *   filters      bf16 [K][R][S][C] (K output channels, R x S window,
 *                R, S <= 8), K a multiple of 8
 *   bias         fp32 [K]
 *   gradients    d(activations) bf16 NHWC; d(filters) and d(bias) fp32
 * Convolutions are cross-correlations with zero padding `pad` and stride
 * `stride` (1 or 2): out[n, p, q, k] = bias[k] + sum_{r, s, c}
 * in[n, p stride + r - pad, q stride + s - pad, c] w[k, r, s, c], P =
 * (H + 2 pad - R) / stride + 1.  The matrix products run on the tensor cores
 * in BF16 with FP32 accumulation; every reduction runs in a fixed order.
 * All calls are asynchronous on `stream` and return OSOG_OK or
 * OSOG_ERR_INVALID_ARG (bad shape or NULL pointer) / OSOG_ERR_WORKSPACE /
 * OSOG_ERR_CUDA.
 */
#ifndef OSOG_CNN_H
#define OSOG_CNN_H

#include <stddef.h>
#include <stdint.h>

#include "osog.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t N, H, W, C;   /* input */
    int32_t K, R, S;      /* filters */
    int32_t stride, pad;
} osog_conv_shape_t;

/* Output height and width of a convolution (0 for an invalid shape). */
int32_t osog_conv_out_h(const osog_conv_shape_t *shape);
int32_t osog_conv_out_w(const osog_conv_shape_t *shape);

/* y = act(conv(x, w) + bias); relu = 1 applies max(0, .).  y is bf16 NHWC
 * [N][P][Q][K]; when y_f32 is not NULL the same values are also written as
 * fp32 (before rounding to bf16). */
int osog_conv2d_forward(const osog_conv_shape_t *shape, const uint16_t *x, const uint16_t *w,
                        const float *bias, int32_t relu, uint16_t *y, float *y_f32,
                        osog_stream_t stream);

/* dx = (d conv / dx)^T dy, then multiplied by the mask (x_act > 0) when
 * x_act is not NULL (the derivative of the ReLU that produced x).  dy is the
 * gradient at the convolution's output (after its own ReLU derivative).
 * w_t is a workspace of R*S*K*C bf16 holding the filters reordered to
 * [C][R][S][K] (filled by this call). */
int osog_conv2d_backward_data(const osog_conv_shape_t *shape, const uint16_t *dy,
                              const uint16_t *w, const uint16_t *x_act, uint16_t *dx,
                              uint16_t *w_t, osog_stream_t stream);

/* dw = sum over pixels of dy (x) and dbias = sum of dy, by a split
 * reduction over pixel chunks followed by a fixed-order sum.  ws must hold
 * osog_conv2d_backward_filter_workspace(shape) bytes. */
size_t osog_conv2d_backward_filter_workspace(const osog_conv_shape_t *shape);
int osog_conv2d_backward_filter(const osog_conv_shape_t *shape, const uint16_t *dy,
                                const uint16_t *x, float *dw, float *dbias, void *ws,
                                size_t ws_bytes, osog_stream_t stream);

/* Engine of osog_conv2d_forward, osog_conv2d_backward_data and
 * osog_conv2d_backward_filter for later
 * calls of this process: 1 (default) the fifth-generation tensor cores
 * (tcgen05.mma with the accumulator in tensor memory), 0 the warp-level
 * MMA (mma.sync).  Both compute the same products in BF16 with FP32
 * accumulation; summation order inside the tensor core differs.  With
 * tcgen05 selected, forward convolutions whose reduction R S C is below 128
 * and filter gradients with fewer than 128 output channels and fewer than
 * 64 filter entries R S C still run on the warp-level MMA (faster there);
 * filter gradients with fewer than 128 output channels but at least 64
 * filter entries take the filter entries as the tensor cores' rows.  The
 * switch also covers osog_conv2d_backward_filter. */
void osog_conv_use_tcgen05(int32_t enable);

/* Synchronise `stream` and report a latched device error of the
 * convolution kernels (OSOG_ERR_TIMEOUT: a bounded wait for the tensor
 * cores gave up; results of that call are invalid), clearing it. */
int osog_conv_sync_status(osog_stream_t stream);

/* Failure-detection test hook.  With polls > 0, every later tcgen05
 * convolution CTA also waits, for at most `polls` polls, on a barrier that
 * nothing arrives on: the wait runs out, the kernel latches the status that
 * osog_conv_sync_status reports as OSOG_ERR_TIMEOUT, still waits for its own
 * tensor-core work, releases its tensor memory and finishes (its results stay
 * valid).  polls <= 0 turns the hook off (the default).  Returns OSOG_OK or
 * OSOG_ERR_CUDA. */
int osog_conv_test_wait_limit(int32_t polls);

/* Derivative of a ReLU: dy_out[i] = dy[i] where act[i] > 0, else 0 (bf16). */
int osog_relu_backward(const uint16_t *dy, const uint16_t *act, uint16_t *dy_out, int64_t count,
                       osog_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* OSOG_CNN_H */
