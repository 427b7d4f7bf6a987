/* C ABI of the learned warm start of the FFT Lippmann-Schwinger solver.
 *
 * A small 3D convolutional network maps a phase image (indicator of phase 1)
 * and the stiffness contrast to an initial strain field eps^0, which is handed
 * to fftls_solve as opt->eps_init.  The solver still decides: the same
 * equilibrium criterion (eq. criterion of the paper) decides convergence, so a
 * poor prediction costs iterations, never accuracy.  The paper has no learned
 * component: every call below is an implementation feature of this library,
 * not a step of the paper's method.
 *
 * Conventions.  Activations are FP32, [batch][channel][n3][n2][n1] with n1
 * fastest; N = n1 n2 n3.  3D convolutions have stride 1, circular (periodic)
 * padding and odd kernel size k in {1, 3}; weights are [c_out][c_in][k][k][k]
 * (kx fastest), biases [c_out].  All pointers are device pointers on the
 * current CUDA device unless stated; `stream` is a cudaStream_t (NULL: default
 * stream).  Calls are asynchronous on `stream`.  Errors: FFTLS_E_INVALID_ARG for
 * null pointers or sizes out of range (nothing is launched),
 * FFTLS_E_CUDA when a launch fails.  The caller owns every buffer.
 */
#ifndef FFTLS_NN_H
#define FFTLS_NN_H

#include <stddef.h>
#include <stdint.h>

#include "fftls.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest channel count of a convolution (input or output). */
#define FFTLS_NN_MAX_CHANNELS 128

/* y = act(conv(x, w) + bias + skip): x [batch][c_in][N], y and skip (may be NULL)
 * [batch][c_out][N], w [c_out][c_in][k^3].  act = ReLU when relu = 1, identity
 * when 0.  y must not alias x. */
fftls_status fftls_nn_conv3d(const float* x, const float* w, const float* bias, const float* skip, float* y,
                             int batch, int c_in, int c_out, const int n[3], int ksize, int relu, void* stream);

/* Gradient with respect to the input of fftls_nn_conv3d: dx = conv^T(dy, w)
 * (accumulate = 0) or dx += conv^T(dy, w) (accumulate = 1); dy is the gradient
 * with respect to the pre-activation output, [batch][c_out][N]; dx [batch][c_in][N]. */
fftls_status fftls_nn_conv3d_backward_data(const float* dy, const float* w, float* dx, int batch, int c_in, int c_out,
                                           const int n[3], int ksize, int accumulate, void* stream);

/* Gradients with respect to the weights and bias: dw[o][i][k] = sum over batch
 * and voxels of dy[o](v) x[i](v + offset(k)), db[o] = sum of dy[o].  Written
 * (not accumulated).  scratch: at least fftls_nn_wgrad_scratch(...) floats of
 * device memory for the deterministic two-stage reduction. */
fftls_status fftls_nn_conv3d_backward_weights(const float* x, const float* dy, float* dw, float* db, int batch,
                                              int c_in, int c_out, const int n[3], int ksize, float* scratch,
                                              size_t scratch_floats, void* stream);
size_t fftls_nn_wgrad_scratch(int batch, int c_in, int c_out, const int n[3], int ksize);

/* dy[i] = y[i] > 0 ? dy[i] : 0 (backward of a ReLU whose output is y), count values. */
fftls_status fftls_nn_relu_backward(float* dy, const float* y, long long count, void* stream);

/* 2x2x2 mean pooling: x [planes][n3][n2][n1] -> y [planes][n3/2][n2/2][n1/2]
 * (n even); planes = batch * channels.  Backward: dx (=|+=) dy / 8 spread over
 * each 2x2x2 block. */
fftls_status fftls_nn_pool2(const float* x, float* y, int planes, const int n[3], void* stream);
fftls_status fftls_nn_pool2_backward(const float* dy, float* dx, int planes, const int n[3], int accumulate,
                                     void* stream);

/* Nearest-neighbour 2x upsampling: x [planes][nc3][nc2][nc1] -> y [planes][2nc3][2nc2][2nc1]
 * (nc = coarse sizes).  Backward: dx = sum of dy over each 2x2x2 block (written). */
fftls_status fftls_nn_upsample2(const float* x, float* y, int planes, const int nc[3], void* stream);
fftls_status fftls_nn_upsample2_backward(const float* dy, float* dx, int planes, const int nc[3], void* stream);

/* y += x, count values. */
fftls_status fftls_nn_add(float* y, const float* x, long long count, void* stream);

/* Mean squared error over count values: *loss (device double) = mean((y - t)^2),
 * dy = 2 (y - t) / count. */
fftls_status fftls_nn_mse(const float* y, const float* t, float* dy, double* loss, long long count, void* stream);

/* One Adam step (Kingma and Ba 2015) on count parameters with bias-corrected
 * moments: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps); step >= 1. */
fftls_status fftls_nn_adam(float* p, const float* g, float* m, float* v, long long count, float lr, float beta1,
                           float beta2, float eps, int step, void* stream);

/* Network input from a phase image (uint8 ids, N voxels, device): channel 0 =
 * indicator of phase 1, channel 1 = log_contrast everywhere; x [2][N]. */
fftls_status fftls_nn_features(const uint8_t* phase, float* x, const int n[3], float log_contrast, void* stream);

/* Initial strain from a network output y [6][N] (components 11,22,33,23,13,12 of
 * the fluctuation for the unit load eps_bar = e1 (x) e1): eps [6][N] FP64 =
 * eps_bar + scale * (y - <y>).  The component means are compensated FP32 sums
 * combined in FP64; the fluctuation scale * (y - <y>) is formed in FP32 (this is
 * an initial guess) and widened exactly, so <eps> = eps_bar up to FP32
 * rounding of the fluctuation.  scratch: FFTLS_NN_STRAIN_SCRATCH doubles of
 * device memory (partial sums). */
#define FFTLS_NN_STRAIN_SCRATCH 1536
fftls_status fftls_nn_strain_init(const float* y, double* eps, const int n[3], const double eps_bar[6], double scale,
                                  double* scratch, void* stream);

/* Training target from a solved strain field: t [6][N] (FP32) = eps - eps_bar,
 * eps [6][N] FP64 (device). */
fftls_status fftls_nn_strain_target(const double* eps, float* t, const int n[3], const double eps_bar[6], void* stream);

/* ---- Tensor-core path: BF16 operands, FP32 accumulation, channels-last BF16 activations ----
 *
 * An activation with c channels is stored channels-last, [batch][n3][n2][n1][cs],
 * in BF16 with cs = 8, 16, 32 or 64 (the smallest of these >= c; channels c..cs-1
 * zero).  Device pointers must be 16-byte aligned.  The convolutions are the
 * same periodic convolutions as fftls_nn_conv3d, with the input and the weights
 * rounded to BF16 and FP32 accumulation. */

/* Bytes of the packed weights of a layer with w [c_out][c_in][k^3] (1 <= c_in, c_out <= 64,
 * k = 1 or 3): transposed = 0 for the convolution x (c_in channels) -> y (c_out), 1 for the
 * input gradient dy (c_out channels) -> dx (c_in).  0 for invalid arguments. */
size_t fftls_nn_tc_packed_bytes(int c_in, int c_out, int ksize, int transposed);

/* Round w (FP32 device) to BF16 and lay it out as the tensor-core operand of
 * fftls_nn_tc_conv3d; packed: fftls_nn_tc_packed_bytes(...) bytes of device memory. */
fftls_status fftls_nn_tc_pack(const float* w, void* packed, int c_in, int c_out, int ksize, int transposed,
                              void* stream);

/* y = act(conv(x', W) + bias + skip) (+ y when accumulate = 1) on the output grid n, where W comes
 * from fftls_nn_tc_pack for (c_in, c_out) = the channels of x and y here (for transposed packing:
 * the layer's c_out and c_in), and x' is, by in_mode:
 *   0: x itself, on the grid n;
 *   1: the nearest-neighbour 2x upsampling of x, x on the grid n/2 (n even);
 *   2: the 2x2x2 mean pooling of x, x on the grid 2n (the mean rounded to BF16).
 * x, skip (may be NULL) and y (when out_planar = 0) are channels-last BF16; with out_planar = 1,
 * y is FP32 [batch][c_out][N] instead.  act = ReLU when relu = 1.  y must not alias x or skip.
 * Returns FFTLS_E_UNSUPPORTED_SIZE when no voxel tile fits in shared memory. */
fftls_status fftls_nn_tc_conv3d(const void* x, const void* packed, const float* bias, const void* skip, void* y,
                                int batch, int c_in, int c_out, const int n[3], int ksize, int in_mode, int relu,
                                int out_planar, int accumulate, void* stream);

/* First layer from the phase image (uint8 ids, [n3][n2][n1], device): y = act(conv(x, w) + bias)
 * for the two-channel input x of fftls_nn_features (indicator of phase 1, log_contrast), w FP32
 * [c_out][2][27], c_out <= 8, computed in FP32 from the phase bytes; y channels-last BF16
 * (8 stored channels). */
fftls_status fftls_nn_tc_conv_phase(const uint8_t* phase, const float* w, const float* bias, void* y, const int n[3],
                                    int c_out, float log_contrast, int relu, void* stream);

/* ---- Tensor-core training pieces (same layouts as above) ---- */

/* Scratch floats of fftls_nn_tc_conv3d_backward_weights (0 for invalid arguments). */
size_t fftls_nn_tc_wgrad_scratch(int batch, int c_in, int c_out, const int n[3], int ksize);

/* Weight and bias gradients of fftls_nn_tc_conv3d on the tensor cores: dw[o][i][k] = sum over the
 * batch and the output voxels v of dy(v)[o] x'(v + offset(k))[i] and db[o] = sum of dy(v)[o] (db may be
 * NULL), FP32 [c_out][c_in][k^3], written.  x: the layer input (channels-last BF16, c_in channels) on
 * the grid in_mode gives (as in fftls_nn_tc_conv3d: 0 the grid n, 1 n/2 upsampled, 2 2n pooled); dy:
 * the gradient at the layer output before its activation, channels-last BF16 on the grid n.  Products
 * of BF16 values accumulated in FP32 per voxel tile, the tiles summed in a fixed order in FP64.
 * scratch: at least fftls_nn_tc_wgrad_scratch(...) floats of device memory. */
fftls_status fftls_nn_tc_conv3d_backward_weights(const void* x, const void* dy, float* dw, float* db, int batch,
                                                 int c_in, int c_out, const int n[3], int ksize, int in_mode,
                                                 float* scratch, size_t scratch_floats, void* stream);

/* Scratch floats of fftls_nn_tc_conv_phase_backward_weights. */
size_t fftls_nn_tc_phase_wgrad_scratch(const int n[3]);

/* Weight and bias gradients of fftls_nn_tc_conv_phase (one sample): dw [c_out][2][27] FP32 (channel 0:
 * sums of dy(v)[o] over the voxels whose neighbour at offset k is phase 1; channel 1: log_contrast
 * times the sum of dy(v)[o], the constant input channel), db [c_out] (may be NULL), written; dy
 * channels-last BF16 with 8 stored channels. */
fftls_status fftls_nn_tc_conv_phase_backward_weights(const uint8_t* phase, const void* dy, float* dw, float* db,
                                                     const int n[3], int c_out, float log_contrast, float* scratch,
                                                     size_t scratch_floats, void* stream);

/* Channels-last BF16 y [batch][voxels][cs] from planar FP32 x [batch][channels][voxels] (channels <= 64,
 * cs the stored channel count, the padding channels zero). */
fftls_status fftls_nn_tc_from_planar(const float* x, void* y, int batch, int channels, long long voxels, void* stream);

/* Channels-last BF16 elementwise pieces of the backward pass; count = values (a multiple of 8):
 * dy = y > 0 ? dy : 0 (ReLU backward, y the activation); y += x. */
fftls_status fftls_nn_tc_relu_backward(void* dy, const void* y, long long count, void* stream);
fftls_status fftls_nn_tc_add(void* y, const void* x, long long count, void* stream);

/* Adjoints of the 2x resampling on channels-last BF16 (nc = the coarse grid): upsampling's, dx on nc =
 * the sum of dy (grid 2 nc) over each 2x2x2 block (written); mean pooling's, dx on 2 nc (=|+=) dy (grid
 * nc) / 8 spread over each block. */
fftls_status fftls_nn_tc_upsample2_backward(const void* dy, void* dx, int batch, int channels, const int nc[3],
                                            void* stream);
fftls_status fftls_nn_tc_pool2_backward(const void* dy, void* dx, int batch, int channels, const int nc[3],
                                        int accumulate, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FFTLS_NN_H */
