/*
 * lbm_nn.h -- C ABI of the learned warm start (not in the paper).
 *
 * A small 3D convolutional network predicts an initial density and velocity
 * field from a geometry mask so that the lattice Boltzmann solve reaches its
 * steady state in fewer steps; the LBM residual alone still decides
 * convergence.  These entry points are the network's GPU kernels: 3x3x3
 * convolutions on tensor cores (BF16 operands, FP32 accumulation; tcgen05 or
 * mma.sync by shape) for the
 * forward pass and both backward passes, plus the pooling, upsampling,
 * concatenation, loss and optimiser steps of training.
 *
 * Conventions
 *   - Activations are channels-last BF16 (or FP32 where stated) tensors
 *     [n][z][y][x][c] with dims n, d (z), h (y), w (x) and c channels.
 *   - Convolution weights are BF16 [27][cin][cout] (tap = 9 dz + 3 dy + dx,
 *     offsets dz, dy, dx in 0..2 meaning -1, 0, +1), zero padding 1, stride 1.
 *   - Every pointer is a device pointer; `stream` is a cudaStream_t.  Calls are
 *     asynchronous.  Return LBM_OK (0) or LBM_ERR_ARG / LBM_ERR_CUDA (lbm.h);
 *     lbm_last_error() has the message.
 */
#ifndef LBM_NN_H
#define LBM_NN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* y[p][co] = act( sum_{tap,ci} wgt[tap][ci][co] * x[p + off(tap)][ci] + bias[co] ),
 * act = ReLU when relu != 0; bias may be NULL.  x[p + off] is zero outside the
 * box except along the axes set in `wrap` (bit 0 = x, bit 1 = y, bit 2 = z),
 * which are periodic.  Output BF16 (y) and/or FP32 (y32); either may be NULL.
 * Any cout (output channels are tiled over the grid).  The backward-data pass
 * is this same call on dy with the weights from lbm_nn_weight_flip and the
 * same `wrap`. */
int lbm_nn_conv3d(const void* x, int n, int d, int h, int w, int cin, const void* wgt,
                  const float* bias, int cout, int relu, int wrap, void* y, float* y32, void* stream);

/* lbm_nn_conv3d on the 5th-generation tensor cores (tcgen05), FP32
 * accumulator in tensor memory.  With cin % 16 == 0 a block computes up to
 * four bricks of 8 x 16 x 1 voxels stacked along z and the tensor cores read
 * the activations straight from a shared-memory halo tile (up to 64 input
 * channels at a time); with cin % 8 == 0 otherwise, an implicit GEMM gathers
 * them into a three-stage ring.  Same
 * arguments and results; needs cin % 8 == 0, cout % 16 == 0 and 16-byte
 * aligned x, wgt, y, y32 (else LBM_ERR_ARG).  lbm_nn_conv3d uses the halo-tile
 * kernel by itself whenever cin % 16 == 0 and cout % 16 == 0. */
int lbm_nn_conv3d_tc(const void* x, int n, int d, int h, int w, int cin, const void* wgt,
                     const float* bias, int cout, int relu, int wrap, void* y, float* y32, void* stream);

/* c[i][j] = sum_l a[i][l] * b[j][l] on the 5th-generation tensor cores
 * (tcgen05): a BF16 [m][k], b BF16 [n][k] (both with k contiguous), c FP32
 * [m][n], row-major, device memory.  Needs m % 128 == 0, n % 16 == 0 with
 * 16 <= n <= 256, k % 64 == 0 (else LBM_ERR_ARG).  Every wait inside the
 * kernel is bounded; a block whose wait ran out writes NaN over its rows and
 * counts itself (lbm_nn_tc_timeouts). */
int lbm_nn_gemm_bf16(const void* a, const void* b, float* c, int m, int n, int k, void* stream);

/* Launch shape of the halo-tile convolution for every later call in this
 * process: bricks_z bricks per block along z (1..4) and cout_tile output
 * channels per block (a multiple of 16 up to 128, with bricks_z * cout_tile
 * <= 512 when both are fixed); 0 leaves either chosen per shape (the default).
 * For tuning and tests; results do not depend on it.  LBM_ERR_ARG otherwise. */
int lbm_nn_conv_tune(int bricks_z, int cout_tile);

/* Number of tensor-core kernel blocks whose bounded waits ran out since the
 * last call (a device counter, read and cleared; synchronises the device). */
int lbm_nn_tc_timeouts(unsigned* count);

/* dx-ready weights: wt[tap][co][ci] = wgt[26 - tap][ci][co] (BF16). */
int lbm_nn_weight_flip(const void* wgt, int cin, int cout, void* wt, void* stream);

/* dw[tap][ci][co] += sum_p x[p + off(tap)][ci] * dy[p][co] (off and `wrap`
 * as in lbm_nn_conv3d) and, when dbias is not NULL, dbias[co] += sum_p
 * dy[p][co] (FP32 accumulators).  The voxels are split into chunks whose
 * partial sums are stored, then added to dw / dbias in chunk order: the
 * result is the same bits on every call (no atomics).  For 8 <= cin <= 256
 * the sums run on the tcgen05 tensor cores as one GEMM per tap over operands
 * packed channel-major; the packed operands and the partial sums live in
 * library-owned device buffers (grown on demand, kept for the process; calls
 * must not overlap on different streams).  Errors: LBM_ERR_ARG, LBM_ERR_OOM
 * (no room for the partial sums), LBM_ERR_CUDA. */
int lbm_nn_conv3d_wgrad(const void* x, const void* dy, int n, int d, int h, int w, int cin, int cout,
                        int wrap, float* dw, float* dbias, void* stream);

/* g[i] *= (act[i] > 0), over count BF16 values (ReLU backward in place). */
int lbm_nn_relu_mask(void* g, const void* act, size_t count, void* stream);

/* 2x2x2 average pooling (d, h, w even) and its adjoint. */
int lbm_nn_pool2(const void* x, int n, int d, int h, int w, int c, void* y, void* stream);
int lbm_nn_pool2_bwd(const void* dy, int n, int d, int h, int w, int c, void* dx, void* stream);

/* Nearest-neighbour upsampling by 2 (input dims given) and its adjoint. */
int lbm_nn_up2(const void* x, int n, int d, int h, int w, int c, void* y, void* stream);
int lbm_nn_up2_bwd(const void* dy, int n, int d, int h, int w, int c, void* dx, void* stream);

/* Channel concatenation y = [a | b] over `voxels` voxels, and its split. */
int lbm_nn_concat(const void* a, int ca, const void* b, int cb, size_t voxels, void* y, void* stream);
int lbm_nn_split(const void* y, int ca, int cb, size_t voxels, void* a, void* b, void* stream);

/* Masked mean-squared error of FP32 predictions against FP32 targets over
 * `voxels` voxels of c channels where mask[p] != 0 (`count` such voxels):
 * loss (device, 1 double, overwritten) and dpred = 2 (pred - target) mask /
 * (count * c) as BF16. */
int lbm_nn_mse(const float* pred, const float* target, const uint8_t* mask, size_t voxels, int c,
               size_t count, double* loss, void* dpred, void* stream);

/* One Adam step on FP32 master weights p with gradient g (then zeroed), moment
 * buffers m, v, writing the BF16 copy pb.  t is the step number (1-based). */
int lbm_nn_adam(float* p, float* g, float* m, float* v, void* pb, size_t count, float lr, float beta1,
                float beta2, float eps, int t, void* stream);

/* y = a + b over count BF16 values (y may alias a or b). */
int lbm_nn_add(const void* a, const void* b, size_t count, void* y, void* stream);

/* Network input from a geometry: x[v] = (mask[v] != 0, value) as two BF16
 * channels (value = the body-force channel, F / 1e-6). */
int lbm_nn_mask_input(const uint8_t* mask, size_t voxels, float value, void* x, void* stream);

/* Training target from steady moments (dense FP64 rho[v] and u[c][v] as
 * lbm_moments writes them): t[v] = ((rho - rho0) / s_rho, u_x / s_u, u_y / s_u,
 * u_z / s_u) in FP32; 0 where rho or u is not finite (solid nodes). */
int lbm_nn_fields_to_target(const double* rho, const double* u, size_t voxels, double rho0,
                            double s_rho, double s_u, float* t, void* stream);

/* The inverse: warm-start fields rho[v] = rho0 + s_rho t[v][0] and
 * u[c][v] = s_u t[v][1 + c] (FP64, the layout lbm_init reads). */
int lbm_nn_target_to_fields(const float* t, size_t voxels, double rho0, double s_rho, double s_u,
                            double* rho, double* u, void* stream);

/* Format conversions. */
int lbm_nn_f32_to_bf16(const float* x, size_t count, void* y, void* stream);
int lbm_nn_bf16_to_f32(const void* x, size_t count, float* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_NN_H */
