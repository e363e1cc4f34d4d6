/*
 * sde_mlp.h -- C ABI of the surrogate network of the GB300 engine.
 *
 * The paper has no surrogate; this is the learned screening part of the
 * engine's parameter scans.  A multilayer perceptron 7 -> 256 -> 256 -> 256 -> 2
 * maps the seven model parameters of a point (gamma, a, omega, F, Q and the
 * two parameters of the jump noise) to (<v>, log stderr) of its Monte Carlo
 * estimate (Eq. 31).  Hidden layers use SiLU, x sigmoid(x).  Weights and
 * activations are BF16, every product is accumulated in FP32 on the tensor
 * cores, the master weights and the Adam moments are FP32.  All arithmetic of
 * forward, backward and Adam runs in the library's own CUDA kernels.
 *
 * Parameter vector (FP32, padded for the tensor-core tiles; the padding stays
 * zero): W1[256][16] (input 7 padded to 16), b1[256], W2[256][256], b2[256],
 * W3[256][256], b3[256], W4[8][256] (output 2 padded to 8), b4[8];
 * SDE_MLP_NPARAMS = 137992 floats (134146 of them live).
 *
 * Inputs are raw parameters (M x 7, row-major FP32); the network applies its
 * input map x' = (g(x) - shift) * scale with g = log10 where the log mask bit
 * is set.  Outputs are de-standardised: y = y' * out_scale + out_shift.  The
 * training targets are given raw in the same units as the outputs.
 *
 * Errors: 0 on success, negative SDE_E* codes of sde.h; sde_mlp_last_error().
 */
#ifndef SDE_MLP_H
#define SDE_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SDE_MLP_IN 7
#define SDE_MLP_HIDDEN 256
#define SDE_MLP_OUT 2
#define SDE_MLP_NPARAMS 137992u

typedef struct sde_mlp sde_mlp;

/* Create a network on the current device, bound to `cuda_stream` (borrowed;
 * NULL = a stream of its own).  Weights: Glorot-uniform from `seed`, biases
 * zero, identity input and output maps. */
int sde_mlp_create(sde_mlp** out, uint64_t seed, void* cuda_stream);

/* Input map: shift[7], scale[7] (host arrays) and the log10 mask (bit i:
 * feature i enters as log10(x_i)).  Output map: out_shift[2], out_scale[2]. */
int sde_mlp_set_maps(sde_mlp* net, const float* shift, const float* scale, uint32_t log_mask,
                     const float* out_shift, const float* out_scale);

/* Copy the FP32 master parameters from / to the host (SDE_MLP_NPARAMS floats).
 * Setting them also refreshes the BF16 copies and zeroes the Adam state. */
int sde_mlp_set_params(sde_mlp* net, const float* host_params);
int sde_mlp_get_params(sde_mlp* net, float* host_params);

/* Forward pass: x (device, M x 7 FP32 raw inputs) -> y (device, M x 2 FP32).
 * Any M >= 1; large M runs in chunks (2^20 rows on the tcgen05 path, 65536
 * on the mma.sync path).  Asynchronous. */
int sde_mlp_forward(sde_mlp* net, const float* x, uint64_t M, float* y);

/* Gradients of the mean squared error of the standardised outputs,
 * L = 1/(2M) sum_m sum_o (y'_mo - t'_mo)^2, with respect to the FP32 master
 * parameters (host array of SDE_MLP_NPARAMS floats) and the loss (host).
 * M <= 65536.  Synchronises the stream. */
int sde_mlp_gradients(sde_mlp* net, const float* x, const float* t, uint64_t M,
                      float* host_grad, double* host_loss);

/* One Adam step (beta1, beta2, eps, learning rate lr) on the batch (x, t) of
 * M <= 65536 rows (device arrays).  loss_dev (device float or NULL) receives
 * the batch loss before the step.  Asynchronous. */
int sde_mlp_train_step(sde_mlp* net, const float* x, const float* t, uint64_t M, float lr,
                       float beta1, float beta2, float eps, float* loss_dev);

/* Adam training on the device: `steps` steps on minibatches of `batch` rows
 * of the labels X (device, N x 7 FP32 raw inputs) and T (device, N x 2 FP32
 * targets), the loss of sde_mlp_gradients.  Rows are visited in epochs of
 * N / batch whole minibatches, each epoch in a fresh order: a bijection of
 * [0, N) keyed by (seed, epoch), a four-round Feistel network with cycle
 * walking.  The learning rate decays from lr to lr_final along a half cosine,
 * lr_k = lr_final + (lr - lr_final)(1 + cos(pi k / (steps - 1))) / 2; Adam's
 * bias corrections continue the network's step count (earlier
 * sde_mlp_train_step or sde_mlp_fit calls).  losses (device, `steps` floats,
 * or NULL) receives each step's minibatch loss before its update.  One step is
 * captured as a CUDA graph on a private stream and replayed, ordered after
 * the work already on the network's stream; returns when the steps are done.
 * Requires 1 <= batch <= min(N, 65536), N <= 2^30, 1 <= steps <= 2^22 (else
 * SDE_EINVAL); the step schedule takes 12 bytes per step on the host and the
 * device for the duration of the call.  No other call may use the same
 * network meanwhile (the capture runs the network's kernels on the private
 * stream). */
int sde_mlp_fit(sde_mlp* net, const float* X, const float* T, uint64_t N, uint64_t steps,
                uint32_t batch, float lr, float lr_final, float beta1, float beta2, float eps,
                uint64_t seed, float* losses);

/* Matrix path of the forward pass: 1 (default) two fused kernels on the
 * fifth-generation tensor cores (input map and layers 1-2; layers 3-4 and
 * the output map; tcgen05.mma with FP32 accumulators in tensor memory,
 * persistent CTAs holding a 256 x 256 layer's weights in shared memory, SiLU
 * through tanh), 0 the layer-by-layer warp-level mma.sync kernels that also
 * serve training.  Results agree within the BF16 rounding of the
 * activations. */
int sde_mlp_set_tensor_path(sde_mlp* net, int use_tcgen05);

/* Wait for the network's stream and report device-side failures: SDE_ETIMEDOUT
 * if a tensor-core completion wait ran out of its iteration limit. */
int sde_mlp_sync(sde_mlp* net);

/* Building block exposed for tests: C[M][N] (FP32, device) = op(A) op(B) with
 * BF16 operands on the tensor cores.  a_layout 0: A is [M][K] row-major,
 * 1: A is [K][M]; b_layout 0: B is given as [N][K] (row n holds column n of
 * B), 1: B is [K][N].  Leading dimensions are the row lengths of the stored
 * arrays.  Synchronises the stream. */
int sde_mlp_gemm_bf16(sde_mlp* net, int a_layout, int b_layout, uint32_t M, uint32_t N,
                      uint32_t K, const void* A, uint32_t lda, const void* B, uint32_t ldb,
                      float* C, uint32_t ldc);

/* Selection step of the surrogate-guided scan over an nx x ny grid (row-major,
 * index i * ny + j; all arrays device).  v1, v2: <v> predicted by two
 * independently trained networks; lse: their mean log10 stderr of the Monte
 * Carlo label; se_scale: factor from the label's path count to the re-run's
 * (sqrt(N_label / N_rerun)).  Point p is flagged (flags[p] = 1) when
 *   - its predicted model error kappa |v1 - v2| + r0 exceeds tol, or
 *   - its predicted Monte Carlo stderr se_scale 10^lse exceeds se_tol, or
 *   - the sign of (v1 + v2) / 2 differs from that of a grid 4-neighbour.
 * `count` (device u32, accumulated) receives the number of flagged points.
 * Asynchronous on the network's stream. */
int sde_guided_flags(sde_mlp* net, const float* v1, const float* v2, const float* lse,
                     uint32_t nx, uint32_t ny, float kappa, float r0, float se_scale, float tol,
                     float se_tol, uint8_t* flags, uint32_t* count);

void sde_mlp_destroy(sde_mlp* net);
const char* sde_mlp_last_error(const sde_mlp* net);

#ifdef __cplusplus
}
#endif
#endif
