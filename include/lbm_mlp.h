/* lbm_mlp.h - learned thermodynamic closure of the non-ideal lattice Boltzmann
 * solver (include/lbm.h).
 *
 * The solver's closure maps the node state (rho, e), e the specific internal
 * energy, to temperature, pressure and squared sound speed; for the van der
 * Waals fluid these are Eqs. lbm_temp, Pvdw and vdW_speed_of_sound of Sec. 2
 * and Sec. 3.2 (T from e by the caloric relation, P from the EOS, c_s^2 in
 * the bulk-viscosity correction alpha of Eq. corr_bulk).  This interface
 * trains a 2 -> 64 -> 64 -> 3 multilayer perceptron (tanh-form GELU, bfloat16
 * weights, FP32 biases and accumulation) to stand in for that closure:
 *
 *   x = ((rho - c_rho)/s_rho, (e - c_e)/s_e)
 *   y = W3 gelu(W2 gelu(W1 x + b1) + b2) + b3
 *   T = m_T + r_T y0,  P = m_P + r_P y1,  c_s^2 = m_c + r_c y2
 *
 * Training data are (rho, e) states the solver itself produced
 * (lbm_mlp_collect); labels are the exact closure, evaluated in FP64 on the
 * GPU.  Training runs on the GPU: minibatch assembly, forward and backward
 * passes (the 64 x 64 contractions on the tensor cores, BF16 x BF16 -> FP32),
 * fixed-order gradient reduction and AdamW, all in this library's kernels.
 *
 * Once attached to an FP32 solver handle (lbm_mlp_attach) the network is
 * evaluated inside the fused step for every node whose normalised input lies
 * in the training box |x0| <= 1, |x1| <= 1; other nodes use the exact closure
 * (range gate).  The exact closure remains the reference: lbm_moments reports
 * T from the exact caloric relation whatever the closure of the step.
 *
 * Conventions: as include/lbm.h.  "device" pointers are CUDA device memory
 * of the current device, "host" pointers are ordinary host memory.  Every
 * call returns LBM_OK or an LBM_E* code with a message in
 * lbm_mlp_last_error().  Calls are synchronous unless stated otherwise.
 * Parameter vectors are FP32, NPARAM = 4547 values in the order W1 (64 x 2),
 * b1 (64), W2 (64 x 64), b2 (64), W3 (3 x 64), b3 (3), matrices row-major
 * [out][in].
 */
#ifndef LBM_MLP_H
#define LBM_MLP_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MLP_HIDDEN 64
#define LBM_MLP_NPARAM 4547
#define LBM_MLP_NSCALE 10

typedef struct lbm_mlp_s* lbm_mlp_t;

/* New network for the van der Waals closure with constants a, b, R, c_v in
 * the units of the data it will see.  Weights start uniform in
 * +-sqrt(6 / (fan_in + fan_out)) from the SplitMix64 stream `seed` (value k
 * of the stream mapped to [-1, 1) as in the input generators), biases zero;
 * the scaling is unset (lbm_mlp_fit_scaling or lbm_mlp_set_scaling). */
int lbm_mlp_create(lbm_mlp_t* out, double a, double b, double R, double cv, uint64_t seed);

/* Stream for the asynchronous parts of the calls (NULL = legacy default). */
int lbm_mlp_set_stream(lbm_mlp_t net, void* stream);

/* Append the current state of solver `h` as Nx*Ny*Nz samples: d_rho[k] =
 * rho, d_e[k] = e_scale * (c_v T - a rho) for the interior nodes in node
 * order, at offsets 0 .. Nx*Ny*Nz - 1 of the two device arrays (the caller
 * offsets the pointers).  e_scale converts the solver's lattice energy to the
 * units of the network (the ratio of the velocity scales squared when the
 * solver runs in other lattice units).  Enqueued on the solver's stream. */
int lbm_mlp_collect(lbm_t h, double* d_rho, double* d_e, double e_scale);

/* Set the input box and output normalisation from n device samples: c and s
 * are the midpoints and half-widths of the sample ranges of rho and e, m and
 * r those of the exact T, P, c_s^2 over the samples. */
int lbm_mlp_fit_scaling(lbm_mlp_t net, const double* d_rho, const double* d_e, long long n);

/* Read / write the 10 scaling constants (host): c_rho, s_rho, c_e, s_e,
 * m_T, r_T, m_P, r_P, m_c, r_c (every s and r > 0). */
int lbm_mlp_get_scaling(lbm_mlp_t net, double* scale);
int lbm_mlp_set_scaling(lbm_mlp_t net, const double* scale);

/* Read / write the FP32 master parameters (host, NPARAM values).  Setting
 * them resets the AdamW state. */
int lbm_mlp_get_params(lbm_mlp_t net, float* theta);
int lbm_mlp_set_params(lbm_mlp_t net, const float* theta);

/* Loss and gradient of the current network on n given samples: x (host,
 * n x 2 normalised inputs), y (host, n x 3 normalised targets).  loss = mean
 * squared error over n x 3 outputs; grad (host, NPARAM) is its gradient with
 * respect to the parameters, the forward pass taken with bfloat16-rounded
 * weights (the gradient of the rounded weights is that of the FP32 master
 * weights).  1 <= n <= 2^20. */
int lbm_mlp_loss_grad(lbm_mlp_t net, const float* x, const float* y, int n, double* loss, float* grad);

/* Contraction path of the training kernels.  LBM_MLP_MMA_TCGEN05 (the
 * default): one kernel takes the minibatch through forward pass, backward
 * pass and all weight gradients on the fifth-generation tensor cores
 * (tcgen05.mma, BF16 x BF16 -> FP32 accumulators in tensor memory, groups of
 * 128 samples), every FP32 operand split into two bfloat16 terms, so all
 * gradients are at the FP32 level.  LBM_MLP_MMA_WARP: warp-level mma.sync
 * m16n8k16 for the 64 x 64 products, with dL/dz2 rounded to bfloat16 in dW2
 * and in the input gradient of layer 2 (relative error about 1e-3 there).
 * A tensor-core completion wait that runs out makes lbm_mlp_loss_grad and
 * lbm_mlp_train return LBM_ECUDA.
 * Errors: LBM_EINVAL (NULL network, unknown kind). */
#define LBM_MLP_MMA_WARP 0
#define LBM_MLP_MMA_TCGEN05 1
int lbm_mlp_set_mma(lbm_mlp_t net, int kind);
/* The contraction path in use (LBM_MLP_MMA_*). */
int lbm_mlp_get_mma(lbm_mlp_t net);

/* `steps` AdamW steps (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight
 * decay wd) on minibatches of `batch` samples drawn uniformly with
 * replacement from the n device samples (d_rho, d_e), index k of step t from
 * SplitMix64 stream `seed`; the learning rate falls from lr0 to lr1 along a
 * half cosine over the call.  losses (host, `steps` values, may be NULL):
 * minibatch loss before each step.  Needs the scaling set.
 * 32 <= batch <= 2^20. */
int lbm_mlp_train(lbm_mlp_t net, const double* d_rho, const double* d_e, long long n, int batch, int steps,
                  double lr0, double lr1, double wd, uint64_t seed, float* losses);

/* The closure as the fused step evaluates it, for n device samples:
 * d_out[4k .. 4k+3] = T, P, c_s^2 and 1 if the network was used (the sample
 * is inside the box) else 0 (exact van der Waals values). */
int lbm_mlp_predict(lbm_mlp_t net, const double* d_rho, const double* d_e, long long n, double* d_out);

/* Use the network as the closure of solver `h` (FP32 storage, fused step):
 * a snapshot of the current weights and scaling is copied to the handle, so
 * later training does not change it until the next attach.  net = NULL goes
 * back to the exact closure.  The handle's units must be those of the
 * network's data. */
int lbm_mlp_attach(lbm_t h, lbm_mlp_t net);

/* Closure in use by `h`: LBM_CLOSURE_EXACT or LBM_CLOSURE_MLP. */
int lbm_get_closure(lbm_t h);

int lbm_mlp_destroy(lbm_mlp_t net);
const char* lbm_mlp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_MLP_H */
