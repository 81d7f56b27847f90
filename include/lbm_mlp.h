/*
 * lbm_mlp.h -- C ABI of the surrogate network: a small multilayer
 * perceptron that maps the parameters of one reactive capillary run
 * (width, reaction rate, adhesion strength, viscosity ratio) to its
 * infiltration curve (front position at fixed times) and its pore-closure
 * time.  The paper has no such network; it is trained on trajectories of
 * the lattice Boltzmann solver of lbm.h, which stays the reference that
 * judges it and the fallback where it is not trusted.
 *
 * Network (all sizes fixed at create):
 *   h_1 = tanh(W_1 x + b_1),  h_l = tanh(W_l h_{l-1} + b_l)  (l = 2..L),
 *   y = W_{L+1} h_L + b_{L+1},
 * with n_in inputs, L hidden layers of n_hidden units, n_out outputs.
 * Every matrix product runs on the tensor cores with BF16 operands (the
 * weights and the activations rounded to BF16 where they enter a product)
 * and FP32 accumulation; biases, activations, gradients and the optimizer
 * state are FP32.  The FP32 master weights are the parameters the calls
 * below set and get; the BF16 copies follow them.
 *
 * Parameter vector layout (FP32, packed in this order):
 *   W_1 [n_hidden][n_in], b_1 [n_hidden],
 *   W_l [n_hidden][n_hidden], b_l [n_hidden]      for l = 2..L,
 *   W_{L+1} [n_out][n_hidden], b_{L+1} [n_out].
 * Matrices are row-major: W[j][i] multiplies input i into unit j.
 *
 * Training minimizes the mean squared error over the batch and the
 * outputs; target entries that are NaN are left out (they add nothing to
 * the loss or the gradient; the mean still divides by batch * n_out).
 * The optimizer is Adam (beta_1 = 0.9, beta_2 = 0.999, eps = 1e-8) with
 * bias correction.
 *
 * Memory: x, target, y and grad arguments are DEVICE pointers to FP32
 * arrays, row-major [batch][n_in], [batch][n_out], [batch][n_out] and
 * [param_count]; params passed to set/get are HOST arrays.  The handle
 * owns its weights, optimizer state and activation buffers (sized for
 * max_batch) until lbm_mlp_destroy.  Calls are asynchronous on the
 * handle's stream except those returning host data (get_params and the
 * loss of train_step / grad, when requested), which synchronize it.
 *
 * Errors: an lbm_status (lbm.h); the message is kept per handle
 * (lbm_mlp_last_error).  A handle is not thread-safe.
 */
#ifndef LBM_MLP_H
#define LBM_MLP_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_mlp lbm_mlp;

typedef struct {
    int32_t n_in;      /* inputs, 1..256 */
    int32_t n_hidden;  /* units per hidden layer, 16..1024, multiple of 16 */
    int32_t n_layers;  /* hidden layers L, 1..8 */
    int32_t n_out;     /* outputs, 1..1024 */
    int32_t max_batch; /* largest batch of any later call, >= 1 */
} lbm_mlp_shape;

/* Allocates a network; its parameters are zero until lbm_mlp_set_params.
 * EINVAL on a shape outside the ranges above, ENOMEM / ECUDA otherwise. */
lbm_status lbm_mlp_create(const lbm_mlp_shape *shape, lbm_mlp **out);

/* Number of FP32 parameters (the packed layout above); -1 on NULL. */
int64_t lbm_mlp_param_count(const lbm_mlp *h);

/* Copies n = param_count host values in as the master weights, refreshes
 * the BF16 copies and resets the optimizer (moments and step count). */
lbm_status lbm_mlp_set_params(lbm_mlp *h, const float *host, int64_t n);

/* Copies the n = param_count master weights out to the host. */
lbm_status lbm_mlp_get_params(lbm_mlp *h, float *host, int64_t n);

/* Binds a CUDA stream (cudaStream_t) for every later call; NULL selects
 * the handle's own non-blocking stream (cudaStreamLegacy selects the
 * legacy default stream).  Callers that produce inputs or consume outputs
 * on another stream bind that stream first. */
lbm_status lbm_mlp_set_stream(lbm_mlp *h, void *cuda_stream);

/* Inference: y = network(x) for `batch` rows (1 <= batch <= max_batch). */
lbm_status lbm_mlp_forward(lbm_mlp *h, const float *x, int32_t batch,
                           float *y);

/* Gradient of the loss at the current weights, written to grad (device,
 * packed like the parameters); loss (host, may be NULL) receives the
 * loss, which synchronizes the stream.  Weights are not changed. */
lbm_status lbm_mlp_grad(lbm_mlp *h, const float *x, const float *target,
                        int32_t batch, float *grad, double *loss);

/* One optimizer step: forward, backward and an Adam update with learning
 * rate lr > 0.  loss (host, may be NULL) receives the loss before the
 * update, which synchronizes the stream. */
lbm_status lbm_mlp_train_step(lbm_mlp *h, const float *x,
                              const float *target, int32_t batch, float lr,
                              double *loss);

/* Releases the handle and its device memory (NULL is a no-op). */
void lbm_mlp_destroy(lbm_mlp *h);

/* Message of the last failure on h, or of the last failed create when h
 * is NULL; never NULL. */
const char *lbm_mlp_last_error(const lbm_mlp *h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_MLP_H */
