/*
 * lbfe_mlp.h -- C ABI of the small multilayer perceptron that proposes the
 * critical-Capillary-number bracket of a droplet (the paper finds Ca_cr by
 * bracketing the largest stable and the smallest breaking wall velocity,
 * Sec. 3; the proposal only orders those full simulations, it never replaces
 * their verdict).
 *
 * Network: 6 inputs -> 128 -> 128 -> 128 -> 128 -> 4 outputs, GELU
 * (0.5 x (1 + erf(x / sqrt 2))) after each hidden layer, no activation on
 * the output.  Inputs are the scaled case descriptors (Ca, De, lambda,
 * 2R/W, L^2, viscoelastic phase); outputs are (steady D, theta / 90 deg,
 * break-up logit, neck count / 4).  The forward and backward kernels read
 * the weights in BF16 (weights_bf16 = 1) or FP32 and accumulate in FP32;
 * AdamW updates FP32 master weights and refreshes the BF16 copy.
 *
 * Parameter vector (FP32, lbfe_mlp_param_count() values): for each layer
 * l = 0..4 with sizes in -> out, the transposed weights Wt[in][out]
 * (Wt[i][o] multiplies input i into output o) followed by the bias b[out].
 *
 * Memory: as for the solver, the caller owns one device block of at least
 * lbfe_mlp_required_bytes(max_batch) bytes, 256-byte aligned, carved into
 * parameters, AdamW moments, gradients and activations; device inputs and
 * outputs are caller-owned device pointers; every call is enqueued on the
 * stream given at creation.  Calls return an lbfe_status (lbfe.h).
 */
#ifndef LBFE_MLP_H
#define LBFE_MLP_H

#include <stddef.h>

#include "lbfe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbfe_mlp lbfe_mlp;

/* Number of parameters (50,948). */
size_t lbfe_mlp_param_count(void);

/* Device bytes for batches of up to max_batch rows (1 <= max_batch <= 65536). */
lbfe_status lbfe_mlp_required_bytes(int max_batch, size_t *bytes);

/* Create a network in the caller's device block.  The parameters start at 0:
 * set them with lbfe_mlp_set_params.  weights_bf16 selects BF16 weights in
 * the forward and backward kernels (1) or FP32 (0). */
lbfe_status lbfe_mlp_create(lbfe_mlp **m, int max_batch, int weights_bf16, void *device_block, size_t bytes,
                            void *stream);

/* Copy the FP32 parameter vector in / out (host memory, param_count floats).
 * Setting the parameters also resets the AdamW moments and step counter. */
lbfe_status lbfe_mlp_set_params(lbfe_mlp *m, const float *host_params);
lbfe_status lbfe_mlp_get_params(lbfe_mlp *m, float *host_params);

/* y[batch][4] = network(x[batch][6]); x and y are device pointers. */
lbfe_status lbfe_mlp_forward(lbfe_mlp *m, const float *x_dev, int batch, float *y_dev);

/* Loss of a batch and its gradient with respect to the parameters (kept in
 * the network; read with lbfe_mlp_get_grads).  Targets t[batch][4] hold
 * (D, theta/90, broken in {0,1}, necks/4); the loss is the mean over the
 * batch of (y0-t0)^2 + (y1-t1)^2 + (y3-t3)^2 + BCE(sigmoid(y2), t2), with
 * the three squared terms multiplied by mask[batch] (0 drops a sample's
 * shape terms, e.g. after break-up).  loss_host may be NULL. */
lbfe_status lbfe_mlp_loss_grad(lbfe_mlp *m, const float *x_dev, const float *t_dev, const float *mask_dev,
                               int batch, float *loss_host);
lbfe_status lbfe_mlp_get_grads(lbfe_mlp *m, float *host_grads);

/* One AdamW step with the gradient of the last lbfe_mlp_loss_grad:
 * m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;  t += 1;
 * w -= lr (m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps) + wd w). */
lbfe_status lbfe_mlp_adamw(lbfe_mlp *m, float lr, float beta1, float beta2, float eps, float weight_decay);

lbfe_status lbfe_mlp_destroy(lbfe_mlp *m);

#ifdef __cplusplus
}
#endif

#endif /* LBFE_MLP_H */
