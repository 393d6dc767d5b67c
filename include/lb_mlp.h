/*
 * lb_mlp.h - surrogate network for the surface-tension sweep, trained and evaluated on
 * the GPU by the library's own kernels (part of the same shared library as lb.h).
 *
 * The paper tunes the surface tension with kappa (Eq. 18 source term; Eq. 22 gives
 * sigma = (1 - kappa) sigma_0 to leading order, and Table 2 shows where that law
 * departs from measurement). This network learns, from Laplace-law measurements of
 * batched droplet runs (lb_batch_measure), the map
 *     x = (T/T_c, kappa, tau_v)  ->  y = (sigma, rho_l, rho_v)
 * and inverts it to pick kappa for a target sigma at given T/T_c and tau_v, so that a
 * target surface tension needs no second Laplace sweep. The paper has no network; the
 * architecture is this library's.
 *
 * Network: 3 -> 64 -> 64 -> 3, GELU(z) = z Phi(z) = z/2 (1 + erf(z / sqrt 2)) on both
 * hidden layers, linear output. The inputs enter as the features
 * (ln(1 - T/T_c), ln(1 - kappa), tau_v), in which sigma ~ (1 - kappa)(1 - T/T_c)^p is
 * nearly linear, standardised with the data's means and scales; the outputs are learnt
 * as (log sigma, rho_l, log rho_v), standardised the same way.
 * Scale = population standard deviation, or 1 where that is no more than 1e-9 of the
 * mean's magnitude (a constant column). Inputs need T/T_c < 1 and kappa < 1.
 *
 * Precision: an FP32 master copy of the 4611 parameters is kept for Adam; forward and
 * backward use the weights rounded to BF16 (round to nearest even) and accumulate in
 * FP32. The gradient is taken with respect to the BF16 weights and applied to the FP32
 * master copy.
 *
 * Parameter vector (FP32, 4611 values, row-major out x in):
 *     W1[64][3], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]
 * Loss: mean over samples and outputs of the squared error in the standardised output
 * space. Adam (Kingma & Ba 2015) with bias correction; the step count starts at 0 at
 * lb_mlp_set_params and increases by one per training step.
 *
 * All host arrays are owned by the caller; functions that return data to the host
 * synchronise the network's stream. Status codes are those of lb.h; a network is not
 * poisoned by errors (every call validates its own arguments). Calls on one network are
 * not thread-safe.
 */
#ifndef PAPER_1306_6445_GB300_LB_MLP_H
#define PAPER_1306_6445_GB300_LB_MLP_H

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LB_MLP_IN 3
#define LB_MLP_HIDDEN 64
#define LB_MLP_OUT 3
#define LB_MLP_PARAMS 4611

typedef struct lb_mlp lb_mlp;

/* Means and scales of the inputs and of the transformed targets. */
typedef struct {
    float in_mean[3], in_scale[3], out_mean[3], out_scale[3];
} lb_mlp_norm;

/* Create a network able to hold up to max_samples training samples (1 <= max_samples
 * <= 1 << 20) on `stream` (a cudaStream_t; NULL = the legacy default stream). Parameters
 * start at zero and the normalisation at (0, 1). Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA. */
lb_status lb_mlp_create(lb_mlp **out, int max_samples, void *stream);

/* Copy LB_MLP_PARAMS host floats into the FP32 master copy (and its BF16 image); reset
 * the Adam moments and step count to zero. Errors: LB_EINVAL (NULL), LB_ECUDA. */
lb_status lb_mlp_set_params(lb_mlp *m, const float *params);
/* Copy the FP32 master parameters to the host (LB_MLP_PARAMS floats). */
lb_status lb_mlp_get_params(lb_mlp *m, float *params);

/* Training data from host arrays x[n][3] = (T/T_c, kappa, tau_v) and y[n][3] = (sigma,
 * rho_l, rho_v), 1 <= n <= max_samples, every y > 0, T/T_c < 1, kappa < 1. The
 * normalisation is computed on the device from these samples (FP64 sums) and the
 * standardised features and targets are kept resident for training. Errors: LB_EINVAL
 * (n out of range, NULL, a y <= 0, T/T_c or kappa >= 1, anything non-finite), LB_ECUDA. */
lb_status lb_mlp_set_data(lb_mlp *m, const float *x, const float *y, int n);

lb_status lb_mlp_get_norm(lb_mlp *m, lb_mlp_norm *out);
/* Replace the normalisation (for a network whose parameters were trained elsewhere).
 * Errors: LB_EINVAL if a scale is not positive and finite. */
lb_status lb_mlp_set_norm(lb_mlp *m, const lb_mlp_norm *norm);

/* Loss and gradient (with respect to the BF16 weights) over the resident training data
 * for the current parameters; grad may be NULL. Deterministic: fixed per-CTA sample
 * tiles, partial gradients summed in a fixed order. Errors: LB_EINVAL (no data). */
lb_status lb_mlp_loss_grad(lb_mlp *m, float *loss, float *grad);

/* Run `steps` >= 0 full-batch Adam steps (forward, backward, reduction + update: two
 * kernels per step, replayed from a captured CUDA graph in runs of 50) with learning
 * rate lr > 0 and beta1, beta2 in [0, 1), eps > 0. If loss is not NULL it receives the
 * loss of the last step's forward pass (before that step's update). Synchronises. */
lb_status lb_mlp_train(lb_mlp *m, int steps, float lr, float beta1, float beta2, float eps,
                       float *loss);

long long lb_mlp_steps_done(const lb_mlp *m);

/* Predictions y[n][3] = (sigma, rho_l, rho_v) for host inputs x[n][3], 0 <= n <= 1 << 22.
 * Errors: LB_EINVAL (also for T/T_c >= 1 or kappa >= 1), LB_ENOMEM, LB_ECUDA. */
lb_status lb_mlp_forward(lb_mlp *m, const float *x, float *y, int n);

/* For each query q[i] = (T/T_c, tau_v, sigma_target), bisection on kappa in
 * [kappa_lo, kappa_hi] (kappa_lo < kappa_hi < 1, T/T_c < 1) for predicted sigma =
 * sigma_target, using that sigma decreases with kappa (Eq. 22): 40 halvings, each one
 * forward pass on the GPU (one thread per query). kappa[i] receives the midpoint of the final bracket, or
 * NaN when the target lies outside [sigma(kappa_hi), sigma(kappa_lo)] as predicted.
 * 0 <= n <= 1 << 20. Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA. */
lb_status lb_mlp_invert_kappa(lb_mlp *m, const float *q, int n, float kappa_lo,
                              float kappa_hi, float *kappa);

const char *lb_mlp_last_error(const lb_mlp *m);
void lb_mlp_free(lb_mlp *m);

#ifdef __cplusplus
}
#endif

#endif
