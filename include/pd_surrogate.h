/* libpd: learned surrogate for the restricted macro time derivative.
 *
 * The paper has no surrogate.  This part of the library replaces the
 * micro-burst of a patch (Section 3.3 (ii)-(iv)) by a small network that maps
 * 35 features of the patch to F = (U^1 - U^0)/tau (eq. (Time_Derivative)),
 * with an a-posteriori check against a one-micro-step burst and the full burst
 * as fallback.
 *
 * Network: 35 -> 256 -> 256 -> 256 -> 1, GELU in its tanh form
 *   g(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))),
 * (the first two hidden layers evaluate tanh with the hardware approximation,
 * absolute error of order 2^-11, below their BF16 output rounding),
 * BF16 weights and activations into the tensor cores (tcgen05), FP32
 * accumulation, FP32 master weights and Adam state.  Inputs are padded to 64
 * columns with zeros; a network input row holds 128 BF16 values: the high
 * parts hi = bf16(v) of the 64 standardised inputs v, then the low parts
 * bf16(v - hi), both multiplied by the same first-layer weights (so the
 * inputs reach the first product with 16 significant bits).  Flat FP32 parameter vector (PD_MLP_N_PARAM floats):
 *   W1[256][64], b1[256], W2[256][256], b2[256], W3[256][256], b3[256],
 *   w4[256], b4[1]   (row n of W_l holds the weights into unit n).
 *
 * Features of patch (i, j), in order:
 *   0..24  the 5x5 macro stencil U(i+p, j+q) (xi wraps on periodic grids and
 *          clamps otherwise, eta clamps) through the 1-D difference basis
 *          e0 = u0, e1 = (u1-u-1)/2, e2 = u1-2u0+u-1, e3 = (u2-2u1+2u-1-u-2)/2,
 *          e4 = u2-4u1+6u0-4u-1+u-2 in xi then eta, feature 5*q_ord + p_ord;
 *          term k >= 1 over s = max_k>=1 |term k|, term 0 as U00/(|U00| + s);
 *   25..28 2 alpha/(dxi^2 R) x2, 2 gamma/(deta^2 R) x10, nu/(dxi R) x1,
 *          omega/(deta R) x5 at the patch centre (metric term times the
 *          feature of the derivative it multiplies), R = 2 alpha/dxi^2 +
 *          2 gamma/deta^2 + |beta|/(dxi deta) + |nu|/dxi + |omega|/deta + |phi|;
 *   29..34 half the trace of the diffusion tensor at the centre, its relative
 *          change at the edge midpoints E, W, N, S, and tau R.
 * The network sees (x - mu)/sigma rounded to BF16 and predicts y/y_scale with
 * y = F/(R s).
 *
 * Residual check: F1 = restricted change of a one-micro-step burst / dt; the
 * prediction is kept when |F - F1| <= eps (|F1| + rms(F1)), rms over the
 * instance's patches; other patches take the full K-step burst.  After one
 * micro step from w = 0 the departure is the forcing, which is linear in the
 * interpolant's nine coefficients, so F1 is evaluated from a per-patch basis
 * of ten numbers built once from the burst records.
 *
 * All calls are asynchronous on the object's stream unless stated; errors
 * are pd_status codes, pd_mlp_last_error gives the message.
 */
#ifndef PD_SURROGATE_H
#define PD_SURROGATE_H

#include "pd.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PD_MLP_N_IN 35
#define PD_MLP_N_PAD 64
#define PD_MLP_IN_COLS 128
#define PD_MLP_WIDTH 256
#define PD_MLP_N_PARAM 148481

typedef struct pd_mlp pd_mlp;

/* Network on the current CUDA device, parameters zero, Adam state zero.
 * max_batch (a multiple of 128, <= 65536) bounds pd_mlp_gradient and the
 * training minibatch.  Errors: PD_EINVAL, PD_ENOMEM, PD_ECUDA. */
pd_status pd_mlp_create(int max_batch, void* cuda_stream, pd_mlp** out);
pd_status pd_mlp_destroy(pd_mlp* m);
pd_status pd_mlp_set_stream(pd_mlp* m, void* cuda_stream);

/* Copy the flat FP32 parameters from / to host memory (n == PD_MLP_N_PARAM).
 * Setting resets the Adam moments.  Synchronous. */
pd_status pd_mlp_set_params(pd_mlp* m, const float* theta_host, int n);
pd_status pd_mlp_get_params(pd_mlp* m, float* theta_host, int n);

/* Fan-in uniform initialisation on the device: every weight and bias of a
 * layer with fan-in f from U(-1/sqrt f, 1/sqrt f) (f = 35, then 256), W1's
 * padding columns zero; parameter i draws splitmix64(seed + (i+1) 0x9E3779B97F4A7C15)
 * / 2^64.  Resets the Adam moments. */
pd_status pd_mlp_init(pd_mlp* m, unsigned long long seed);

/* Feature standardisation mu[35], sigma[35] (sigma > 0) and the target scale.
 * Synchronous. */
pd_status pd_mlp_set_norm(pd_mlp* m, const float* mu_host, const float* sigma_host, float y_scale);
pd_status pd_mlp_get_norm(pd_mlp* m, float* mu_host, float* sigma_host, float* y_scale);

/* Fit mu, sigma (per feature, over n rows of raw FP32 features [n][35]) and
 * y_scale = mean |y| over n raw targets, on the device.  Synchronous. */
pd_status pd_mlp_fit_norm(pd_mlp* m, const float* X_raw_dev, const float* y_raw_dev, long long n);

/* Standardise raw features [n][35] into network input rows [n][128] (BF16
 * bit patterns: high parts, then low parts, padding zero) and, when y_raw_dev
 * is given, targets y/y_scale into t_dev (FP32). */
pd_status pd_mlp_pack(pd_mlp* m, const float* X_raw_dev, const float* y_raw_dev, long long n,
                      uint16_t* X_dev, float* t_dev);

/* Network output for n input rows X [n][128] (BF16) into y_dev[n] (FP32);
 * n = 0 does nothing (the pointers may then be NULL). */
pd_status pd_mlp_forward(pd_mlp* m, const uint16_t* X_dev, long long n, float* y_dev);

/* Gradient of the loss (1/n) sum (y - t)^2 over n <= max_batch rows with
 * respect to the flat parameters, into grad_dev[PD_MLP_N_PARAM] (FP32), and
 * the loss into *loss_host (synchronous when loss_host is given). */
pd_status pd_mlp_gradient(pd_mlp* m, const uint16_t* X_dev, const float* t_dev, int n,
                          float* grad_dev, float* loss_host);

/* Train with Adam (beta 0.9, 0.999, eps 1e-8) on n samples for `epochs`
 * epochs of minibatches of `batch` rows (a multiple of 128, <= max_batch):
 * the learning rate rises linearly over the first 5% of the steps to lr_max
 * and decays as a half cosine to zero; each epoch visits the samples in the
 * order (a k + b) mod n with seeded a coprime to n.  Writes the mean loss of
 * each epoch to loss_hist_host[epochs] when given.  Synchronous. */
pd_status pd_mlp_train(pd_mlp* m, const uint16_t* X_dev, const float* t_dev, long long n, int batch,
                       int epochs, float lr_max, unsigned long long seed, float* loss_hist_host);

/* One Adam step with the gradient currently held (after pd_mlp_gradient),
 * learning rate lr; the step counter advances by one. */
pd_status pd_mlp_adam_step(pd_mlp* m, float lr);

pd_status pd_mlp_sync(pd_mlp* m);
const char* pd_mlp_last_error(const pd_mlp* m);

/* ------------------------------------------------------------------------
 * The surrogate on a grid.  Grids of one instance with per-point coefficient
 * records (the default for one instance), m_xi == m_eta in {3,5,7,9,11} and
 * the lifted restriction (the default).  Work runs on the grid's stream; the
 * network runs there too. */
typedef struct pd_surrogate pd_surrogate;

/* Allocates the per-patch work buffers (about 190 bytes per patch) and
 * computes the features that do not depend on U.  Errors: PD_EINVAL (grid not
 * covered), PD_ESTATE (coefficients not set), PD_ENOMEM, PD_ECUDA. */
pd_status pd_surrogate_create(pd_grid* g, pd_mlp* m, pd_surrogate** out);
pd_status pd_surrogate_destroy(pd_surrogate* s);

/* Features of every patch for the field U: the network input rows
 * [n_patch][128] (BF16 bit patterns) and the output scale R s y_scale, and/or
 * the raw FP32 features [n_patch][35] and R s.  Any output may be NULL. */
pd_status pd_surrogate_features(pd_surrogate* s, const double* U_dev, uint16_t* X_dev, double* scale_dev,
                                float* X_raw_dev, double* Rs_dev);

/* Training targets y = F / (R s) of every patch from the plain patch solver:
 * F = restricted change after K micro steps from time t, divided by tau
 * (Section 3.3 (ii)-(v)); Rs_dev as written by pd_surrogate_features. */
pd_status pd_surrogate_targets(pd_surrogate* s, const double* U_dev, double t, const double* Rs_dev, float* y_dev);

/* Per patch: the network's F (F_hat_dev), the check estimate F1 from one
 * micro step (F1_dev) and the full-burst F (F_dev), at time t.  Any output
 * may be NULL. */
pd_status pd_surrogate_evaluate(pd_surrogate* s, const double* U_dev, double t, double* F_hat_dev, double* F1_dev,
                                double* F_dev);

/* n_macro macro steps of eq. (Extrapolation) from t0 with step dt_macro
 * (<= 0: the grid's suggested step) in which each patch's F comes from the
 * network when |F_hat - F1| <= eps (|F1| + rms F1) and from the full K-step
 * burst otherwise (eps < 0: every patch takes the burst). */
pd_status pd_surrogate_step(pd_surrogate* s, double* U_dev, double t0, double dt_macro, int n_macro, double eps);

/* The same macro steps without the network: every patch's F is the check's
 * estimate F1, the restricted change of a burst of one micro step over that
 * step (eq. (Time_Derivative) with tau = dt_micro; Section 4.1.1's Table 3
 * and Section 4.2's Table 6 show F insensitive to tau), evaluated in closed
 * form from the per-patch one-step basis.  The baseline that shows what the
 * network gains.  Errors: PD_EINVAL, PD_ECUDA. */
pd_status pd_surrogate_step_f1(pd_surrogate* s, double* U_dev, double t0, double dt_macro, int n_macro);

/* V = U + rel_sigma max|U| z on the interior nodes (boundary rows and, on
 * non-periodic grids, boundary columns copied): grid-scale perturbations for
 * training data.  z = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller) with
 * u1, u2 = (mix(seed + c 0x9E3779B97F4A7C15) >> 11 + 1/2) / 2^53, c = 2 node
 * and 2 node + 1, mix the splitmix64 finaliser.  V may alias U. */
pd_status pd_surrogate_perturb(pd_surrogate* s, const double* U_dev, double rel_sigma, unsigned long long seed,
                               double* V_dev);

/* Patch-steps taken by pd_surrogate_step and how many fell back to the burst
 * since creation.  Synchronous. */
pd_status pd_surrogate_counts(pd_surrogate* s, long long* patch_steps, long long* fallbacks);

#ifdef __cplusplus
}
#endif
#endif
