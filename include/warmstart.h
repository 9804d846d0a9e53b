/* warmstart.h — learned warm start for ASPOT.
 *
 * The paper has no counterpart: this is an addition.  Lemma 2 bounds ASPOT's
 * dual gap by a constant times |z* - z~0|^2 / t^2 and Algorithm 2 starts from
 * the zero dual point; a start closer to z* shortens the run.  A small network
 * predicts the dual u_i of every row point and v_j of every column point of a
 * squared-Euclidean problem; uniform shifts of u, v and w then follow from
 * one exact minimisation of phi along them (it includes the w-step
 * |B(u, v, w)|_1 = s), and aspot_solve with POT_FLAG_WARM_CHECK keeps the
 * zero start whenever E(z_warm) > E(0) (E = |grad phi|_1 of Algorithm 2).
 *
 * The network's output y is gamma log K (see pot_ws_targets), and the start
 * is u_i = log r_i - softplus(y_i / gamma), v_j = log c_j - softplus(y_j / gamma).
 *
 * Network (H = POT_WS_HIDDEN = 128, F = d + 5 inputs per point):
 *   a1 = W1 x + b1,  h1 = GELU(a1)                       per point
 *   ctx_k = mean of h1 over the points of instance k     (both clouds)
 *   q_k = U [ctx_k; |r|_1/s; |c|_1/s]
 *   a2 = W2 h1 + q_k + b2,  h2 = GELU(a2),  y = w3 . h2 + b3
 * with GELU(a) = a Phi(a) (erf form).  Per-point features x (F floats):
 *   (point - mean of all n + m points) * sqrt(cost_scale)   d values
 *   n r_i / |r|_1  (rows)  or  m c_j / |c|_1  (columns)
 *   +1 (rows) or -1 (columns)
 *   T log sum_j (c_j / |c|_1) exp(-C_ij / T), T = gamma, 4 gamma, 16 gamma
 *                                                  (rows; columns: with r)
 * where cost_scale is the problem's (1 / max |x - y|^2 when it is 0) and C
 * the scaled cost.  The last three features, soft minima of a point's cost
 * to the other cloud's mass, are c-transforms of the normalised log-masses:
 * at the optimum u_i of a transported row point is such a soft minimum at
 * temperature gamma (of v instead of log c), so the network learns a
 * correction to it; the higher temperatures show the mass around the point
 * at larger scales.  Each costs one pass over the cost (pot_marginals).
 * Training minimises the weighted mean squared error
 *   L = (1/N) sum_p omega_p (y_p - target_p)^2
 * over the N points of a batch, against the targets of converged ASPOT runs
 * (pot_ws_targets), with Adam.  The weight omega = sigmoid(log K)^2 (the
 * squared transported fraction of the point) is the factor by which an
 * output error reaches the duals (du_i = sigmoid(y_i / gamma) dy_i / gamma), so
 * L measures the start's distance to z*, the constant of Lemma 2.
 *
 * Parameters are one FP32 device array (pot_ws_param_count floats), row-major:
 *   W1[H][F], b1[H], W2[H][H], U[H][H+2], b2[H], w3[H], b3[1].
 * Modes: POT_WS_FP32 computes everything in FP32 on CUDA cores;
 * POT_WS_BF16 runs the three H x H contractions per point (forward and
 * backward) on tcgen05 tensor cores with BF16 operands and FP32
 * accumulation, the rest in FP32.
 *
 * Conventions as in aspot.h: device pointers unless marked "host", caller
 * owns every buffer, scratch from the caller's workspace, work enqueued on
 * `stream` (these calls do not synchronise it unless stated), POT_EINVAL for
 * bad arguments before any launch, message in pot_last_error().
 * Reductions are deterministic (fixed order, no floating-point atomics).
 */
#ifndef ASPOT_WARMSTART_H
#define ASPOT_WARMSTART_H

#include "aspot.h"

#ifdef __cplusplus
extern "C" {
#endif

#define POT_WS_HIDDEN 128
#define POT_WS_MAX_D 6          /* point dimension limit */
#define POT_WS_EXTRA 5          /* features per point besides the d coordinates (F = d + 5 <= 11) */
#define POT_WS_TEMPS 3          /* soft-minimum features at temperatures gamma, 4 gamma, 16 gamma */

#define POT_WS_FP32 0
#define POT_WS_BF16 1

/* A set of instances in feature form.  Instance k owns points
 * [off[k], off[k+1]) of feats / target: its n row points, then its m column
 * points (the layout pot_ws_features writes). */
typedef struct {
  int64_t count;          /* instances */
  int32_t d;              /* point dimension, 1 <= d <= POT_WS_MAX_D */
  int32_t pad;
  const int64_t* off;     /* host, count + 1 non-decreasing offsets, off[0] = 0 */
  const float* feats;     /* [off[count]][d + 5] */
  const float* extra;     /* [count][2]: |r|_1 / s, |c|_1 / s */
  const float* target;    /* [off[count]] from pot_ws_targets; NULL when only predicting */
  const float* weight;    /* [off[count]] loss weights from pot_ws_targets, or NULL (all 1) */
} pot_ws_set;

typedef struct {           /* Adam (Kingma & Ba, 2015) */
  float lr, beta1, beta2, eps;
} pot_ws_adam;

/* Number of FP32 parameters for point dimension d (host out). */
POT_API pot_status pot_ws_param_count(int32_t d, int64_t* count);

/* Initial parameters: weights N(0, 1 / fan_in) from a counter-based
 * generator (SplitMix64 outputs, Box-Muller), biases 0.  Enqueued only. */
POT_API pot_status pot_ws_init(float* params, int32_t d, uint64_t seed, void* stream);

/* Features of one squared-Euclidean problem (any point kind, d <= 6) at
 * entropic parameter gamma: feats [(n + m)][d + 5] (rows first) and
 * extra [2].  Workspace size from pot_ws_features_workspace_size.  Runs the
 * max-cost pass when prob->cost_scale is 0 (and synchronises the stream for
 * it), then three pot_marginals passes. */
POT_API pot_status pot_ws_features_workspace_size(const pot_problem* prob, size_t* bytes /* host */);
POT_API pot_status pot_ws_features(const pot_problem* prob, double gamma, void* workspace, size_t ws_bytes,
                                   float* feats, float* extra, void* stream);

/* Training targets from the converged duals (u, v, w) of `prob`, n + m floats:
 *   target_i = gamma log K_i,  K_i = sum_j B_ij / e^{u_i} = e^w sum_j e^{v_j - C_ij/gamma},
 *   target_{n+j} = gamma log K'_j,  K'_j = sum_i B_ij / e^{v_j},
 * the log of the ratio of a point's transported mass to its slack at the
 * optimum (where (B1)_i + e^{u_i} = r_i, so u_i = log r_i - softplus(log K_i)).
 * gamma log K_i is a smooth function of the point (a soft minimum over the
 * other cloud); the sharp softplus is applied in closed form by the warm
 * start.  `weight` (may be NULL) receives the loss weights
 * sigmoid(log K)^2.  One pot_marginals pass (and the max pass when
 * prob->cost_scale is 0, which synchronises the stream); workspace as
 * pot_ws_features. */
POT_API pot_status pot_ws_targets(const pot_problem* prob, double gamma, const double* u, const double* v, double w,
                                  float* target, float* weight, void* workspace, size_t ws_bytes, void* stream);

/* Workspace for batches of at most max_batch instances of `set` (the
 * largest ones are assumed). */
POT_API pot_status pot_ws_workspace_size(const pot_ws_set* set, int32_t max_batch, size_t* bytes /* host */);

/* Prediction for the instances idx[0..nb) (host int32 indices into set):
 * y receives their points' outputs in batch order (instance idx[0]'s points,
 * then idx[1]'s, ...).  The batch-forming host step copies a small tile list
 * into the workspace.  Enqueued only. */
POT_API pot_status pot_ws_forward(const pot_ws_set* set, const int32_t* idx, int32_t nb, const float* params,
                                  int32_t mode, float* y, void* workspace, size_t ws_bytes, void* stream);

/* Weighted mean squared error of the batch (device scalar `loss`) and its gradient
 * with respect to every parameter (`grad`, pot_ws_param_count floats, same
 * layout as the parameters).  Needs set->target.  Enqueued only. */
POT_API pot_status pot_ws_gradient(const pot_ws_set* set, const int32_t* idx, int32_t nb, const float* params,
                                   int32_t mode, float* grad, float* loss, void* workspace, size_t ws_bytes,
                                   void* stream);

/* One Adam step on the batch: gradient as pot_ws_gradient, then
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * params -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps),
 * step >= 1.  `loss` (device scalar, may be NULL) receives the batch loss
 * before the step.  Enqueued only. */
POT_API pot_status pot_ws_train_step(const pot_ws_set* set, const int32_t* idx, int32_t nb, float* params,
                                     float* adam_m, float* adam_v, const pot_ws_adam* opt, int64_t step,
                                     int32_t mode, float* loss, void* workspace, size_t ws_bytes, void* stream);

/* Workspace for pot_ws_warm_start on this problem. */
POT_API pot_status pot_ws_warm_workspace_size(const pot_problem* prob, size_t* bytes /* host */);

/* Warm start of one problem: features, network prediction,
 * u0 = log r - softplus(y / gamma) on the rows and v0 = log c - softplus(y / gamma)
 * on the columns (device FP64, n and m; masses below 1e-12 times their mean
 * floored in the log), then the exact minimiser of phi along the three uniform shifts
 * (u + a 1, v + b 1, w), a closed form from |B(u0, v0, 0)|_1 and the sums of
 * e^{u0}, e^{v0}:
 *   e^a = (|r|_1 - s) / sum e^{u0_i},  e^b = (|c|_1 - s) / sum e^{v0_j},
 *   w0 = log s - log |B(u0, v0, 0)|_1 - a - b      (host out)
 * (a = 0 when |r|_1 = s, b = 0 when |c|_1 = s; w0 alone is the exact w-step).
 * At the optimum of phi all three shifts vanish.  Pass u0, v0, w0 to
 * aspot_solve through pot_params together with POT_FLAG_WARM_CHECK.
 * Synchronises the stream. */
POT_API pot_status pot_ws_warm_start(const pot_problem* prob, double gamma, const float* params, int32_t d,
                                     int32_t mode, double* u0, double* v0, double* w0, void* workspace,
                                     size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ASPOT_WARMSTART_H */
