/* registration.h — rigid point-cloud registration steps through POT
 * (appendix "Point Cloud Registration", experiment of Section 4.2).
 *
 * Model: target cloud x_1..x_n, source cloud y_1..y_m, rigid motion
 * F(y) = R y + t of the source, and
 *   min over (R, t, pi) of sum_ij pi_ij |x_i - (R y_j + t)|^2,  pi in U(r, c, s).
 * The registration loop alternates a POT solve (aspot_solve_batched on the
 * current source F(y)) with the weighted Procrustes fit below, for many
 * independent cloud pairs at once.  Host loop: `registration.py` in the
 * Python package.
 *
 * Fit (pot_rigid_fit), from the rounded plan
 *   pi_ij = exp(f_i + g_j - cost_scale |x_i - y_cur_j|^2 / gamma) + kappa p_i q_j
 * of each instance (pot_plan of the solve, y_cur = the instance's current
 * source points prob->Y) and the ORIGINAL source points y0:
 *   u_x = sum_i (pi 1)_i x_i / |pi|_1,   u_y = sum_j (pi^T 1)_j y0_j / |pi|_1,
 *   M = sum_ij pi_ij (x_i - u_x)(y0_j - u_y)^T = U S V^T,
 *   R = U diag(1, 1, det(U V^T)) V^T,   t = u_x - R u_y,
 * so R y0 + t is the whole motion from the original cloud.  (The appendix
 * prints V diag(1, 1, det(V U^T)) U^T, the transpose of the minimiser for
 * F(y) = R y + t; see the oracle's reading N19.)  The 3 x 3 SVD is a
 * one-sided Jacobi iteration (Hestenes, 1958) in FP64; a rank-deficient M
 * (planar or degenerate clouds) completes U by a cross product.
 *
 * Conventions as in aspot.h.  Instances must be squared-Euclidean problems
 * with FP32 points, d = 3 and an explicit cost_scale > 0.
 */
#ifndef ASPOT_REGISTRATION_H
#define ASPOT_REGISTRATION_H

#include "aspot.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Number of doubles per instance in the `fit` array. */
#define POT_RIGID_FIT_STRIDE 16

/* Workspace bytes for pot_rigid_fit / pot_rigid_apply on `count` instances. */
POT_API pot_status pot_rigid_workspace_size(int32_t count, size_t* bytes /* host */);

/* Weighted Procrustes fit of each instance's rounded plan.  probs, plans, y0
 * are host arrays of `count` entries (y0[k]: device FP32 [m_k][3], the
 * instance's original source points; probs[k].Y its current source points,
 * on which the plan was solved); gamma is the solve's.  fit: device FP64
 * [count][16] = R row-major (9), t (3), |pi|_1, det(U V^T) sign, Jacobi
 * sweeps, 0.  One CTA per instance; plan entries in FP32, moments and the
 * SVD in FP64.  Enqueued only. */
POT_API pot_status pot_rigid_fit(const pot_problem* probs, int32_t count, const pot_plan* plans, double gamma,
                                 const float* const* y0, double* fit, void* workspace, size_t ws_bytes,
                                 void* stream);

/* probs[k].Y <- R_k y0_k + t_k (device FP32, overwritten) for every instance,
 * with (R_k, t_k) from fit.  Enqueued only. */
POT_API pot_status pot_rigid_apply(const pot_problem* probs, int32_t count, const float* const* y0,
                                   const double* fit, void* workspace, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ASPOT_REGISTRATION_H */
