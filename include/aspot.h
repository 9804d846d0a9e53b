/* aspot.h — C-ABI of the GB300 (sm_103a) entropic Partial Optimal Transport
 * library: Accelerated Sinkhorn for POT (ASPOT, arXiv 2601.17196,
 * Algorithm 2), the feasible Sinkhorn baseline it improves on (Algorithm 3
 * with the setup of Algorithm 2, Section 4.1), the rounding of an entropic
 * plan to a feasible plan of mass s, and the transport cost <C, X>.
 *
 * Problem (Section 2.1):  POT(r, c, s) = min <C, X> over
 *   U(r, c, s) = { X >= 0 : X 1 <= r, X^T 1 <= c, 1^T X 1 = s },
 * with r in R^n_+, c in R^m_+ of possibly different total mass and
 * 0 < s <= min(|r|_1, |c|_1).  The entropic dual (Eq. dual) is
 *   phi(u, v, w) = |B|_1 + sum e^{u_i} + sum e^{v_j} - <u, r> - <v, c> - w s,
 *   B_ij = exp(-C_ij / gamma + u_i + v_j + w).
 *
 * Conventions (every entry point):
 *  - All array pointers are DEVICE pointers unless the comment says "host".
 *    The caller owns every buffer; the library keeps no pointer after the
 *    call returns and allocates no device memory: scratch comes from the
 *    caller's workspace (size from pot_workspace_size).
 *  - Row-major layouts: cost C[i*ldc + j] (FP32, ldc >= m); points
 *    X[i*ldx + k], Y[j*ldy + k] (BF16, FP16 or FP32 by pot_cost_kind,
 *    ldx, ldy >= d).
 *  - Work is enqueued on `stream` (cudaStream_t passed as void*, NULL =
 *    legacy default stream).  The solvers synchronise the stream before they
 *    return (they poll a device stop flag); pot_marginals and
 *    pot_plan_dense do not.
 *  - Every call returns a pot_status; on failure pot_last_error() returns a
 *    thread-local message.  Invalid arguments are rejected with POT_EINVAL
 *    before anything is launched.
 */
#ifndef ASPOT_H
#define ASPOT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define POT_API __attribute__((visibility("default")))
#else
#define POT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  POT_OK = 0,
  POT_EINVAL = 1,      /* bad argument (sizes, pointers, s, eps, workspace) */
  POT_ENOMEM = 2,      /* workspace too small */
  POT_ECUDA = 3,       /* a CUDA call failed (message in pot_last_error) */
  POT_ENOCONV = 4,     /* max_iter reached before the stop test; the plan is still rounded and feasible */
  POT_ENONFINITE = 5,  /* NaN/Inf in a potential or a sum */
  POT_ETIMEOUT = 6     /* the stop flag was never set, or a tcgen05 pass's bounded pipeline wait ran out
                          (its sums are then invalid; see pot_params.wait_limit_ns) */
} pot_status;

typedef enum {
  POT_COST_DENSE_F32 = 0,      /* C given as an n x m FP32 matrix */
  POT_COST_SQEUCLID_BF16 = 1,  /* C_ij = cost_scale * |x_i - y_j|^2, BF16 points (tcgen05 path when d % 64 == 0) */
  POT_COST_SQEUCLID_F16 = 2,   /* same with FP16 points */
  POT_COST_SQEUCLID_F32 = 3    /* same with FP32 points (CUDA cores; meant for small d such as 2 or 3) */
} pot_cost_kind;

/* flags of pot_params.flags */
#define POT_FLAG_STOP_RAW_EPS 1   /* stop at E_t <= eps instead of eps/(8 max C) */
#define POT_FLAG_NO_SMOOTH 2      /* skip the marginal smoothing of Algorithm 2's setup */
#define POT_FLAG_TRACE 4          /* record E_t, phi(z^t), phi(z_check^{t+1}), argmin per iteration */
#define POT_FLAG_NO_STOP 8        /* run exactly max_iter iterations (fixed-iteration mode) */
#define POT_FLAG_FORCE_SIMT 16    /* use the CUDA-core pass even where the tcgen05 pass applies */
#define POT_FLAG_PROFILE 32       /* time every main-loop pass with CUDA events (res->pass_ms, pass_launches) */
#define POT_FLAG_WARM_CHECK 64    /* with u0 / v0: start from zero instead when E(z_warm) > E(0) (res->warm_used) */
#define POT_FLAG_AUTOTUNE 128     /* aspot_solve_batched: tile shape of the batched pass from the autotune cache,
                                     else the fastest candidate timed on this batch (then cached) */
#define POT_FLAG_STAGED 256       /* aspot_solve: run the iterations as separate kernels in CUDA graphs even where
                                     the single-cluster loop applies (see pot_result.cluster_loop) */

typedef struct {
  int64_t n, m;
  int32_t kind;                 /* pot_cost_kind */
  const float* C; int64_t ldc;  /* dense cost (kind 0) */
  const void* X; const void* Y; /* point clouds (kinds 1-3) */
  int32_t d; int64_t ldx, ldy;
  double cost_scale;            /* effective cost = cost_scale * C (or * |x-y|^2); 0 => 1 / max entry, computed */
  const double* r;              /* FP64 [n], finite, >= 0 */
  const double* c;              /* FP64 [m], finite, >= 0 */
  double s;                     /* 0 < s <= min(|r|_1, |c|_1) */
} pot_problem;

/* Complete state of an ASPOT solve between two iterations (Algorithm 2): the
 * gradient sequence z~ = (u~, v~, w~), the Greenkhorn sequence z_check with
 * phi(z_check), theta_t and the iteration count t.  Filled by
 * aspot_state_export; passed back through pot_params.resume, the solve goes
 * on from iteration t exactly as if it had not stopped.  Vectors are device
 * FP64 buffers owned by the caller. */
typedef struct {
  double* u_tilde;     /* [n] */
  double* v_tilde;     /* [m] */
  double* u_check;     /* [n] */
  double* v_check;     /* [m] */
  double w_tilde, w_check, phi_check, theta;
  int32_t t, pad;
} pot_aspot_state;

typedef struct {
  double gamma;        /* entropic parameter; <= 0 => eps / (4 log max(n, m)) (Algorithm 2 setup) */
  double eps;          /* accuracy; stop threshold eps~ = eps / (8 max C) (Algorithm 2 setup) */
  double p_tune;       /* feasible Sinkhorn only: >= 1 => gamma = (2 eps/(49 H_min))^(1/p), eps' = H_min gamma^p (Theorem 2) */
  int32_t max_iter;    /* iteration cap (> 0) */
  int32_t block_rule;  /* ASPOT Greenkhorn block choice: 0 = cyclic t mod 3 (Algorithm 1); 1 = greedy,
                          the block whose step decreases phi the most (the choice of Theorem 3's proof),
                          scored exactly from a two-sided pass (P2 then costs a full pass); ASPOT and
                          aspot_solve_batched */
  int32_t flags;       /* POT_FLAG_* */
  int32_t check_every; /* iterations per captured CUDA graph between host polls of the stop flag (0 => 24) */
  const double* u0;    /* optional warm start of ASPOT (device FP64 [n]) or NULL */
  const double* v0;    /* optional warm start (device FP64 [m]) or NULL */
  double w0;
  const pot_aspot_state* resume;  /* ASPOT only: continue from an exported state (NULL => start from z~ = z_check
                                     = the warm start or zero); excludes u0 / v0 / w0; max_iter counts from 0,
                                     so it must exceed the state's t */
  int64_t wait_limit_ns;  /* bound, in ns, of every pipeline wait inside the tcgen05 passes (0 => 2 s).  A pass
                             whose wait runs out stops, drains its own copies and MMAs, frees its tensor memory
                             and raises a flag: the solve then returns POT_ETIMEOUT.  A negative value is a
                             test hook: the solve's hot-loop tcgen05 passes also withhold their first
                             accumulator hand-off, so their waits run out after |wait_limit_ns| ns */
} pot_params;

/* Rounded plan, kept implicit (O(n + m) storage):
 *   X_ij = exp(f_i + g_j - cost_scale * C_ij / gamma) + kappa * p_i * q_j
 * which lies in U(r, c, s).  All pointers device FP64, caller-allocated. */
typedef struct {
  double* u; double* v; double* w;     /* final duals z^t (n, m, 1); for Sinkhorn the first n / m extended potentials and w = 0 */
  double* f; double* g;                /* plan potentials (n, m) */
  double* p; double* q;                /* rank-one factors (n, m) */
  double* kappa;                       /* scalar */
} pot_plan;

typedef struct {            /* host struct filled by the solvers */
  int32_t status;
  int32_t iters;            /* iterations run */
  double objective;         /* <C_eff, X> of the rounded plan (FP64 accumulation) */
  double err_final;         /* E_t (ASPOT) or the l1 marginal residual (Sinkhorn) at the returned duals */
  double eps_stop;          /* threshold the stop test used */
  double gamma;             /* gamma used */
  double cost_scale;        /* effective cost scale (1 / max C when computed) */
  double mass;              /* total mass of the rounded plan (= s) */
  double ms;                /* device time of the whole call (CUDA events) */
  int32_t rounding_branch;  /* 3: uniform scale to s, 4: rank-one fill */
  int32_t nonfinite;
  double pass_ms;           /* POT_FLAG_PROFILE: summed CUDA-event time of the main-loop passes */
  int64_t pass_launches;    /* POT_FLAG_PROFILE: number of passes timed */
  int64_t kernel_launches;  /* kernels this call launched (all of them this library's own) */
  double err_warm;          /* POT_FLAG_WARM_CHECK: E at the given start (u0, v0, w0) */
  double err_zero;          /* POT_FLAG_WARM_CHECK: E at the zero start */
  int32_t warm_used;        /* 1 if the iterations started from (u0, v0, w0) */
  int32_t tile_rows;        /* aspot_solve_batched: rows x columns of the batched pass's tiles */
  int32_t tile_cols;
  int32_t cluster_loop;     /* aspot_solve: 1 if the iterations ran in the single-cluster loop kernel (small
                               problems with CUDA-core passes, no PROFILE / STAGED flag), else 0 */
  double tune_ms;           /* aspot_solve_batched, POT_FLAG_AUTOTUNE: device time spent timing candidates
                               (0 when the shape came from the cache) */
} pot_result;

/* Bytes of device workspace the solvers / pot_round / pot_objective /
 * pot_marginals need for this problem.  Returns POT_EINVAL for bad sizes. */
POT_API pot_status pot_workspace_size(const pot_problem* prob, const pot_params* params, size_t* bytes /* host */);

/* ASPOT (Algorithm 2): setup, accelerated loop with Greenkhorn couplings
 * (Algorithm 1), primal B(z^t), rounding (pot_round) and the objective.
 * `plan` receives the duals and the rounded plan; `res` (host) the summary. */
POT_API pot_status aspot_solve(const pot_problem* prob, const pot_params* params, void* workspace, size_t ws_bytes,
                       pot_plan* plan, pot_result* res, void* stream);

/* Feasible Sinkhorn baseline: alternating exact row / column scalings of the
 * (n+1) x (m+1) dummy-extended kernel (appendix, Algorithm 3), gamma and the
 * stop threshold from Algorithm 2's setup (or the tuned rule when
 * params->p_tune >= 1), then the same rounding of the top-left block. */
POT_API pot_status sinkhorn_pot_solve(const pot_problem* prob, const pot_params* params, void* workspace,
                              size_t ws_bytes, pot_plan* plan, pot_result* res, void* stream);

/* ROUND-POT (cited by Algorithm 2; reading R1-R4): rounds B(u, v, w) to
 * U(r, c, s) with the ORIGINAL r, c, s of `prob`:
 *   a = min(1, r / B1), b = min(1, c / (diag(a)B)^T 1), X'' = diag(a) B diag(b);
 *   mass m'' >= s: X = (s/m'') X'';  else X = X'' + (s - m'') p q^T / (|p| |q|),
 *   p = r - X'' 1, q = c - X''^T 1.
 * u, v device FP64; w host.  Fills plan->f, g, p, q, kappa; writes the
 * branch taken (3 or 4) to *branch (host, may be NULL). */
POT_API pot_status pot_round(const pot_problem* prob, double gamma, const double* u, const double* v, double w,
                     void* workspace, size_t ws_bytes, pot_plan* plan, int32_t* branch, void* stream);

/* <C_eff, X> of an implicit plan (Definition 1), FP64 accumulation. */
POT_API pot_status pot_objective(const pot_problem* prob, const pot_plan* plan, double gamma, void* workspace,
                         size_t ws_bytes, double* out /* host */, void* stream);

/* Log row and column sums of B(u, v, w): lrow[i] = log sum_j B_ij,
 * lcol[j] = log sum_i B_ij (device FP64, either may be NULL), and
 * *tot = |B|_1 (device FP64 scalar, may be NULL).  With lrow NULL and lcol
 * given, one columns-only pass runs and *tot is the sum over the columns.  Enqueued only; w is
 * passed by value to a kernel, so the call may be captured into a CUDA graph.
 * If the tcgen05 pass gave up waiting on its pipeline, every output is NaN
 * and pot_pass_status reports POT_ETIMEOUT. */
POT_API pot_status pot_marginals(const pot_problem* prob, double gamma, const double* u, const double* v, double w,
                         void* workspace, size_t ws_bytes, double* lrow, double* lcol, double* tot,
                         void* stream);

/* Bytes of workspace pot_marginals needs (one pass: less than
 * pot_workspace_size, which covers the solvers' iteration state). */
POT_API pot_status pot_marginals_workspace_size(const pot_problem* prob, size_t* bytes /* host */);

/* Status of the last pot_marginals that used `workspace`: synchronises
 * `stream`, then returns POT_ETIMEOUT if its tcgen05 pass gave up waiting on
 * its pipeline (the outputs are then NaN), else POT_OK. */
POT_API pot_status pot_pass_status(void* workspace, void* stream);

/* Batched ASPOT: `count` independent problems (host array `probs`, each with
 * its own device buffers, sizes and s; squared-Euclidean point clouds of one
 * kind with d <= 4, as in the 3-D registration workloads of Section 4.2)
 * solved in lockstep with the shared `params` (gamma, eps, max_iter, flags).
 * Every O(nm) pass of an iteration is one launch over a work list of tiles of
 * all instances still running; an instance stops at its own threshold.
 * `plans` and `res` are host arrays of `count` entries (plan buffers on the
 * device); the return value is the worst instance status.  Workspace size
 * from pot_workspace_size_batched.  The call synchronises `stream` (setup,
 * autotuning, stop polling), so a stream under graph capture is rejected with
 * POT_EINVAL, as for the single-instance solvers. */
POT_API pot_status pot_workspace_size_batched(const pot_problem* probs, int32_t count, size_t* bytes /* host */);
POT_API pot_status aspot_solve_batched(const pot_problem* probs, int32_t count, const pot_params* params,
                                       void* workspace, size_t ws_bytes, pot_plan* plans, pot_result* res,
                                       void* stream);

/* Decisions of the last aspot_solve_batched that used this workspace: for
 * each of the `count` instances (the same probs as the solve), the first
 * `iters` iterations (0 <= iters <= 1024) as one byte each, took + 2 k + 8 k2:
 * took = 1 when the argmin kept z^, k the block of the Greenkhorn step at
 * z_grave, k2 that of the step at z^t (k2 = k for the cyclic rule).  Bytes of
 * iterations an instance did not run are undefined.  out: host [count][iters].
 * Synchronises the stream. */
POT_API pot_status pot_trace_batched(void* workspace, const pot_problem* probs, int32_t count, int32_t iters,
                                     uint8_t* out /* host */, void* stream);

/* Autotuner of the batched pass.  A tile is tile_rows x tile_cols entries of
 * one instance, handled by one CTA; the candidates are 32, 64, 128, 256 rows
 * x 128, 256 columns (default 256 x 256).  With POT_FLAG_AUTOTUNE,
 * aspot_solve_batched takes the shape cached for the batch's signature (cost
 * kind, largest d, count, total and largest n and m) or, on a miss, times
 * every candidate on one two-sided pass of this batch (CUDA events, three
 * repetitions after a warm-up; the call synchronises its stream) and caches
 * the fastest.  The cache lives in the process; access is thread-safe.
 *   pot_autotune_set:    pin a shape for the signature of `probs` (POT_EINVAL
 *                        for a shape outside the candidates);
 *   pot_autotune_lookup: the cached shape (host outs), 0 x 0 when none;
 *   pot_autotune_clear:  drop every entry;
 *   pot_autotune_save / _load: the cache as text lines "signature rows cols"
 *                        (load merges; POT_EINVAL for an unreadable or
 *                        malformed file, which then leaves the cache as it was). */
POT_API pot_status pot_autotune_set(const pot_problem* probs, int32_t count, int32_t tile_rows, int32_t tile_cols);
POT_API pot_status pot_autotune_lookup(const pot_problem* probs, int32_t count, int32_t* tile_rows /* host */,
                                       int32_t* tile_cols /* host */);
POT_API pot_status pot_autotune_clear(void);
POT_API pot_status pot_autotune_save(const char* path);
POT_API pot_status pot_autotune_load(const char* path);

/* pot_marginals without a workspace, for callers that cannot allocate
 * device memory (for example while a framework's caching allocator owns the
 * device, or in a loop that forbids allocation after start-up).  The paper
 * has no counterpart: this is a deployment convenience.  Scratch comes from a
 * 16 MiB array inside the library (held on every GPU that loads it);
 * problems whose pot_marginals_workspace_size exceeds it are rejected with
 * POT_ENOMEM.  All calls share that array, so
 * calls that overlap on the GPU race.  The first call on a device looks up
 * the array's address and should come before any stream capture.
 * Arguments and results as pot_marginals.  Enqueued only. */
POT_API pot_status pot_marginals_static(const pot_problem* prob, double gamma, const double* u, const double* v,
                                        double w, double* lrow, double* lcol, double* tot, void* stream);

/* Largest entry of the raw cost (max C_ij or max |x_i - y_j|^2), host out. */
POT_API pot_status pot_cost_max(const pot_problem* prob, void* workspace, size_t ws_bytes, double* out, void* stream);

/* Materialise an implicit plan into X (device FP32, row-major, ldx >= m). */
POT_API pot_status pot_plan_dense(const pot_problem* prob, const pot_plan* plan, double gamma, float* X, int64_t ldx,
                          void* stream);

/* State of the last aspot_solve that used `workspace`, with the same prob and
 * params->flags: z~ and z_check are copied into state's device vectors and
 * the scalars are filled, for a later resume.  Synchronises the stream. */
POT_API pot_status aspot_state_export(const pot_problem* prob, const pot_params* params, void* workspace,
                                      size_t ws_bytes, pot_aspot_state* state, void* stream);

/* Per-iteration record of the last solve that set POT_FLAG_TRACE, copied
 * into host `out` as [iters][4] doubles (E_t, phi(z^t), phi(z_check^{t+1}),
 * argmin took z^; with the greedy block rule the last entry is
 * took + 2 k + 8 k2, k the block of the step at z_grave and k2 that of the
 * step at z^t).  Keeps the last 4096 iterations. */
POT_API pot_status pot_trace(void* workspace, int32_t iters, double* out /* host */, void* stream);

/* Name of the CUDA kernel that runs the O(nm) passes of a solver's main loop
 * for this problem and these flags: "tc2_pass_kernel" (tcgen05, d = 64 or
 * 128), "tc_pass_kernel" (tcgen05, other d), "dense_pass_kernel" (dense FP32
 * cost, 16-byte aligned rows) or "pass_simt_kernel" (every other case);
 * "" for an invalid problem.  A static string; host only, launches nothing. */
POT_API const char* pot_pass_kernel(const pot_problem* prob, int32_t flags);

/* Thread-local message of the last failure ("" if none). */
POT_API const char* pot_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ASPOT_H */
