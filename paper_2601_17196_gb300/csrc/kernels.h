// Internal (host-side) declarations shared by the translation units of the
// library.  Nothing here is part of the public C-ABI (include/aspot.h).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include "pass.h"

namespace pot {

// ------------------------------------------------------------- launches --
// Launches of the staged solver loops.  While pdl_scope is alive on the host
// thread (set around the capture of a loop's CUDA graph), launch_k adds the
// programmatic-serialisation attribute: the kernel's blocks may be scheduled
// as soon as its predecessor's blocks have all called pdl_release(); the
// kernel itself starts with pdl_enter() (common.cuh), which waits for the
// predecessor to complete.  Kernels launched through launch_k call it first.
bool pdl_active();
struct pdl_scope {
  bool prev;
  explicit pdl_scope(bool on);
  ~pdl_scope();
};
template <class... KA, class... A>
inline void launch_k(void (*kern)(KA...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = pdl_active() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// ---------------------------------------------------------------- passes --
struct SimtLayout {
  int V; int H; int64_t ncolblk, nrowblk;   // generic tiles: ncolblk x nrowblk CTAs of H x 128V
  int dense_fast;                            // persistent dense pass (rows / columns) applies
  int64_t G, nrg, U, nslots;                 // its CTAs, 32-row units per panel, units, column slots
};
SimtLayout simt_layout(int64_t n, int64_t m);
void simt_dense_layout(SimtLayout& L, int64_t n, int64_t m, int num_sms);
void launch_pass_simt(const PassDesc& P, const SimtLayout& L, cudaStream_t st);
// per-pass FP32 hi/lo row and column terms (rowA / colA / colB of the descriptor)
void launch_prep(const PassDesc& P, int64_t n_pad, int64_t m_pad, cudaStream_t st);
void launch_sqnorm(int kind, const void* X, int64_t n, int d, int64_t ldx, float* out, cudaStream_t st);

// tcgen05 on-the-fly squared-Euclidean pass (BF16 points)
struct TcLayout {
  int64_t ncolblk, nrowblk;          // partial counts of the row / column passes (what the combines read)
  int64_t nchunks, tiles_per_chunk;  // general kernel: 128-row units x column chunks
  int64_t v1_nrowblk, v1_units;
  int v3;                            // hot-loop kernel (pass_tc3.cu) serves rows / columns passes
  int64_t G, T, ntiles2, nrb2, nslots, n_pad2;
  int64_t n_pad, m_pad;              // padding of the per-pass row / column terms
  // columns-only passes as rows-only passes of the transposed problem (the
  // point sets swapped): its layout, and sw_nslots partials per column
  int swap;
  int64_t sw_G, sw_T, sw_ntiles2, sw_nrb2, sw_nslots, sw_rows_pad, sw_cols_pad;
  int ok;
};
TcLayout tc_layout(int64_t n, int64_t m, int d);
bool tc_supported(const PassDesc& P);
cudaError_t launch_pass_tc(const PassDesc& P, const TcLayout& L, cudaStream_t st, cudaEvent_t before_main = nullptr);
// the pass runs transposed: its column partials number L.sw_nslots
inline bool tc_swaps_cols(const TcLayout& L, const PassDesc& P) {
  return L.v3 && L.swap && P.transpose && P.mode == PASS_COLS;
}
bool tc3_applicable(int d);
int tc3_tile_cols();
void tc3_fill_layout(TcLayout& L, int64_t n, int64_t m, int num_sms);
void tc3_fill_layout_swap(TcLayout& L, int64_t n, int64_t m, int num_sms);
cudaError_t launch_pass_tc3(const PassDesc& P, const TcLayout& L, const CUtensorMap& mx, const CUtensorMap& my,
                            cudaStream_t st);
cudaError_t launch_pass_tc3_cols_swapped(const PassDesc& P, const TcLayout& L, const CUtensorMap& my_rows,
                                         const CUtensorMap& mx_cols, cudaStream_t st);

// --------------------------------------------------------- device state --
struct DevState {
  double theta;
  double w_tilde, w_check, w_bar, w_grave, w_hat, w_z, w_out;
  double phi_check, phi_hat, phi_z;
  double E, tot;
  double L, s, thr, log_s;
  double sum_rt, sum_ct;
  double m2, sum_p, sum_q, kappa, log_k1, obj;
  double A_over_g;
  double theta_next;         // theta_{t+1}, formed once per iteration by the gradient kernel
  double e_start[2];         // E(z_warm), E(0) for the warm-start check
  int t, take_hat, done, max_iter, nonfinite, tc_err;
  int warm_used, pad3;
  unsigned int counter;
  unsigned int pad2;
  int kg, k2;                // greedy rule: block of the step at z_grave / at z^t
  int run_r3, run_c3;        // greedy rule: one-sided passes needed at z^t = z^
  double trace[4096][4];     // E, phi_z, phi_check, take_hat per iteration (ring)
};

struct RedBuf { double* part; unsigned int* counter; int nblk; };

struct AspotVecs {
  int64_t n, m;
  const double *rt, *ct, *lrt, *lct;
  double *ut, *vt, *uc, *vc, *ub, *vb, *ug, *vg, *uh, *vh, *uo, *vo;
  const float2* row_part; const float2* col_part;
  const double* lrow; const double* lcol;   // combined log row / column sums of the last pass
  int64_t ncolblk, nrowblk;
  double* red; unsigned int* counter;
  DevState* S;
  int trace;
  int fused;                 // the loop kernels combine the pass partials themselves (no combine launch)
};

struct SinkVecs {
  int64_t n, m;
  int drow, dcol;
  const double *re, *ce, *lre, *lce;   // extended marginals (n+1, m+1)
  double *u, *v, *uprev;               // extended potentials
  const float2* row_part; const float2* col_part;
  const double* lrow; const double* lcol;   // combined log row / column sums of the last pass
  int64_t ncolblk, nrowblk;
  double* red; unsigned int* counter;
  DevState* S;
  int trace;
  int fused;                 // the loop kernels combine the pass partials themselves (no combine launch)
};

struct RoundVecs {
  int64_t n, m;
  const double *r, *c;        // original marginals
  const double *u, *v;        // duals to round (w in S->w_out)
  double *f, *g, *p, *q;      // plan
  double* kappa;
  const float2* row_part; const float2* col_part;
  const double* lrow; const double* lcol;   // combined log row / column sums of the last pass
  int64_t ncolblk, nrowblk;
  double* red; unsigned int* counter;
  DevState* S;
};

// ------------------------------------------------------- batched solves --
// One instance of a batched solve: problem, setup scalars, iteration state
// and the caller's plan pointers.  Rows / columns of all instances are
// concatenated (row0 / col0 offsets).
struct BInst {
  int64_t n, m, row0, col0, tile0, ntile;
  const void* X; const void* Y; int32_t d, kind; int64_t ldx, ldy;
  const double* r; const double* c;
  double s, cost_scale, gC, maxc;
  double L, thr, log_s, sum_rt, sum_ct, eps_s;
  double theta, w_tilde, w_check, w_bar, w_grave, w_hat, w_z, w_out;
  double phi_check, phi_hat, phi_z, E, tot, m2, sum_q, kappa, obj;
  double mass_r, mass_c, min_r, min_c, bad;
  int32_t t, take_hat, done, nonfinite, branch, max_iter;
  int32_t kg, ticket;                // greedy rule: block of the step at z_grave; fused sweep: tiles done this pass
  double *pu, *pv, *pw, *pf, *pg, *pp, *pq, *pkappa;
};
struct BTile { int32_t inst, rb, cb, pad; };
struct BatchPass {
  int mode, kind, H, W;                                // W: tile columns, 128 or 256
  int64_t Ntot, Mtot;
  const BTile* tiles; int64_t ntiles;
  BInst* inst; int64_t count;
  const float* xn; const float* yn;                    // concatenated squared norms
  float4* rowA; float2* colA; float2* colB;           // concatenated per-pass terms (batched prep)
  const double *arow0, *bcol0, *arow1, *bcol1;          // concatenated potentials (set 0 / set 1)
  int aoff0, aoff1;                                    // byte offset of the scalar w in BInst, -1: none
  int use_sel;                                         // set 1 when the instance's take_hat is set
  int check_done;                                      // tiles of finished instances return at once
  float2* row_part; float2* col_part; double* red_part;
  const double *p, *q;                                 // concatenated rank-one factors (objective)
};
void launch_pass_simt_batched(const BatchPass& B, cudaStream_t st);
void launch_prep_batched(const BatchPass& B, cudaStream_t st);

// ------------------------------------------- single-cluster ASPOT loop --
// One small problem iterated by one thread-block cluster (cluster.cu): the
// CTAs share each pass's tiles, CTA 0 runs the per-instance update of the
// batched solver on the single-instance solver's own vectors.
struct ClusterLoop {
  PassDesc P;        // base pass: problem, logit multiplier, FP32 terms, partial buffers
  AspotVecs vecs;    // the solver's vectors
  BInst* inst;       // device record of the instance (entered from / left to DevState)
  int* ndone;        // device int the bodies count the instance in when it stops
  int H, V;          // tile rows (a multiple of 32); 128-column groups per tile (1 or 2)
  int ncta;          // CTAs of the cluster (8 or 16)
  double* trace4;    // DevState::trace rows to fill (POT_FLAG_TRACE), or NULL
};
int cluster_loop_kind(const PassDesc& P);           // 0: not supported; 1 / 3 dense FP32 (aligned / not), 2 FP32 points d <= 4
int cluster_loop_size(const PassDesc& P, int V);    // largest resident cluster, 0 if none
cudaError_t launch_cluster_enter(BInst* I, const DevState* S, cudaStream_t st);
cudaError_t launch_cluster_exit(const BInst* I, DevState* S, cudaStream_t st);
cudaError_t launch_cluster_loop(const ClusterLoop& A, int iters, int greedy, int first, cudaStream_t st);

constexpr int kVecThreads = 256;
inline int vec_blocks(int64_t len) { return (int)((len + kVecThreads - 1) / kVecThreads); }
// the solver loops' O(n + m) kernels run 64-thread blocks up to this length (vec.cu)
constexpr int64_t kLoopSmallLen = 32768;
inline int64_t loop_blocks_max(int64_t len) { return (len + 63) / 64; }   // bound for reduction buffers

// prologue: masses, minima, finiteness of r and c -> S (sum_rt/ct reused as raw masses)
void launch_marg_stats(const double* r, const double* c, int64_t n, int64_t m, double* red,
                       unsigned int* counter, double* out6, cudaStream_t st);
void launch_reduce_parts(const double* part, int64_t count, int op_max, double* out, cudaStream_t st);
void launch_aspot_init(const AspotVecs& V, const double* r, const double* c, double eps_s,
                       const double* u0, const double* v0, double w0, cudaStream_t st);
void launch_aspot_extrap(const AspotVecs& V, cudaStream_t st);
void launch_aspot_after_grad(const AspotVecs& V, cudaStream_t st);
void launch_aspot_after_greenkhorn(const AspotVecs& V, int k, cudaStream_t st);
void launch_aspot_after_final(const AspotVecs& V, int k, cudaStream_t st);
void launch_aspot_greedy_pick(const AspotVecs& V, cudaStream_t st);
void launch_aspot_greedy_final(const AspotVecs& V, cudaStream_t st);
void launch_aspot_greedy_apply(const AspotVecs& V, cudaStream_t st);
void launch_aspot_start_eval(const AspotVecs& V, const double* u, const double* v, int slot, cudaStream_t st);
void launch_aspot_zero_bar(const AspotVecs& V, cudaStream_t st);
void launch_aspot_start_select(const AspotVecs& V, cudaStream_t st);

void launch_sink_init(const SinkVecs& V, const double* r, const double* c, double eps_s, double s,
                      cudaStream_t st);
void launch_sink_after_rows(const SinkVecs& V, cudaStream_t st);
void launch_sink_after_cols(const SinkVecs& V, cudaStream_t st);

void launch_round_r1(const RoundVecs& V, cudaStream_t st);
void launch_round_r2(const RoundVecs& V, cudaStream_t st);
void launch_round_r3(const RoundVecs& V, cudaStream_t st);
void launch_round_r4(const RoundVecs& V, cudaStream_t st);

void launch_marginals_setup(DevState* S, double w, unsigned int* counter, cudaStream_t st);
// err: a raised pass error flag turns every output into NaN
void launch_marginals_out(int64_t n, int64_t m, const double* lrow_in, const double* lcol_in, double* lrow,
                          double* lcol, double* red, unsigned int* counter, double* tot_out, const int* err,
                          cudaStream_t st);
void launch_combine(const float2* row_part, int64_t ncolblk, int64_t n, double* lrow, const float2* col_part,
                    int64_t nrowblk, int64_t m, double* lcol, const int* done, cudaStream_t st,
                    const int* skip = nullptr, int skip_if = 0);
void launch_dense_plan(const PassDesc& P, const double* f, const double* g, const double* p,
                       const double* q, const double* kappa, float* X, int64_t ldx, cudaStream_t st);

}  // namespace pot
