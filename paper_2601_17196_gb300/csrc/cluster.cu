// ASPOT loop of one small problem on one thread-block cluster.
//
// For a problem of a few hundred thousand cost entries an iteration of
// Algorithm 2 is three passes and three O(n + m) updates whose work is a few
// microseconds each; run as separate kernels, every step pays a launch and a
// dependent chain of global-memory round trips.  Here one cluster of up to
// 16 CTAs runs `iters` whole iterations in one launch: per pass the CTAs
// share the tiles of the CUDA-core pass (simt_tile, the same tile body as the
// single-instance and batched passes), a hardware cluster barrier, then CTA 0
// alone runs the per-instance epilogue of the fused batched sweep (combine of
// the partials into FP64 log-sums, the update of the block rule, the
// extrapolation, the next pass's FP32 terms) and a second barrier.  Six
// cluster barriers per iteration and no grid-wide synchronisation.
//
// The iteration state lives in the single-instance solver's own vectors (the
// loop is entered and left through cl_enter / cl_exit, which move the scalars
// between DevState and the one BInst the bodies use), so warm starts, resume,
// state export, rounding and the objective are those of the staged loop.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aspot.h"
#include "common.cuh"
#include "kernels.h"
#include "simt_tile.cuh"
#include "inst_body.cuh"

using namespace pot;
using namespace pot::simt;
using namespace pot::inst;

namespace {

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; release / acquire at cluster scope
// orders the partials and per-pass terms written before it with the reads after
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// store to the shared memory of CTA `rank` of the cluster, at the address
// `p` has in this CTA's (every CTA has the same layout)
__device__ __forceinline__ void st_cluster(double* p, unsigned rank, double v) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}

constexpr int kMaxCta = 16;
constexpr int kXW = 12;       // doubles per CTA in an exchange (up to 9 sums, or one log-sum)

// The CTAs of the cluster update the instance together.  Entry i (a row or a
// column) belongs to CTA i mod ncta, thread i / ncta, so every CTA takes an
// interleaved share and only the first `nwa` warps hold entries.  Every CTA
// keeps its own copy of the instance record and runs the scalar part of each
// update on it: a sum's block totals are exchanged through distributed shared
// memory and added in rank order, so every CTA gets the same totals, the
// copies stay equal, and no CTA reads a record field another CTA is writing.
// FP64 work here is spread so: on this GPU a warp-wide FP64 instruction
// occupies an SM sub-partition for many cycles.
struct ClusterTeam {
  unsigned rank, ncta;
  int nwa;                 // warps with entries
  int round;               // exchanges so far (the same sequence in every CTA)
  double* xbuf;            // [2][kMaxCta][kXW], the same offset in every CTA
  BInst* I;                // this CTA's copy of the record
  __device__ int64_t first() const { return (int64_t)threadIdx.x * ncta + rank; }
  __device__ int64_t step() const { return (int64_t)blockDim.x * ncta; }
  __device__ bool writer() const { return rank == 0 && threadIdx.x == 0; }
  __device__ BInst& inst(const BVecs&, int) const { return *I; }

  template <int NV>
  __device__ void sums(double (&v)[NV]) {
    static_assert(NV <= kXW, "exchange too small");
    __shared__ double sh[NV][8];
    __shared__ double tot[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < nwa) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const double x = warp_sum_d(v[k]);
        if (lane == 0) sh[k][warp] = x;
      }
    }
    __syncthreads();
    double* buf = xbuf + (round & 1) * (kMaxCta * kXW);
    if (threadIdx.x < NV) {
      double b = 0.0;
      for (int w = 0; w < nwa; ++w) b += sh[threadIdx.x][w];
      for (unsigned r = 0; r < ncta; ++r) st_cluster(buf + rank * kXW + threadIdx.x, r, b);
    }
    cl_sync();
    if (threadIdx.x < NV) {
      double t = 0.0;
      for (unsigned r = 0; r < ncta; ++r) t += buf[r * kXW + threadIdx.x];
      tot[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = tot[k];
    ++round;
  }

  // natural log of sum over all threads of the team of e^x (x: log-sums from
  // FP32 pass partials, so exp_sum is accurate enough); POT_NEG_BIG if none
  __device__ double lse(double x, bool act) {
    __shared__ double wm[8], ws[8];
    __shared__ double res;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < nwa) {
      double m = act ? x : -INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      double e = (act && m > -INFINITY) ? exp_sum(x - m) : 0.0;
      e = warp_sum_d(e);
      if (lane == 0) { wm[warp] = m; ws[warp] = e; }
    }
    __syncthreads();
    double* buf = xbuf + (round & 1) * (kMaxCta * kXW);
    if (warp == 0) {             // the CTA's (max, sum), then its log-sum to every CTA
      const double m0 = (lane < nwa && ws[lane] > 0.0) ? wm[lane] : -INFINITY;
      double M = m0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) M = fmax(M, __shfl_xor_sync(0xffffffffu, M, o));
      double S = (m0 > -INFINITY) ? ws[lane] * exp_sum(m0 - M) : 0.0;
      S = warp_sum_d(S);
      const double L = (M > -INFINITY && S > 0.0) ? M + log(S) : POT_NEG_BIG;
      if (lane < (int)ncta) st_cluster(buf + rank * kXW, lane, L);
    }
    cl_sync();
    if (warp == 0) {             // rank-order log-sum-exp of the ncta values, one per lane
      const double Lr = lane < (int)ncta ? buf[lane * kXW] : POT_NEG_BIG;
      const bool ok = Lr > POT_NEG_BIG;
      double M = ok ? Lr : -INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) M = fmax(M, __shfl_xor_sync(0xffffffffu, M, o));
      double S = ok ? exp_sum(Lr - M) : 0.0;
      S = warp_sum_d(S);
      if (lane == 0) res = (M > -INFINITY && S > 0.0) ? M + log(S) : POT_NEG_BIG;
    }
    __syncthreads();
    const double r = res;
    ++round;
    return r;
  }
};

template <int KIND, int VV, int DM, bool VEC, int MT>
__device__ __forceinline__ void cl_tiles(const PassDesc& P, int H, int64_t ncb, int64_t nt, unsigned rank,
                                         unsigned ncta) {
  for (int64_t tau = rank; tau < nt; tau += ncta)
    simt_tile<KIND, VV, DM, VEC, MT>(P, H, tau % ncb, tau / ncb, P.n, P.m, tau);
}

// One pass and its epilogue (every CTA: its share of the combine, the update
// and the next pass's terms).  MT: 1 rows + columns, 2 rows, 3 columns.
template <int KIND, int VV, int DM, bool VEC, int MT>
__device__ __forceinline__ void cl_sweep(const PassDesc& P, const BatchPass& B, const BVecs& V, int64_t ncb,
                                         int64_t nt, ClusterTeam& tm, int epi, int k) {
  cl_tiles<KIND, VV, DM, VEC, MT>(P, B.H, ncb, nt, tm.rank, tm.ncta);
  cl_sync();
  b_epilogue(B, V, 0, epi, k, tm);
  cl_sync();
}

// `iters` iterations (fewer when the instance stops).  first: form z_bar and
// the first pass's terms (the state comes from the solver's set-up).  The
// record is read from global memory at the start and written back by CTA 0
// at the end (the host polls its stop flag between launches).
template <int KIND, int VV, int DM, bool VEC>
__global__ void __launch_bounds__(kThreads, 1)
cl_loop_kernel(PassDesc P, BatchPass B, BVecs V, int iters, int greedy, int first) {
  __shared__ BInst sI;
  __shared__ double xbuf[2 * kMaxCta * kXW];
  ClusterTeam tm;
  tm.rank = cl_rank();
  tm.ncta = cl_size();
  tm.round = 0;
  tm.xbuf = xbuf;
  tm.I = &sI;
  {
    const int64_t per = (((P.n > P.m ? P.n : P.m) + tm.ncta - 1) / tm.ncta);
    const int64_t w = (per + 31) / 32;
    tm.nwa = (int)(w < kWarps ? (w < 1 ? 1 : w) : kWarps);
  }
  if (threadIdx.x == 0) sI = V.inst[0];
  __syncthreads();
  const int64_t ncb = (P.m + 128 * VV - 1) / (128 * VV);
  const int64_t nt = ncb * ((P.n + B.H - 1) / B.H);
  if (first) {
    if (!sI.done) {
      b_extrap_body(V, 0, tm);
      __syncthreads();
      b_prep_body(B, sI, V.ub, V.vb, sI.w_bar, tm);
    }
    cl_sync();
  }
  constexpr int RC = 1, R = 2, C = 3;
  for (int it = 0; it < iters; ++it) {
    if (sI.done) break;                               // the same in every CTA's copy
    const int k = sI.t % 3;                           // the cyclic rule's block t mod 3
    cl_sweep<KIND, VV, DM, VEC, RC>(P, B, V, ncb, nt, tm, E_GRAD, k);
    if (greedy) {
      cl_sweep<KIND, VV, DM, VEC, RC>(P, B, V, ncb, nt, tm, E_GGK, k);
      cl_sweep<KIND, VV, DM, VEC, RC>(P, B, V, ncb, nt, tm, E_GFINAL, k);
    } else {
      if (k == 1) cl_sweep<KIND, VV, DM, VEC, C>(P, B, V, ncb, nt, tm, E_GK, k);
      else cl_sweep<KIND, VV, DM, VEC, R>(P, B, V, ncb, nt, tm, E_GK, k);
      cl_sweep<KIND, VV, DM, VEC, RC>(P, B, V, ncb, nt, tm, E_FINAL, k);
    }
  }
  if (tm.rank == 0 && threadIdx.x == 0) V.inst[0] = sI;
}

// DevState -> the instance record of the bodies (set-up scalars and the
// iteration state; sizes and pointers were written by the host)
__global__ void cl_enter_kernel(BInst* I, const DevState* S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  I->L = S->L; I->thr = S->thr; I->log_s = S->log_s; I->sum_rt = S->sum_rt; I->sum_ct = S->sum_ct; I->s = S->s;
  I->theta = S->theta; I->w_tilde = S->w_tilde; I->w_check = S->w_check; I->w_bar = S->w_bar;
  I->w_grave = S->w_grave; I->w_hat = S->w_hat; I->w_z = S->w_z; I->w_out = S->w_out;
  I->phi_check = S->phi_check; I->phi_hat = S->phi_hat; I->phi_z = S->phi_z; I->E = S->E; I->tot = S->tot;
  I->t = S->t; I->take_hat = S->take_hat; I->done = S->done; I->nonfinite = S->nonfinite;
  I->max_iter = S->max_iter; I->kg = S->kg; I->ticket = 0;
}

__global__ void cl_exit_kernel(const BInst* I, DevState* S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  S->theta = I->theta; S->w_tilde = I->w_tilde; S->w_check = I->w_check; S->w_bar = I->w_bar;
  S->w_grave = I->w_grave; S->w_hat = I->w_hat; S->w_z = I->w_z; S->w_out = I->w_out;
  S->phi_check = I->phi_check; S->phi_hat = I->phi_hat; S->phi_z = I->phi_z; S->E = I->E; S->tot = I->tot;
  S->t = I->t; S->take_hat = I->take_hat; S->done = I->done; S->nonfinite = I->nonfinite; S->kg = I->kg;
}

template <int KIND, int VV, int DM, bool VEC>
cudaError_t cl_launch(const PassDesc& P, const BatchPass& B, const BVecs& V, int ncta, int iters, int greedy,
                      int first, cudaStream_t st) {
  auto kern = cl_loop_kernel<KIND, VV, DM, VEC>;
  if (ncta > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ncta, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ncta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, P, B, V, iters, greedy, first);
}

// Largest cluster (16, else 8) that can be resident for this kernel, 0 if none.
template <int KIND, int VV, int DM, bool VEC>
int cl_max_cluster() {
  auto kern = cl_loop_kernel<KIND, VV, DM, VEC>;
  for (int c : {16, 8}) {
    if (c > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) return c;
    cudaGetLastError();
  }
  return 0;
}

}  // namespace

namespace pot {

int cluster_loop_kind(const PassDesc& P) {
  if (P.kind == COST_DENSE_F32)   // 1: 16-byte row loads; 3: scalar loads
    return (P.ldc % 4 == 0 && (uintptr_t)P.C % 16 == 0) ? 1 : 3;
  if (P.kind == COST_SQEUCLID_F32 && P.d >= 1 && P.d <= 4) return 2;
  return 0;
}

int cluster_loop_size(const PassDesc& P, int V) {
  static int cache[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};
  const int kind = cluster_loop_kind(P);
  if (kind == 0 || (V != 1 && V != 2)) return 0;
  int& c = cache[kind - 1][V - 1];
  if (c < 0) {
    if (kind == 1) c = (V == 1) ? cl_max_cluster<COST_DENSE_F32, 1, 0, true>() : cl_max_cluster<COST_DENSE_F32, 2, 0, true>();
    else if (kind == 3) c = (V == 1) ? cl_max_cluster<COST_DENSE_F32, 1, 0, false>() : cl_max_cluster<COST_DENSE_F32, 2, 0, false>();
    else c = (V == 1) ? cl_max_cluster<COST_SQEUCLID_F32, 1, 4, false>() : cl_max_cluster<COST_SQEUCLID_F32, 2, 4, false>();
  }
  return c;
}

cudaError_t launch_cluster_enter(BInst* I, const DevState* S, cudaStream_t st) {
  cl_enter_kernel<<<1, 32, 0, st>>>(I, S);
  return cudaGetLastError();
}

cudaError_t launch_cluster_exit(const BInst* I, DevState* S, cudaStream_t st) {
  cl_exit_kernel<<<1, 32, 0, st>>>(I, S);
  return cudaGetLastError();
}

cudaError_t launch_cluster_loop(const ClusterLoop& A, int iters, int greedy, int first, cudaStream_t st) {
  const PassDesc& P = A.P;
  BatchPass B{};
  B.kind = P.kind; B.H = A.H; B.W = 128 * A.V; B.Ntot = P.n; B.Mtot = P.m;
  B.inst = A.inst; B.count = 1;
  B.xn = P.xn; B.yn = P.yn;
  B.rowA = P.rowA; B.colA = P.colA; B.colB = P.colB;
  B.row_part = P.row_part; B.col_part = P.col_part; B.red_part = P.red_part;
  B.aoff0 = -1; B.aoff1 = -1;
  BVecs V{};
  const AspotVecs& W = A.vecs;
  V.inst = A.inst;
  V.rt = const_cast<double*>(W.rt); V.ct = const_cast<double*>(W.ct);
  V.lrt = const_cast<double*>(W.lrt); V.lct = const_cast<double*>(W.lct);
  V.ut = W.ut; V.vt = W.vt; V.uc = W.uc; V.vc = W.vc; V.ub = W.ub; V.vb = W.vb;
  V.ug = W.ug; V.vg = W.vg; V.uh = W.uh; V.vh = W.vh; V.uo = W.uo; V.vo = W.vo;
  V.fc = nullptr; V.gc = nullptr;
  V.lrow = W.lrow; V.lcol = W.lcol;
  V.ndone = A.ndone;
  V.trace = nullptr;
  V.trace4 = A.trace4;
  const int kind = cluster_loop_kind(P);
  if (kind == 1)
    return A.V == 1 ? cl_launch<COST_DENSE_F32, 1, 0, true>(P, B, V, A.ncta, iters, greedy, first, st)
                    : cl_launch<COST_DENSE_F32, 2, 0, true>(P, B, V, A.ncta, iters, greedy, first, st);
  if (kind == 3)
    return A.V == 1 ? cl_launch<COST_DENSE_F32, 1, 0, false>(P, B, V, A.ncta, iters, greedy, first, st)
                    : cl_launch<COST_DENSE_F32, 2, 0, false>(P, B, V, A.ncta, iters, greedy, first, st);
  if (kind == 2)
    return A.V == 1 ? cl_launch<COST_SQEUCLID_F32, 1, 4, false>(P, B, V, A.ncta, iters, greedy, first, st)
                    : cl_launch<COST_SQEUCLID_F32, 2, 4, false>(P, B, V, A.ncta, iters, greedy, first, st);
  return cudaErrorInvalidValue;
}

}  // namespace pot
