// O(n + m) kernels around the passes: combining log-sum-exp partials, the
// dual updates of ASPOT (Algorithm 2) and of the feasible Sinkhorn baseline
// (Algorithm 3 on the extended kernel), the rounding reading R1-R4 and the
// scalar bookkeeping.  Potentials, updates and scalar sums are FP64; the
// combine of the passes' FP32 partials sums in FP32 (compensated) and takes
// its logarithm on an exact mantissa / exponent split.
//
// Scalar reductions are deterministic: every block writes its partial, the
// last block to finish (atomic ticket) sums the partials in block order and
// performs the scalar part of the update.
#include "common.cuh"
#include "kernels.h"

namespace pot {

namespace {

// Partials -> FP64 log-sums for rows and / or columns.  Block = 32 entries x
// 8 slices of the partials (coalesced: a warp reads 32 consecutive entries of
// one partial row); the slices meet in shared memory.
__global__ void combine_kernel(const float2* row_part, int64_t ncolblk, int64_t n, double* lrow,
                               const float2* col_part, int64_t nrowblk, int64_t m, double* lcol, int64_t nbr,
                               const int* done, const int* skip, int skip_if) {
  // no early release: the loop kernel that follows spreads its FP64 work one
  // block per SM, which holds only for blocks placed on an idle GPU
  pdl_wait();
  if ((done && *done) || (skip && *skip == skip_if)) return;
  __shared__ float sM[8][32], sS[8][32];
  const bool is_row = blockIdx.x < nbr;
  const float2* part = is_row ? row_part : col_part;
  const int64_t nblk = is_row ? ncolblk : nrowblk;
  const int64_t len = is_row ? n : m;
  double* out = is_row ? lrow : lcol;
  const int64_t blk = is_row ? blockIdx.x : blockIdx.x - nbr;
  const int jj = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int64_t j = blk * 32 + jj;
  float M = -INFINITY, S = 0.f;
  if (j < len) {
    for (int64_t b = sl; b < nblk; b += 8) {
      const float2 p = part[b * len + j];
      if (p.y > 0.f) M = fmaxf(M, p.x);
    }
    if (M > -INFINITY)
      for (int64_t b = sl; b < nblk; b += 8) {
        const float2 p = part[b * len + j];
        if (p.y > 0.f) S = fmaf(p.y, ex2(p.x - M), S);
      }
  }
  sM[sl][jj] = M;
  sS[sl][jj] = S;
  __syncthreads();
  if (sl == 0 && j < len) {
    float Mt = -INFINITY;
#pragma unroll
    for (int k = 0; k < 8; ++k) Mt = fmaxf(Mt, sM[k][jj]);
    // compensated (Kahan) FP32 sum of the eight slices' sum * 2^(max - Mt)
    float St = 0.f, comp = 0.f;
    if (Mt > -INFINITY) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (sS[k][jj] > 0.f) {
          const float y = sS[k][jj] * ex2(sM[k][jj] - Mt) - comp;
          const float t = St + y;
          comp = (t - St) - y;
          St = t;
        }
    }
    out[j] = St > 0.f ? log_shifted_sum(Mt, St) : POT_NEG_BIG;
  }
}

// Warp sums of NV <= 4 values by a transposing butterfly: at the first
// levels each lane keeps half of its values and adds its partner's copies of
// them, so the four sums take 6 FP64 additions per lane instead of 20 (a
// warp-wide FP64 instruction holds an SM sub-partition for dozens of cycles
// on this GPU).  Value k's total ends in lane sum_lane<NV>(k); other NV use
// one butterfly per value (total in lane 0).
template <int NV>
__device__ __forceinline__ int sum_lane(int k) { return NV <= 1 ? 0 : (NV == 2 ? 16 * k : 8 * k); }
template <int NV>
__device__ __forceinline__ void warp_sums(double (&v)[NV], int lane) {
  if constexpr (NV == 1) {
    v[0] = warp_sum_d(v[0]);
  } else if constexpr (NV == 2) {
    const bool up = lane & 16;
    double keep = up ? v[1] : v[0];
    keep += __shfl_xor_sync(0xffffffffu, up ? v[0] : v[1], 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
    v[0] = v[1] = keep;              // lanes 0..15 hold sum 0, lanes 16..31 sum 1
  } else if constexpr (NV == 3 || NV == 4) {
    const double v3 = NV == 4 ? v[NV - 1] : 0.0;
    const bool up = lane & 16;
    double k0 = up ? v[2] : v[0], k1 = up ? v3 : v[1];
    k0 += __shfl_xor_sync(0xffffffffu, up ? v[0] : v[2], 16);
    k1 += __shfl_xor_sync(0xffffffffu, up ? v[1] : v3, 16);
    const bool up8 = lane & 8;
    double keep = up8 ? k1 : k0;
    keep += __shfl_xor_sync(0xffffffffu, up8 ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = keep;   // lanes 8k .. 8k+7 hold sum k
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum_d(v[k]);
  }
}
template <int NV>
__device__ __forceinline__ bool holds_sum(int lane, int k) {
  return (NV == 1 || NV > 4) ? lane == 0 : lane == sum_lane<NV>(k);
}

template <int NV>
__device__ bool reduce_last(const double (&v)[NV], double* part, unsigned int* counter, double (&tot)[NV]) {
  __shared__ double sh[NV][kVecThreads / 32];
  __shared__ double st[NV];
  __shared__ int amlast;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  double w[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) w[k] = v[k];
  warp_sums<NV>(w, lane);
#pragma unroll
  for (int k = 0; k < NV; ++k)
    if (holds_sum<NV>(lane, k)) sh[k][warp] = w[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[k][w];
      part[(int64_t)blockIdx.x * NV + k] = s;
    }
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    amlast = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  // value pairs (k, k + nw) per warp, summed together by the transposing butterfly
  for (int k = warp; k < NV; k += 2 * nw) {
    const int k2 = k + nw;
    double s2[2] = {0.0, 0.0};
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      s2[0] += __ldcg(part + (int64_t)b * NV + k);
      if (k2 < NV) s2[1] += __ldcg(part + (int64_t)b * NV + k2);
    }
    warp_sums<2>(s2, lane);
    if (lane == sum_lane<2>(0)) st[k] = s2[0];
    if (k2 < NV && lane == sum_lane<2>(1)) st[k2] = s2[1];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = st[k];
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// NV sums plus one log-sum-exp over the grid: each thread contributes v[] and
// (x, active) to log sum exp(x).  The last block gets the totals (sums in
// block order, the log-sum-exp in natural log).
template <int NV>
__device__ bool reduce_last_lse(const double (&v)[NV], double x, bool active, double* part,
                                unsigned int* counter, double (&tot)[NV], double* lse_out, bool lse_on = true) {
  // lse_on (the same in every thread): whether the log-sum-exp is wanted at
  // all; when not, its FP64 maxima, exponentials and logarithm are skipped
  // and *lse_out is log 0
  constexpr int NW = kVecThreads / 32;
  constexpr int NP = NV + 2;
  __shared__ double sh[NV > 0 ? NV : 1][NW];
  __shared__ double smx[NW], ssm[NW];
  __shared__ double st[NV > 0 ? NV : 1];
  __shared__ double slse;
  __shared__ int amlast;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  double w[NV > 0 ? NV : 1];
#pragma unroll
  for (int k = 0; k < NV; ++k) w[k] = v[k];
  if constexpr (NV > 0) warp_sums<NV>(w, lane);
#pragma unroll
  for (int k = 0; k < NV; ++k)
    if (holds_sum<NV>(lane, k)) sh[k][warp] = w[k];
  double mx = -INFINITY, sm = 0.0;
  if (lse_on) {
    mx = active ? x : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sm = (active && mx > -INFINITY) ? exp(x - mx) : 0.0;
    sm = warp_sum_d(sm);
  }
  if (lane == 0) { smx[warp] = mx; ssm[warp] = sm; }
  __syncthreads();
  if (warp == 0) {
    // block (max, sum) of the NW warp partials: one exp per lane, not a serial chain
    double bm = -INFINITY, bs = 0.0;
    if (lse_on) {
      const double wm = (lane < nw && ssm[lane] > 0.0) ? smx[lane] : -INFINITY;
      bm = wm;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
      bs = (wm > -INFINITY) ? ssm[lane] * exp(wm - bm) : 0.0;
      bs = warp_sum_d(bs);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += sh[k][w];
        part[(int64_t)blockIdx.x * NP + k] = a;
      }
      part[(int64_t)blockIdx.x * NP + NV] = bs > 0.0 ? bm : -INFINITY;
      part[(int64_t)blockIdx.x * NP + NV + 1] = bs;
      __threadfence();
      const unsigned prev = atomicAdd(counter, 1u);
      amlast = (prev == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  // value pairs (k, k + nw) per warp, summed together by the transposing butterfly
  for (int k = warp; k < NV; k += 2 * nw) {
    const int k2 = k + nw;
    double a2[2] = {0.0, 0.0};
    for (int b2 = lane; b2 < (int)gridDim.x; b2 += 32) {
      a2[0] += __ldcg(part + (int64_t)b2 * NP + k);
      if (k2 < NV) a2[1] += __ldcg(part + (int64_t)b2 * NP + k2);
    }
    warp_sums<2>(a2, lane);
    if (lane == sum_lane<2>(0)) st[k] = a2[0];
    if (k2 < NV && lane == sum_lane<2>(1)) st[k2] = a2[1];
  }
  if (lse_on) {
    // grid log-sum-exp of the block partials, in parallel over the block's threads
    double gm = -INFINITY;
    for (int b2 = threadIdx.x; b2 < (int)gridDim.x; b2 += blockDim.x)
      if (__ldcg(part + (int64_t)b2 * NP + NV + 1) > 0.0) gm = fmax(gm, __ldcg(part + (int64_t)b2 * NP + NV));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if (lane == 0) smx[warp] = gm;
    __syncthreads();
    gm = -INFINITY;
    for (int w = 0; w < nw; ++w) gm = fmax(gm, smx[w]);
    double gs = 0.0;
    if (gm > -INFINITY)
      for (int b2 = threadIdx.x; b2 < (int)gridDim.x; b2 += blockDim.x) {
        const double ss = __ldcg(part + (int64_t)b2 * NP + NV + 1);
        if (ss > 0.0) gs += ss * exp(__ldcg(part + (int64_t)b2 * NP + NV) - gm);
      }
    gs = warp_sum_d(gs);
    if (lane == 0) ssm[warp] = gs;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) a += ssm[w];
      slse = (gm > -INFINITY && a > 0.0) ? gm + log(a) : POT_NEG_BIG;
    }
  } else if (threadIdx.x == 0) {
    slse = POT_NEG_BIG;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = st[k];
  *lse_out = slse;
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

__device__ __forceinline__ double clamp_log(double x) { return x > POT_NEG_BIG ? x : POT_NEG_BIG; }
__device__ __forceinline__ double safe_exp(double x) { return x > -700.0 ? exp(x) : 0.0; }

// FP64 log-sum of entry j from the nblk (max, sum) partials of a pass (the
// arithmetic of combine_kernel, one thread per entry): the loop kernels of the
// solvers call it instead of a separate combine launch.
// NB >= nblk: every partial is loaded at once (NB independent loads in
// flight, predicated past nblk) and kept in registers for the two sweeps, the
// same arithmetic in the same order as the streaming form below, without its
// chain of dependent loads.
template <int NB>
__device__ __forceinline__ double comb_part_regs(const float2* part, int64_t nblk, int64_t len, int64_t j) {
  float2 p[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) p[b] = (b < nblk) ? part[b * len + j] : make_float2(0.f, 0.f);
  float M = -INFINITY;
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (p[b].y > 0.f) M = fmaxf(M, p[b].x);
  if (!(M > -INFINITY)) return POT_NEG_BIG;
  float St = 0.f, comp = 0.f;
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (p[b].y > 0.f) {
      const float y = p[b].y * ex2(p[b].x - M) - comp;
      const float t = St + y;
      comp = (t - St) - y;
      St = t;
    }
  return St > 0.f ? log_shifted_sum(M, St) : POT_NEG_BIG;
}
__device__ double comb_part(const float2* part, int64_t nblk, int64_t len, int64_t j) {
  if (nblk <= 16) return comb_part_regs<16>(part, nblk, len, j);
  if (nblk <= 32) return comb_part_regs<32>(part, nblk, len, j);
  float M = -INFINITY;
  for (int64_t b = 0; b < nblk; ++b) {
    const float2 p = part[b * len + j];
    if (p.y > 0.f) M = fmaxf(M, p.x);
  }
  if (!(M > -INFINITY)) return POT_NEG_BIG;
  float St = 0.f, comp = 0.f;
  for (int64_t b = 0; b < nblk; ++b) {
    const float2 p = part[b * len + j];
    if (p.y > 0.f) {
      const float y = p.y * ex2(p.x - M) - comp;
      const float t = St + y;
      comp = (t - St) - y;
      St = t;
    }
  }
  return St > 0.f ? log_shifted_sum(M, St) : POT_NEG_BIG;
}
template <class Vecs>
__device__ __forceinline__ double row_sum_of(const Vecs& V, int64_t i, bool from_parts) {
  if (!from_parts) return V.lrow[i];
  const double R = comb_part(V.row_part, V.ncolblk, V.n, i);
  const_cast<double*>(V.lrow)[i] = R;         // later kernels of the iteration read it
  return R;
}
template <class Vecs>
__device__ __forceinline__ double col_sum_of(const Vecs& V, int64_t j, bool from_parts) {
  if (!from_parts) return V.lcol[j];
  const double C = comb_part(V.col_part, V.nrowblk, V.m, j);
  const_cast<double*>(V.lcol)[j] = C;
  return C;
}

// ----------------------------------------------------------- prologue ---

__global__ void marg_stats_kernel(const double* r, const double* c, int64_t n, int64_t m, double* part,
                                  unsigned int* counter, double* out) {
  // out: [sum r, sum c, min r, min c, #nonfinite-or-negative, 0]
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[4] = {0, 0, 0, 0};
  double mnr = INFINITY, mnc = INFINITY;
  if (t < n) { const double x = r[t]; v[0] = x; mnr = x; if (!(x >= 0.0) || !isfinite(x)) v[2] = 1; }
  else if (t < n + m) { const double x = c[t - n]; v[1] = x; mnc = x; if (!(x >= 0.0) || !isfinite(x)) v[2] = 1; }
  // minima through the sum slot trick: reduce -min separately
  __shared__ double smr[kVecThreads / 32], smc[kVecThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mnr = fmin(mnr, __shfl_xor_sync(0xffffffffu, mnr, o));
    mnc = fmin(mnc, __shfl_xor_sync(0xffffffffu, mnc, o));
  }
  if (lane == 0) { smr[warp] = mnr; smc[warp] = mnc; }
  __syncthreads();
  double bmr = INFINITY, bmc = INFINITY;
  for (int w = 0; w < kVecThreads / 32; ++w) { bmr = fmin(bmr, smr[w]); bmc = fmin(bmc, smc[w]); }
  // store block minima in dedicated slots after the sums (part has 6 per block)
  double tot[3];
  double vv[3] = {v[0], v[1], v[2]};
  if (threadIdx.x == 0) { part[(int64_t)gridDim.x * 3 + 2 * blockIdx.x] = bmr; part[(int64_t)gridDim.x * 3 + 2 * blockIdx.x + 1] = bmc; }
  if (reduce_last<3>(vv, part, counter, tot)) {
    if (threadIdx.x == 0) {
      double mr = INFINITY, mc = INFINITY;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        mr = fmin(mr, __ldcg(part + (int64_t)gridDim.x * 3 + 2 * b));
        mc = fmin(mc, __ldcg(part + (int64_t)gridDim.x * 3 + 2 * b + 1));
      }
      out[0] = tot[0]; out[1] = tot[1]; out[2] = mr; out[3] = mc; out[4] = tot[2]; out[5] = 0.0;
    }
  }
}

__global__ void reduce_parts_kernel(const double* part, int64_t count, int op_max, double* out) {
  __shared__ double sh[32];
  double acc = op_max ? -INFINITY : 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
    const double x = part[i];
    acc = op_max ? nanmax(acc, x) : acc + x;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, acc, o);
    acc = op_max ? nanmax(acc, y) : acc + y;
  }
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = op_max ? -INFINITY : 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) a = op_max ? nanmax(a, sh[w]) : a + sh[w];
    *out = a;
  }
}

// --------------------------------------------------------------- ASPOT ---

// Algorithm 2 setup: smoothed marginals r~ = (1 - e/8) r + e/(8n), their
// logs, and the starting point z~^0 = z_check^0 (zero or a warm start).
__global__ void aspot_init_kernel(AspotVecs V, const double* r, const double* c, double eps_s,
                                  const double* u0, const double* v0, double w0) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double* rt = const_cast<double*>(V.rt);
  double* ct = const_cast<double*>(V.ct);
  double* lrt = const_cast<double*>(V.lrt);
  double* lct = const_cast<double*>(V.lct);
  if (t < V.n) {
    const double x = (1.0 - eps_s / 8.0) * r[t] + eps_s / (8.0 * (double)V.n);
    rt[t] = x; lrt[t] = x > 0.0 ? log(x) : POT_NEG_BIG;
    const double z = u0 ? u0[t] : 0.0;
    V.ut[t] = z; V.uc[t] = z; V.uo[t] = z;
  } else if (t < V.n + V.m) {
    const int64_t j = t - V.n;
    const double x = (1.0 - eps_s / 8.0) * c[j] + eps_s / (8.0 * (double)V.m);
    ct[j] = x; lct[j] = x > 0.0 ? log(x) : POT_NEG_BIG;
    const double z = v0 ? v0[j] : 0.0;
    V.vt[j] = z; V.vc[j] = z; V.vo[j] = z;
  }
  if (t == 0) {
    DevState* S = V.S;
    S->w_tilde = w0; S->w_check = w0; S->w_out = w0; S->w_z = w0;
    S->theta = 1.0; S->t = 0; S->done = 0; S->take_hat = 0; S->nonfinite = 0;
    S->E = INFINITY;
  }
}

// z_bar = (1 - theta) z_check + theta z~
__global__ void aspot_extrap_kernel(AspotVecs V) {
  pdl_enter();
  DevState* S = V.S;
  if (S->done) return;
  const double th = S->theta;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < V.n) V.ub[t] = (1.0 - th) * V.uc[t] + th * V.ut[t];
  else if (t < V.n + V.m) V.vb[t - V.n] = (1.0 - th) * V.vc[t - V.n] + th * V.vt[t - V.n];
  if (t == 0) S->w_bar = (1.0 - th) * S->w_check + th * S->w_tilde;
}

// After the fused pass at z_bar: gradient (r(B)+e^u-r~, c(B)+e^v-c~, |B|-s),
// step z~' = z_bar - grad/(L theta), coupling z_grave = z_bar + theta (z~' - z~).
__global__ void aspot_after_grad_kernel(AspotVecs V) {
  pdl_enter();
  DevState* S = V.S;
  // every operand in one round of loads, the stop flag among them (a loop
  // kernel's time is a few dependent rounds of loads plus its FP64 chain)
  const int done = S->done;
  const double th = S->theta, L = S->L;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool row = t < V.n, col = !row && t < V.n + V.m;
  const int64_t j = t - V.n;
  double z = 0.0, zt = 0.0, a = 0.0, R = 0.0;   // potential at z_bar, z~, marginal, log-sum
  if (row) {
    z = V.ub[t]; zt = V.ut[t]; a = V.rt[t];
    R = V.fused ? comb_part(V.row_part, V.ncolblk, V.n, t) : V.lrow[t];
  } else if (col) {
    z = V.vb[j]; zt = V.vt[j]; a = V.ct[j];
    R = V.fused ? comb_part(V.col_part, V.nrowblk, V.m, j) : V.lcol[j];
  }
  if (done) return;
  const double Lth = L * th;
  double v[3] = {0, 0, 0};   // tot, sum(e^u - u r~) + sum(e^v - v c~), nonfinite
  if (row) {
    if (V.fused) const_cast<double*>(V.lrow)[t] = R;    // later kernels of the iteration read it
    const double rB = exp_sum(R), eu = safe_exp(z);
    const double g = rB + eu - a;
    const double un = z - g / Lth;
    V.ug[t] = z + th * (un - zt);
    V.ut[t] = un;
    v[0] = rB;
    v[1] = eu - z * a;
    if (!isfinite(un)) v[2] = 1;
  } else if (col) {
    if (V.fused) const_cast<double*>(V.lcol)[j] = R;
    const double cB = exp_sum(R), ev = safe_exp(z);
    const double g = cB + ev - a;
    const double vn = z - g / Lth;
    V.vg[j] = z + th * (vn - zt);
    V.vt[j] = vn;
    v[1] = ev - z * a;
    if (!isfinite(vn)) v[2] = 1;
  }
  double tot[3];
  if (reduce_last<3>(v, V.red, V.counter, tot) && threadIdx.x == 0) {
    const double gw = tot[0] - S->s;
    const double wn = S->w_bar - gw / Lth;
    S->w_grave = S->w_bar + th * (wn - S->w_tilde);
    S->w_tilde = wn;
    // theta_{t+1} once here: the final kernel needs it in every thread (for
    // z_bar^{t+1}), where an FP64 square root per thread would be costly
    S->theta_next = th * (sqrt(th * th + 4.0) - th) / 2.0;
    if (S->t == 0) S->phi_check = tot[0] + tot[1] - S->w_bar * S->s;   // phi(z_check^0), z_bar^0 = z_check^0
    if (tot[2] != 0.0 || !isfinite(wn)) S->nonfinite = 1;
  }
}

// After the one-sided pass at z_grave: Greenkhorn step (Algorithm 1) for block
// k, closed-form phi(z^), argmin against phi(z_check).  k < 0: the greedy
// rule's block S->kg (the pass was two-sided); z^ is then written whole to
// (uh, vh), and the flags of the one-sided passes at z^t are set.
__global__ void aspot_after_greenkhorn_kernel(AspotVecs V, int k) {
  pdl_enter();
  DevState* S = V.S;
  // every operand in one round of loads (the greedy rule's block index one
  // round earlier), the stop flag among them
  const int done = S->done;
  const bool greedy = k < 0;
  if (greedy) k = S->kg;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool row = t < V.n, col = !row && t < V.n + V.m;
  const int64_t j = t - V.n;
  const bool comb = V.fused && !greedy;     // greedy: the block choice kernel combined them
  // the side's potential at z_grave, marginal and its log; the side's log-sum
  // where block k needs it (rows: u- and w-steps; columns: v-step, and the
  // w-step's combine for the closed forms of the final kernel)
  double zg = 0.0, a = 0.0, la = 0.0, R = 0.0;
  const bool need = row ? (k == 0 || k == 2) : (col && (k == 1 || (comb && k == 2)));
  if (row) {
    zg = V.ug[t]; a = V.rt[t]; la = V.lrt[t];
    if (need) R = comb ? comb_part(V.row_part, V.ncolblk, V.n, t) : V.lrow[t];
  } else if (col) {
    zg = V.vg[j]; a = V.ct[j]; la = V.lct[j];
    if (need) R = comb ? comb_part(V.col_part, V.nrowblk, V.m, j) : V.lcol[j];
  }
  if (done) return;
  double v[2] = {0, 0};      // phi parts
  double xr = 0.0;           // log row sum (w step: log |B|_1 = LSE_i of these)
  bool act = false;
  if (row) {
    if (need && comb) const_cast<double*>(V.lrow)[t] = R;   // later kernels of the iteration read it
    if (k == 0) {
      const double uh = la - softplus(R - zg);
      V.uh[t] = uh;
      v[0] = -uh * a;
    } else {
      v[0] = safe_exp(zg) - zg * a;
      if (k == 2) { xr = R; act = true; }
      if (greedy) V.uh[t] = zg;
    }
  } else if (col) {
    if (need && comb) const_cast<double*>(V.lcol)[j] = R;
    if (k == 1) {
      const double vh = la - softplus(R - zg);
      V.vh[j] = vh;
      v[1] = -vh * a;
    } else {
      v[1] = safe_exp(zg) - zg * a;
      if (greedy) V.vh[j] = zg;
    }
  }
  double tot[2], ltot = 0.0;
  if (reduce_last_lse<2>(v, xr, act, V.red, V.counter, tot, &ltot, k == 2) && threadIdx.x == 0) {
    double wh = S->w_grave, base;
    if (k == 0) base = S->sum_rt;                 // |B|_1 + sum e^u = |r~|_1 after the u step
    else if (k == 1) base = S->sum_ct;
    else { wh = S->w_grave + S->log_s - ltot; base = S->s; }   // |B|_1 = s after the w step
    S->w_hat = wh;
    const double ph = base + tot[0] + tot[1] - wh * S->s;
    S->phi_hat = ph;
    const int take = ph < S->phi_check;
    S->take_hat = take;
    S->phi_z = take ? ph : S->phi_check;
    S->w_z = take ? wh : S->w_check;
    if (greedy) {
      // at z^t = z^ the side of block k follows in closed form: a rows pass
      // is needed after a v-step, a columns pass after a u-step, none after a
      // w-step; at z^t = z_check both sides are computed
      S->run_r3 = take && k == 1;
      S->run_c3 = take && k == 0;
    }
  }
}

// After the fused pass at z^t: E_t, z_check^{t+1} = Greenkhorn_k(z^t),
// closed-form phi(z_check^{t+1}), theta update and the stop test.
__global__ void aspot_after_final_kernel(AspotVecs V, int k) {
  pdl_enter();
  DevState* S = V.S;
  // every operand in one round of loads, the stop flag and the argmin among
  // them: both candidates for z^t and both sources of its sums are read, then
  // selected
  const int done = S->done, take = S->take_hat;
  const double w_hat = S->w_hat, w_grave = S->w_grave;
  // theta_{t+1} (formed by the gradient kernel of this iteration): the
  // extrapolation z_bar^{t+1} of the next iteration is formed here
  const double thn = S->theta_next;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool row = t < V.n, col = !row && t < V.n + V.m;
  const int64_t j = t - V.n;
  // side of the entry: potential of z^ (block k's Greenkhorn step or z_grave),
  // of z_check, z^ and z_grave of block k's side, marginal, its log, z~
  double zh = 0.0, zc = 0.0, zhk = 0.0, zgk = 0.0, a = 0.0, la = 0.0, zt = 0.0, Rp = 0.0, Rl = 0.0;
  bool parts = false;        // the sums at z^t come from the pass (else in closed form from P2)
  if (row) {
    zh = (k == 0) ? V.uh[t] : V.ug[t]; zc = V.uc[t]; a = V.rt[t]; la = V.lrt[t]; zt = V.ut[t];
    if (k == 0) { zhk = V.uh[t]; zgk = V.ug[t]; }
    if (V.fused) Rp = comb_part(V.row_part, V.ncolblk, V.n, t);
    Rl = V.lrow[t];
  } else if (col) {
    zh = (k == 1) ? V.vh[j] : V.vg[j]; zc = V.vc[j]; a = V.ct[j]; la = V.lct[j]; zt = V.vt[j];
    if (k == 1) { zhk = V.vh[j]; zgk = V.vg[j]; }
    if (V.fused) Rp = comb_part(V.col_part, V.nrowblk, V.m, j);
    Rl = V.lcol[j];
  }
  if (done) return;
  double v[4] = {0, 0, 0, 0};   // Eu+Ev, tot, phi parts, nonfinite
  double xr = 0.0;
  bool act = false;
  // z^t = z^: the sums of block k's side come from the Greenkhorn pass at
  // z_grave in closed form (the other side was computed at z^ by P3a)
  const double dw = (take && k == 2) ? w_hat - w_grave : 0.0;
  if (row) {
    const double uz = take ? zh : zc;
    // rows: from the pass at z^t (P3a for k = 1, P3b when z^t = z_check), else closed form
    parts = V.fused && (k == 1 || !take);
    double R = parts ? Rp : Rl;
    if (parts) const_cast<double*>(V.lrow)[t] = Rp;
    if (take && k == 0) R = clamp_log(R + (zhk - zgk));
    else if (take && k == 2) R = clamp_log(R + dw);
    xr = R;
    act = k == 2;                      // log |B|_1 is needed by the w step only
    const double rB = exp_sum(R), eu = safe_exp(uz);
    v[0] = fabs(rB + eu - a);
    v[1] = rB;
    V.uo[t] = uz;
    const double un = (k == 0) ? la - softplus(R - uz) : uz;
    V.uc[t] = un;
    V.ub[t] = (1.0 - thn) * un + thn * zt;
    v[2] = (k == 0) ? -un * a : eu - un * a;    // un = uz unless k = 0
    if (!isfinite(R) && R != POT_NEG_BIG) v[3] = 1;
  } else if (col) {
    const double vz = take ? zh : zc;
    parts = V.fused && (k == 0 || !take);
    double Cc = parts ? Rp : Rl;
    if (parts) const_cast<double*>(V.lcol)[j] = Rp;
    if (take && k == 1) Cc = clamp_log(Cc + (zhk - zgk));
    else if (take && k == 2) Cc = clamp_log(Cc + dw);
    const double cB = exp_sum(Cc), ev = safe_exp(vz);
    v[0] = fabs(cB + ev - a);
    V.vo[j] = vz;
    const double vn = (k == 1) ? la - softplus(Cc - vz) : vz;
    V.vc[j] = vn;
    V.vb[j] = (1.0 - thn) * vn + thn * zt;
    v[2] = (k == 1) ? -vn * a : ev - vn * a;    // vn = vz unless k = 1
    if (!isfinite(Cc) && Cc != POT_NEG_BIG) v[3] = 1;
  }
  double tot[4], ltot = 0.0;
  if (reduce_last_lse<4>(v, xr, act, V.red, V.counter, tot, &ltot, k == 2) && threadIdx.x == 0) {
    const double s = S->s;
    const double E = fabs(tot[1] - s) + tot[0];
    const double wz = S->w_z;
    S->w_out = wz;
    double wc = wz, base;
    if (k == 0) base = S->sum_rt;
    else if (k == 1) base = S->sum_ct;
    else { wc = wz + S->log_s - ltot; base = s; }   // log |B|_1 in the log domain (it may underflow)
    S->w_check = wc;
    S->phi_check = base + tot[2] - wc * s;
    S->E = E;
    S->tot = tot[1];
    const int it = S->t;
    if (V.trace) {
      double* tr = S->trace[it & 4095];
      tr[0] = E; tr[1] = S->phi_z; tr[2] = S->phi_check; tr[3] = (double)take;
    }
    S->theta = thn;
    S->w_bar = (1.0 - thn) * wc + thn * S->w_tilde;
    S->t = it + 1;
    if (tot[3] != 0.0 || !isfinite(E)) S->nonfinite = 1;
    if (E <= S->thr || it + 1 >= S->max_iter || S->nonfinite) S->done = 1;
  }
}

// ------------------------------------------------- greedy block rule ---
// The block choice of Theorem 3's analysis: the block whose Greenkhorn step
// decreases phi the most.  Those decreases are exact in closed form,
//   D_u = sum_i rho(r~_i, r_i(B) + e^{u_i}),  D_v = sum_j rho(c~_j, c_j(B) + e^{v_j}),
//   D_w = rho(s, |B|_1),                       rho(a, b) = b - a + a log(a / b),
// so one two-sided pass at the point scores all three.  Ties go to the lower
// block index.

// rho(a, b) from log a and log b
__device__ __forceinline__ double rho_log(double a, double la, double lb) {
  return safe_exp(lb) - a + (a > 0.0 ? a * (la - lb) : 0.0);
}
__device__ __forceinline__ int pick_block(double du, double dv, double dw) {
  int k = 0;
  double best = du;
  if (dv > best) { k = 1; best = dv; }
  if (dw > best) k = 2;
  return k;
}

// After the two-sided pass at z_grave: S->kg = argmax of the decreases there.
__global__ void aspot_greedy_pick_kernel(AspotVecs V) {
  pdl_enter();
  DevState* S = V.S;
  if (S->done) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  double xr = 0.0;
  bool act = false;
  if (t < V.n) {
    const double R = row_sum_of(V, t, V.fused);
    v[0] = rho_log(V.rt[t], V.lrt[t], logaddexp(R, V.ug[t]));
    xr = R;
    act = true;
  } else if (t < V.n + V.m) {
    const int64_t j = t - V.n;
    v[1] = rho_log(V.ct[j], V.lct[j], logaddexp(col_sum_of(V, j, V.fused), V.vg[j]));
  }
  double tot[2], ltot = 0.0;
  if (reduce_last_lse<2>(v, xr, act, V.red, V.counter, tot, &ltot) && threadIdx.x == 0)
    S->kg = pick_block(tot[0], tot[1], rho_log(S->s, S->log_s, ltot));
}

// Sums of B(z^t) on both sides: from the passes at z^t, or in closed form
// from the pass at z_grave for the side of the block just stepped (as in
// aspot_after_final_kernel).
__device__ __forceinline__ double greedy_row_sum(const AspotVecs& V, int64_t i, int k, int take, double dw,
                                                 bool from_parts = false) {
  double R = row_sum_of(V, i, from_parts);
  if (take && k == 0) R = clamp_log(R + (V.uh[i] - V.ug[i]));
  else if (take && k == 2) R = clamp_log(R + dw);
  return R;
}
__device__ __forceinline__ double greedy_col_sum(const AspotVecs& V, int64_t j, int k, int take, double dw,
                                                 bool from_parts = false) {
  double Cc = col_sum_of(V, j, from_parts);
  if (take && k == 1) Cc = clamp_log(Cc + (V.vh[j] - V.vg[j]));
  else if (take && k == 2) Cc = clamp_log(Cc + dw);
  return Cc;
}

// After the passes at z^t (greedy rule): E_t, the block k2 of the second
// Greenkhorn step (argmax of the decreases at z^t), phi(z_check^{t+1}) for
// that block, theta update and the stop test.  z^t is written to (uo, vo);
// aspot_greedy_apply_kernel then forms z_check^{t+1}.
__global__ void aspot_greedy_final_kernel(AspotVecs V) {
  pdl_enter();
  DevState* S = V.S;
  if (S->done) return;
  const int k = S->kg, take = S->take_hat;
  const double dw = (take && k == 2) ? S->w_hat - S->w_grave : 0.0;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // E parts, |B|_1, D_u, D_v, phi parts: rows stepped / kept, columns stepped / kept, nonfinite
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double xr = 0.0;
  bool act = false;
  if (t < V.n) {
    const double uz = take ? V.uh[t] : V.uc[t];
    // from the passes at z^t (both sides at z_check, rows after a v-step) or closed form
    const double R = greedy_row_sum(V, t, k, take, dw, V.fused && (!take || k == 1));
    xr = R;
    act = true;
    const double rB = safe_exp(R), eu = safe_exp(uz), a = V.rt[t];
    v[0] = fabs(rB + eu - a);
    v[1] = rB;
    v[2] = rho_log(a, V.lrt[t], logaddexp(R, uz));
    v[4] = -(V.lrt[t] - softplus(R - uz)) * a;
    v[5] = eu - uz * a;
    V.uo[t] = uz;
    if (!isfinite(R) && R != POT_NEG_BIG) v[8] = 1;
  } else if (t < V.n + V.m) {
    const int64_t j = t - V.n;
    const double vz = take ? V.vh[j] : V.vc[j];
    const double Cc = greedy_col_sum(V, j, k, take, dw, V.fused && (!take || k == 0));
    const double cB = safe_exp(Cc), ev = safe_exp(vz), c = V.ct[j];
    v[0] = fabs(cB + ev - c);
    v[3] = rho_log(c, V.lct[j], logaddexp(Cc, vz));
    v[6] = -(V.lct[j] - softplus(Cc - vz)) * c;
    v[7] = ev - vz * c;
    V.vo[j] = vz;
    if (!isfinite(Cc) && Cc != POT_NEG_BIG) v[8] = 1;
  }
  double tot[9], ltot = 0.0;
  if (reduce_last_lse<9>(v, xr, act, V.red, V.counter, tot, &ltot) && threadIdx.x == 0) {
    const double s = S->s;
    const double E = fabs(tot[1] - s) + tot[0];
    const int k2 = pick_block(tot[2], tot[3], rho_log(s, S->log_s, ltot));
    const double wz = S->w_z;
    S->w_out = wz;
    double wc = wz, ph;
    if (k2 == 0) ph = S->sum_rt + tot[4] + tot[7] - wz * s;
    else if (k2 == 1) ph = S->sum_ct + tot[5] + tot[6] - wz * s;
    else { wc = wz + S->log_s - ltot; ph = s + tot[5] + tot[7] - wc * s; }
    S->k2 = k2;
    S->w_check = wc;
    S->phi_check = ph;
    S->E = E;
    S->tot = tot[1];
    const int it = S->t;
    if (V.trace) {
      double* tr = S->trace[it & 4095];
      tr[0] = E; tr[1] = S->phi_z; tr[2] = ph; tr[3] = (double)(take + 2 * k + 8 * k2);
    }
    const double th = S->theta;
    S->theta = th * (sqrt(th * th + 4.0) - th) / 2.0;
    S->t = it + 1;
    if (tot[8] != 0.0 || !isfinite(E)) S->nonfinite = 1;
    if (E <= S->thr || it + 1 >= S->max_iter || S->nonfinite) S->done = 1;
  }
}

// z_check^{t+1} = Greenkhorn_{k2}(z^t) (greedy rule); w_check was set by the
// final kernel.  It also runs in the iteration that set the stop flag (so an
// exported state holds z_check^{t+1}) and after it, where it rewrites the same
// values: it reads only z^t, the pass sums and scalars that no longer change.
__global__ void aspot_greedy_apply_kernel(AspotVecs V) {
  pdl_enter();
  DevState* S = V.S;
  const int k = S->kg, take = S->take_hat, k2 = S->k2;
  const double dw = (take && k == 2) ? S->w_hat - S->w_grave : 0.0;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double th = S->theta;               // theta_{t+1}: the extrapolation of the next iteration
  if (t < V.n) {
    const double uz = V.uo[t];
    const double un = (k2 == 0) ? V.lrt[t] - softplus(greedy_row_sum(V, t, k, take, dw) - uz) : uz;
    V.uc[t] = un;
    V.ub[t] = (1.0 - th) * un + th * V.ut[t];
  } else if (t < V.n + V.m) {
    const int64_t j = t - V.n;
    const double vz = V.vo[j];
    const double vn = (k2 == 1) ? V.lct[j] - softplus(greedy_col_sum(V, j, k, take, dw) - vz) : vz;
    V.vc[j] = vn;
    V.vb[j] = (1.0 - th) * vn + th * V.vt[j];
  }
  if (t == 0) S->w_bar = (1.0 - th) * S->w_check + th * S->w_tilde;
}

// Warm-start check.  E(z) = |r(B) + e^u - r~|_1 + |c(B) + e^v - c~|_1 + ||B|_1 - s|
// from the combined log-sums of a two-sided pass at z = (u, v, .); slot 0
// holds E at the given start, slot 1 E at zero.
__global__ void aspot_start_eval_kernel(AspotVecs V, const double* u, const double* v, int slot) {
  DevState* S = V.S;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double x[2] = {0.0, 0.0};   // l1 residual, |B|_1
  if (t < V.n) {
    const double rB = safe_exp(V.lrow[t]);
    x[0] = fabs(rB + safe_exp(u[t]) - V.rt[t]);
    x[1] = rB;
  } else if (t < V.n + V.m) {
    const int64_t j = t - V.n;
    x[0] = fabs(safe_exp(V.lcol[j]) + safe_exp(v[j]) - V.ct[j]);
  }
  double tot[2];
  if (reduce_last<2>(x, V.red, V.counter, tot) && threadIdx.x == 0) S->e_start[slot] = tot[0] + fabs(tot[1] - S->s);
}

// Zero dual point in the z_bar slots (the pass at z = 0 of the check).
__global__ void aspot_zero_bar_kernel(AspotVecs V) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < V.n) V.ub[t] = 0.0;
  else if (t < V.n + V.m) V.vb[t - V.n] = 0.0;
  if (t == 0) V.S->w_bar = 0.0;
}

// Keep the given start unless E(z_warm) > E(0) (or is not a number).
__global__ void aspot_start_select_kernel(AspotVecs V) {
  DevState* S = V.S;
  const bool warm = S->e_start[0] <= S->e_start[1];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!warm) {
    if (t < V.n) { V.ut[t] = 0.0; V.uc[t] = 0.0; V.uo[t] = 0.0; }
    else if (t < V.n + V.m) { const int64_t j = t - V.n; V.vt[j] = 0.0; V.vc[j] = 0.0; V.vo[j] = 0.0; }
  }
  if (t == 0) {
    if (!warm) { S->w_tilde = 0.0; S->w_check = 0.0; S->w_out = 0.0; S->w_z = 0.0; }
    S->warm_used = warm ? 1 : 0;
  }
}

// ---------------------------------------------------- feasible Sinkhorn ---

__global__ void sink_init_kernel(SinkVecs V, const double* r, const double* c, double eps_s, double s) {
  // r_ext = (r~, |c~| - s), c_ext = (c~, |r~| - s); sums come from S (raw masses)
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double* re = const_cast<double*>(V.re);
  double* ce = const_cast<double*>(V.ce);
  double* lre = const_cast<double*>(V.lre);
  double* lce = const_cast<double*>(V.lce);
  DevState* S = V.S;
  if (t < V.n) {
    const double x = (1.0 - eps_s / 8.0) * r[t] + eps_s / (8.0 * (double)V.n);
    re[t] = x; lre[t] = x > 0.0 ? log(x) : POT_NEG_BIG; V.u[t] = 0.0; V.uprev[t] = 0.0;
  } else if (t < V.n + V.m) {
    const int64_t j = t - V.n;
    const double x = (1.0 - eps_s / 8.0) * c[j] + eps_s / (8.0 * (double)V.m);
    ce[j] = x; lce[j] = x > 0.0 ? log(x) : POT_NEG_BIG; V.v[j] = 0.0;
  }
  if (t == 0) {
    const double dr = S->sum_ct - s, dc = S->sum_rt - s;
    re[V.n] = dr; lre[V.n] = dr > 0.0 ? log(dr) : POT_NEG_BIG;
    ce[V.m] = dc; lce[V.m] = dc > 0.0 ? log(dc) : POT_NEG_BIG;
    V.u[V.n] = 0.0; V.v[V.m] = 0.0; V.uprev[V.n] = 0.0;
    S->t = 0; S->done = 0; S->nonfinite = 0; S->E = INFINITY;
  }
}

// Row update of the extended kernel (u <- log r_ext - log(B 1 / e^u)) after
// a row pass; the l1 row residual of the current point is the stop test of
// the previous iteration (columns are exact right after a column update).
__global__ void sink_after_rows_kernel(SinkVecs V) {
  pdl_enter();
  DevState* S = V.S;
  if (S->done) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double vd = V.dcol ? V.v[V.m] : POT_NEG_BIG;
  double v[2] = {0, 0};      // l1 row residual, nonfinite
  double x = 0.0;
  bool act = false;
  if (t < V.n) {
    const double u = V.u[t];
    const double R = row_sum_of(V, t, V.fused);   // includes u_i
    const double lsum = V.dcol ? logaddexp(R, u + vd) : R;
    v[0] = fabs(safe_exp(lsum) - V.re[t]);
    V.uprev[t] = u;
    V.u[t] = clamp_log(V.lre[t] - (lsum - u));
    if (!isfinite(R) && R != POT_NEG_BIG) v[1] = 1;
  } else if (t < V.n + V.m) {
    x = V.v[t - V.n];       // log-sum-exp of v feeds the dummy row
    act = true;
  }
  double tot[2], lse_v = 0.0;
  if (reduce_last_lse<2>(v, x, act, V.red, V.counter, tot, &lse_v) && threadIdx.x == 0) {
    double res = tot[0];
    if (V.drow) {
      const double ud = V.u[V.n];
      const double lsum = V.dcol ? logaddexp(ud + lse_v, ud + vd - S->A_over_g) : ud + lse_v;
      res += fabs(safe_exp(lsum) - V.re[V.n]);
      V.uprev[V.n] = ud;
      V.u[V.n] = clamp_log(V.lre[V.n] - (lsum - ud));
    }
    S->E = res;
    if (tot[1] != 0.0 || !isfinite(res)) { S->nonfinite = 1; S->done = 3; }
    else if (S->t >= 1 && res <= S->thr) S->done = 2;   // 2: restore u from uprev
  }
}

// restore the pre-update row potentials when the stop test fired
__global__ void sink_restore_kernel(SinkVecs V) {
  pdl_enter();
  DevState* S = V.S;
  if (S->done != 2) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= V.n) V.u[t] = V.uprev[t];
}

__global__ void sink_after_cols_kernel(SinkVecs V) {
  pdl_enter();
  DevState* S = V.S;
  if (S->done) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double ud = V.drow ? V.u[V.n] : POT_NEG_BIG;
  double x = 0.0;
  bool act = false;
  if (t < V.m) {
    const double vj = V.v[t];
    const double Cc = col_sum_of(V, t, V.fused);   // includes v_j
    const double lsum = V.drow ? logaddexp(Cc, vj + ud) : Cc;
    V.v[t] = clamp_log(V.lce[t] - (lsum - vj));
  } else if (t < V.m + V.n) {
    x = V.u[t - V.m];
    act = true;
  }
  double lse_u = 0.0;
  double none[1] = {0};
  double nt[1];
  if (reduce_last_lse<1>(none, x, act, V.red, V.counter, nt, &lse_u) && threadIdx.x == 0) {
    if (V.dcol) {
      const double vd = V.v[V.m];
      const double lsum = V.drow ? logaddexp(vd + lse_u, vd + ud - S->A_over_g) : vd + lse_u;
      V.v[V.m] = clamp_log(V.lce[V.m] - (lsum - vd));
    }
    const int it = S->t + 1;
    S->t = it;
    if (V.trace) S->trace[(it - 1) & 4095][0] = S->E;
    if (it >= S->max_iter) S->done = 1;
  }
}

// -------------------------------------------------------------- rounding ---

// R1: a_i = min(1, r_i / r(B)_i); f_i = u_i + w + log a_i
__global__ void round_r1_kernel(RoundVecs V) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.n) return;
  const double R = V.lrow[i];
  const double lr = V.r[i] > 0.0 ? log(V.r[i]) : POT_NEG_BIG;
  const double la = fmin(0.0, lr - R);
  V.f[i] = clamp_log(V.u[i] + V.S->w_out + la);
}

// R2: b_j = min(1, c_j / c(X')_j); g_j = v_j + log b_j; column masses of X''
__global__ void round_r2_kernel(RoundVecs V) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0, 0};
  if (j < V.m) {
    const double Cc = V.lcol[j];
    const double lc = V.c[j] > 0.0 ? log(V.c[j]) : POT_NEG_BIG;
    const double lb = fmin(0.0, lc - Cc);
    V.g[j] = clamp_log(V.v[j] + lb);
    const double cm = safe_exp(Cc + lb);
    const double qj = fmax(V.c[j] - cm, 0.0);
    V.q[j] = qj;
    v[0] = cm;
    v[1] = qj;
  }
  double tot[2];
  if (reduce_last<2>(v, V.red, V.counter, tot) && threadIdx.x == 0) {
    V.S->m2 = tot[0];
    V.S->sum_q = tot[1];
  }
}

// R3: m'' >= s: scale to mass s (f += log(s/m'')), no rank-one term
__global__ void round_r3_kernel(RoundVecs V) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double lk = log(V.S->s / V.S->m2);
  if (i < V.n) { V.f[i] = clamp_log(V.f[i] + lk); V.p[i] = 0.0; }
  if (i < V.m) V.q[i] = 0.0;
  if (i == 0) *V.kappa = 0.0;
}

// R4: m'' < s: p = r - X'' 1; kappa = (s - m'') / (|p|_1 |q|_1)
__global__ void round_r4_kernel(RoundVecs V) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0};
  if (i < V.n) {
    const double R = V.lrow[i];
    const double pi = fmax(V.r[i] - safe_exp(R), 0.0);
    V.p[i] = pi;
    v[0] = pi;
  }
  double tot[1];
  if (reduce_last<1>(v, V.red, V.counter, tot) && threadIdx.x == 0) {
    V.S->sum_p = tot[0];
    const double den = tot[0] * V.S->sum_q;
    *V.kappa = den > 0.0 ? (V.S->s - V.S->m2) / den : 0.0;
    V.S->kappa = *V.kappa;
  }
}

__global__ void marginals_setup_kernel(DevState* S, double w, unsigned int* counter) {
  if (threadIdx.x < 8) counter[threadIdx.x] = 0u;
  if (threadIdx.x == 0) { S->w_out = w; S->tc_err = 0; }
}

__global__ void marginals_out_kernel(int64_t n, int64_t m, const double* lrow_in, const double* lcol_in,
                                     double* lrow, double* lcol, double* red, unsigned int* counter, double* tot_out,
                                     const int* err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool bad = err && *err;          // a pass that gave up waiting: its sums are invalid
  double v[1] = {0};
  // |B|_1 from the row sums, or from the column sums of a columns-only pass (lrow_in NULL)
  if (t < n) {
    if (lrow_in) {
      const double R = bad ? (double)NAN : lrow_in[t];
      if (lrow) lrow[t] = R;
      v[0] = safe_exp(R);
    }
  } else if (t < n + m) {
    const double Cc = bad ? (double)NAN : (lcol_in ? lcol_in[t - n] : 0.0);
    if (lcol) lcol[t - n] = Cc;
    if (!lrow_in) v[0] = safe_exp(Cc);
  }
  double tot[1];
  if (reduce_last<1>(v, red, counter, tot) && threadIdx.x == 0 && tot_out) *tot_out = bad ? (double)NAN : tot[0];
}

__global__ void dense_plan_kernel(PassDesc P, const double* f, const double* g, const double* p,
                                  const double* q, const double* kappa, float* X, int64_t ldx) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= P.m || i >= P.n) return;
  double cost;
  if (P.kind == COST_DENSE_F32) cost = (double)P.C[i * P.ldc + j];
  else {
    double acc = 0.0;
    for (int t = 0; t < P.d; ++t) {
      double x, y;
      if (P.kind == COST_SQEUCLID_BF16) {
        x = __uint_as_float(((unsigned)reinterpret_cast<const unsigned short*>(P.X)[i * P.ldx + t]) << 16);
        y = __uint_as_float(((unsigned)reinterpret_cast<const unsigned short*>(P.Y)[j * P.ldy + t]) << 16);
      } else if (P.kind == COST_SQEUCLID_F16) {
        x = __half2float(reinterpret_cast<const __half*>(P.X)[i * P.ldx + t]);
        y = __half2float(reinterpret_cast<const __half*>(P.Y)[j * P.ldy + t]);
      } else {
        x = reinterpret_cast<const float*>(P.X)[i * P.ldx + t];
        y = reinterpret_cast<const float*>(P.Y)[j * P.ldy + t];
      }
      acc += (x - y) * (x - y);
    }
    cost = acc;
  }
  const double lg = f[i] + g[j] - P.gC * cost;
  X[i * ldx + j] = (float)(safe_exp(lg) + *kappa * p[i] * q[j]);
}

}  // namespace

static thread_local bool g_pdl = false;   // see pdl_scope

void launch_combine(const float2* row_part, int64_t ncolblk, int64_t n, double* lrow, const float2* col_part,
                    int64_t nrowblk, int64_t m, double* lcol, const int* done, cudaStream_t st, const int* skip,
                    int skip_if) {
  const int64_t nbr = lrow ? (n + 31) / 32 : 0;
  const int64_t nbc = lcol ? (m + 31) / 32 : 0;
  if (nbr + nbc == 0) return;
  launch_k(combine_kernel, dim3((unsigned)(nbr + nbc)), dim3(256), 0, st, row_part, ncolblk, n, lrow, col_part,
           nrowblk, m, lcol, nbr, done, skip, skip_if);
}

void launch_marg_stats(const double* r, const double* c, int64_t n, int64_t m, double* red,
                       unsigned int* counter, double* out6, cudaStream_t st) {
  marg_stats_kernel<<<vec_blocks(n + m), kVecThreads, 0, st>>>(r, c, n, m, red, counter, out6);
}
void launch_reduce_parts(const double* part, int64_t count, int op_max, double* out, cudaStream_t st) {
  reduce_parts_kernel<<<1, 1024, 0, st>>>(part, count, op_max, out);
}
void launch_aspot_init(const AspotVecs& V, const double* r, const double* c, double eps_s,
                       const double* u0, const double* v0, double w0, cudaStream_t st) {
  aspot_init_kernel<<<vec_blocks(V.n + V.m), kVecThreads, 0, st>>>(V, r, c, eps_s, u0, v0, w0);
}
// Block size of the solver loops' O(n + m) kernels: 64 threads (two warps)
// while that still gives at most a few blocks per SM, so the FP64 updates,
// whose instructions each hold an SM sub-partition's narrow FP64 pipe for many
// cycles, spread over as many SMs as the problem allows; 256 beyond.
bool pdl_active() { return g_pdl; }
pdl_scope::pdl_scope(bool on) : prev(g_pdl) { g_pdl = on; }
pdl_scope::~pdl_scope() { g_pdl = prev; }

int loop_threads(int64_t len) { return len <= kLoopSmallLen ? 64 : kVecThreads; }
unsigned loop_blocks(int64_t len) { const int t = loop_threads(len); return (unsigned)((len + t - 1) / t); }

void launch_aspot_extrap(const AspotVecs& V, cudaStream_t st) {
  launch_k(aspot_extrap_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V);
}
void launch_aspot_after_grad(const AspotVecs& V, cudaStream_t st) {
  launch_k(aspot_after_grad_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V);
}
void launch_aspot_after_greenkhorn(const AspotVecs& V, int k, cudaStream_t st) {
  launch_k(aspot_after_greenkhorn_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V, k);
}
void launch_aspot_greedy_pick(const AspotVecs& V, cudaStream_t st) {
  launch_k(aspot_greedy_pick_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V);
}
void launch_aspot_greedy_final(const AspotVecs& V, cudaStream_t st) {
  launch_k(aspot_greedy_final_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V);
}
void launch_aspot_greedy_apply(const AspotVecs& V, cudaStream_t st) {
  launch_k(aspot_greedy_apply_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V);
}
void launch_aspot_after_final(const AspotVecs& V, int k, cudaStream_t st) {
  launch_k(aspot_after_final_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V, k);
}
void launch_aspot_start_eval(const AspotVecs& V, const double* u, const double* v, int slot, cudaStream_t st) {
  aspot_start_eval_kernel<<<vec_blocks(V.n + V.m), kVecThreads, 0, st>>>(V, u, v, slot);
}
void launch_aspot_zero_bar(const AspotVecs& V, cudaStream_t st) {
  aspot_zero_bar_kernel<<<vec_blocks(V.n + V.m), kVecThreads, 0, st>>>(V);
}
void launch_aspot_start_select(const AspotVecs& V, cudaStream_t st) {
  aspot_start_select_kernel<<<vec_blocks(V.n + V.m), kVecThreads, 0, st>>>(V);
}
void launch_sink_init(const SinkVecs& V, const double* r, const double* c, double eps_s, double s,
                      cudaStream_t st) {
  sink_init_kernel<<<vec_blocks(V.n + V.m + 1), kVecThreads, 0, st>>>(V, r, c, eps_s, s);
}
void launch_sink_after_rows(const SinkVecs& V, cudaStream_t st) {
  launch_k(sink_after_rows_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V);
  launch_k(sink_restore_kernel, dim3(vec_blocks(V.n + 1)), dim3(kVecThreads), 0, st, V);
}
void launch_sink_after_cols(const SinkVecs& V, cudaStream_t st) {
  launch_k(sink_after_cols_kernel, dim3(loop_blocks(V.n + V.m)), dim3(loop_threads(V.n + V.m)), 0, st, V);
}
void launch_round_r1(const RoundVecs& V, cudaStream_t st) {
  round_r1_kernel<<<vec_blocks(V.n), kVecThreads, 0, st>>>(V);
}
void launch_round_r2(const RoundVecs& V, cudaStream_t st) {
  round_r2_kernel<<<vec_blocks(V.m), kVecThreads, 0, st>>>(V);
}
void launch_round_r3(const RoundVecs& V, cudaStream_t st) {
  round_r3_kernel<<<vec_blocks(V.n > V.m ? V.n : V.m), kVecThreads, 0, st>>>(V);
}
void launch_round_r4(const RoundVecs& V, cudaStream_t st) {
  round_r4_kernel<<<vec_blocks(V.n), kVecThreads, 0, st>>>(V);
}
void launch_marginals_setup(DevState* S, double w, unsigned int* counter, cudaStream_t st) {
  marginals_setup_kernel<<<1, 32, 0, st>>>(S, w, counter);
}
void launch_marginals_out(int64_t n, int64_t m, const double* lrow_in, const double* lcol_in, double* lrow,
                          double* lcol, double* red, unsigned int* counter, double* tot_out, const int* err,
                          cudaStream_t st) {
  marginals_out_kernel<<<vec_blocks(n + m), kVecThreads, 0, st>>>(n, m, lrow_in, lcol_in, lrow, lcol, red, counter,
                                                                 tot_out, err);
}
void launch_dense_plan(const PassDesc& P, const double* f, const double* g, const double* p,
                       const double* q, const double* kappa, float* X, int64_t ldx, cudaStream_t st) {
  dim3 grid((unsigned)((P.m + 255) / 256), (unsigned)P.n);
  dense_plan_kernel<<<grid, 256, 0, st>>>(P, f, g, p, q, kappa, X, ldx);
}

}  // namespace pot
