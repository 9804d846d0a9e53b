// Per-instance bodies of the ASPOT iteration (Algorithm 2), one CTA per
// instance: the combine of a pass's partials into FP64 log-sums, the
// gradient / Greenkhorn / final updates of the cyclic and greedy block rules,
// the extrapolation and the next pass's FP32 (hi, lo) terms, every scalar a
// deterministic block reduction.  Shared by the fused batched sweep
// (batched.cu) and the single-cluster loop for small problems (cluster.cu).
// Device code only; each translation unit that includes it gets its own copy
// (the non-template functions are static).
#pragma once
#include "common.cuh"
#include "pass.h"
#include "kernels.h"
#include "simt_tile.cuh"

namespace pot {
namespace inst {

using simt::kL2E;

template <int NV>
__device__ void block_sums(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  __shared__ double tot[NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double x = warp_sum_d(v[k]);
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = tot[k];
  __syncthreads();
}

// log-sum-exp over the block of (x, active) -> natural log (all threads)
static __device__ double block_lse(double x, bool act) {
  __shared__ double smx[32], ssm[32];
  __shared__ double res;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  double mx = act ? x : -INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) smx[warp] = mx;
  __syncthreads();
  double M = -INFINITY;
  for (int w = 0; w < nw; ++w) M = fmax(M, smx[w]);
  double s = (act && M > -INFINITY) ? exp(x - M) : 0.0;
  s = warp_sum_d(s);
  if (lane == 0) ssm[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += ssm[w];
    res = (t > 0.0) ? M + log(t) : POT_NEG_BIG;
  }
  __syncthreads();
  const double r = res;
  __syncthreads();
  return r;
}

static __device__ __forceinline__ double sexp(double x) { return x > -700.0 ? exp(x) : 0.0; }
static __device__ __forceinline__ double clampl(double x) { return x > POT_NEG_BIG ? x : POT_NEG_BIG; }

constexpr int kBTrace = 1024;  // iterations of each instance whose decisions are recorded

struct BVecs {
  BInst* inst;
  double *rt, *ct, *lrt, *lct, *ut, *vt, *uc, *vc, *ub, *vb, *ug, *vg, *uh, *vh;
  double *uo, *vo, *fc, *gc;          // concatenated final duals and plan potentials
  const double *lrow, *lcol;
  int* ndone;
  unsigned char* trace;               // [count][kBTrace]: took + 2 k + 8 k2 per iteration
  double* trace4;                     // single solve: rows [4096][4] of (E_t, phi(z^t), phi(z_check^{t+1}),
                                      // took + 2 k + 8 k2), the single-instance solver's trace, or NULL
};

// The threads that update one instance.  The bodies below are written against
// this interface: per-entry loops over first() + t step(), sums and
// log-sum-exps over all of them, global side effects (stop counter, trace) by
// writer() only, the instance record from inst().  BlockTeam: one CTA (the
// batched sweep); the single-cluster loop spreads an instance over a cluster.
struct BlockTeam {
  __device__ int64_t first() const { return threadIdx.x; }
  __device__ int64_t step() const { return blockDim.x; }
  template <int NV>
  __device__ void sums(double (&v)[NV]) { block_sums<NV>(v); }
  __device__ double lse(double x, bool act) { return block_lse(x, act); }
  __device__ bool writer() const { return threadIdx.x == 0; }
  __device__ BInst& inst(const BVecs& V, int k) const { return V.inst[k]; }
};

template <class T>
static __device__ void b_extrap_body(const BVecs& V, int inst, T& tm) {
  BInst& I = tm.inst(V, inst);
  if (I.done) return;
  const double th = I.theta;
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    V.ub[g] = (1.0 - th) * V.uc[g] + th * V.ut[g];
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    V.vb[g] = (1.0 - th) * V.vc[g] + th * V.vt[g];
  }
  if (threadIdx.x == 0) I.w_bar = (1.0 - th) * I.w_check + th * I.w_tilde;
}

// gradient step and coupling (same formulas as the single-instance solver)
template <class T>
static __device__ void b_after_grad_body(const BVecs& V, int inst, T& tm) {
  BInst& I = tm.inst(V, inst);
  if (I.done) return;
  const double th = I.theta, Lth = I.L * th;
  double v[3] = {0, 0, 0};
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    const double ub = V.ub[g];
    const double rB = exp_sum(V.lrow[g]), eu = sexp(ub);
    const double un = ub - (rB + eu - V.rt[g]) / Lth;
    V.ug[g] = ub + th * (un - V.ut[g]);
    V.ut[g] = un;
    v[0] += rB;
    v[1] += eu - ub * V.rt[g];
    if (!isfinite(un)) v[2] = 1.0;
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    const double vb = V.vb[g];
    const double cB = exp_sum(V.lcol[g]), ev = sexp(vb);
    const double vn = vb - (cB + ev - V.ct[g]) / Lth;
    V.vg[g] = vb + th * (vn - V.vt[g]);
    V.vt[g] = vn;
    v[1] += ev - vb * V.ct[g];
    if (!isfinite(vn)) v[2] = 1.0;
  }
  tm.template sums<3>(v);
  if (threadIdx.x == 0) {
    const double wn = I.w_bar - (v[0] - I.s) / Lth;
    I.w_grave = I.w_bar + th * (wn - I.w_tilde);
    I.w_tilde = wn;
    if (I.t == 0) I.phi_check = v[0] + v[1] - I.w_bar * I.s;
    if (v[2] != 0.0 || !isfinite(wn)) I.nonfinite = 1;
  }
}

template <class T>
static __device__ void b_after_greenkhorn_body(const BVecs& V, int inst, int k, T& tm) {
  BInst& I = tm.inst(V, inst);
  if (I.done) return;
  double v[2] = {0, 0};
  double xr = 0.0;
  bool act = false;
  double lt = 0.0;
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    const double ug = V.ug[g];
    if (k == 0) {
      const double uh = V.lrt[g] - softplus(V.lrow[g] - ug);
      V.uh[g] = uh;
      v[0] += -uh * V.rt[g];
    } else {
      v[0] += sexp(ug) - ug * V.rt[g];
    }
  }
  if (k == 2) {
    // log |B|_1 at z_grave over the instance's rows (blockwise log-sum-exp of the row log-sums)
    double acc = -INFINITY, s = 0.0;
    for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
      const double x = V.lrow[I.row0 + i];
      if (x > acc) { s = s * exp(acc - x) + 1.0; acc = x; } else s += exp(x - acc);
    }
    xr = acc > -INFINITY ? acc + log(s) : POT_NEG_BIG;
    act = acc > -INFINITY;
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    const double vg = V.vg[g];
    if (k == 1) {
      const double vh = V.lct[g] - softplus(V.lcol[g] - vg);
      V.vh[g] = vh;
      v[1] += -vh * V.ct[g];
    } else {
      v[1] += sexp(vg) - vg * V.ct[g];
    }
  }
  tm.template sums<2>(v);
  if (k == 2) lt = tm.lse(xr, act);
  if (threadIdx.x == 0) {
    double wh = I.w_grave, base;
    if (k == 0) base = I.sum_rt;
    else if (k == 1) base = I.sum_ct;
    else { wh = I.w_grave + I.log_s - lt; base = I.s; }
    I.w_hat = wh;
    const double ph = base + v[0] + v[1] - wh * I.s;
    I.phi_hat = ph;
    const int take = ph < I.phi_check;
    I.take_hat = take;
    I.phi_z = take ? ph : I.phi_check;
    I.w_z = take ? wh : I.w_check;
  }
}

template <class T>
static __device__ void b_after_final_body(const BVecs& V, int inst, int k, T& tm) {
  BInst& I = tm.inst(V, inst);
  if (I.done) return;
  const int take = I.take_hat;
  const double* uzh = (k == 0) ? V.uh : V.ug;
  const double* vzh = (k == 1) ? V.vh : V.vg;
  double v[4] = {0, 0, 0, 0};
  double acc = -INFINITY, ssum = 0.0;
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    const double uz = take ? uzh[g] : V.uc[g];
    const double R = V.lrow[g];
    const double rB = exp_sum(R), eu = sexp(uz);
    v[0] += fabs(rB + eu - V.rt[g]);
    v[1] += rB;
    I.pu[i] = uz;
    V.uo[g] = uz;
    const double un = (k == 0) ? V.lrt[g] - softplus(R - uz) : uz;
    V.uc[g] = un;
    v[2] += (k == 0) ? -un * V.rt[g] : eu - un * V.rt[g];     // un = uz unless k = 0
    if (!isfinite(R) && R != POT_NEG_BIG) v[3] = 1.0;
    if (k == 2) {                       // log |B|_1 is needed by the w step only
      if (R > acc) { ssum = ssum * exp(acc - R) + 1.0; acc = R; } else ssum += exp(R - acc);
    }
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    const double vz = take ? vzh[g] : V.vc[g];
    const double Cc = V.lcol[g];
    const double cB = exp_sum(Cc), ev = sexp(vz);
    v[0] += fabs(cB + ev - V.ct[g]);
    I.pv[j] = vz;
    V.vo[g] = vz;
    const double vn = (k == 1) ? V.lct[g] - softplus(Cc - vz) : vz;
    V.vc[g] = vn;
    v[2] += (k == 1) ? -vn * V.ct[g] : ev - vn * V.ct[g];     // vn = vz unless k = 1
    if (!isfinite(Cc) && Cc != POT_NEG_BIG) v[3] = 1.0;
  }
  tm.template sums<4>(v);
  const double lt = (k == 2) ? tm.lse(acc > -INFINITY ? acc + log(ssum) : POT_NEG_BIG, acc > -INFINITY) : 0.0;
  if (threadIdx.x == 0) {
    const double s = I.s;
    const double E = fabs(v[1] - s) + v[0];
    const double wz = I.w_z;
    I.w_out = wz;
    double wc = wz, base;
    if (k == 0) base = I.sum_rt;
    else if (k == 1) base = I.sum_ct;
    else { wc = wz + I.log_s - lt; base = s; }
    I.w_check = wc;
    I.phi_check = base + v[2] - wc * s;
    I.E = E;
    I.tot = v[1];
    if (V.trace && tm.writer() && I.t < kBTrace) V.trace[(int64_t)inst * kBTrace + I.t] = (unsigned char)(take + 10 * k);
    if (V.trace4 && tm.writer()) {
      double* tr = V.trace4 + (int64_t)(I.t & 4095) * 4;
      tr[0] = E; tr[1] = I.phi_z; tr[2] = I.phi_check; tr[3] = (double)take;
    }
    const double th = I.theta;
    I.theta = th * (sqrt(th * th + 4.0) - th) / 2.0;
    I.t = I.t + 1;
    if (v[3] != 0.0 || !isfinite(E)) I.nonfinite = 1;
    if (E <= I.thr || I.t >= I.max_iter || I.nonfinite) {
      I.done = 1;
      if (tm.writer()) atomicAdd(V.ndone, 1);
    }
  }
}

// ------------------------------------------------- greedy block rule ---
// Per instance (one CTA): the exact decreases of phi of the three block steps,
//   D_u = sum_i rho(r~_i, r_i(B) + e^{u_i}), D_v likewise, D_w = rho(s, |B|_1),
// rho(a, b) = b - a + a log(a / b), from the two-sided pass at the point; the
// block with the largest is stepped (ties to the lower index), as in the
// single-instance solver.

static __device__ __forceinline__ double b_rho_log(double a, double la, double lb) {
  return sexp(lb) - a + (a > 0.0 ? a * (la - lb) : 0.0);
}
static __device__ __forceinline__ int b_pick(double du, double dv, double dw) {
  int k = 0;
  double best = du;
  if (dv > best) { k = 1; best = dv; }
  if (dw > best) k = 2;
  return k;
}
static __device__ __forceinline__ void lse_add(double x, double& acc, double& s) {
  if (x > acc) { s = s * exp(acc - x) + 1.0; acc = x; } else s += exp(x - acc);
}

// After the two-sided pass at z_grave: choose k, Greenkhorn step, closed-form
// phi(z^), argmin against phi(z_check).  z^ is written whole to (uh, vh).
template <class T>
static __device__ void b_greedy_greenkhorn_body(const BVecs& V, int inst, T& tm) {
  BInst& I = tm.inst(V, inst);
  if (I.done) return;
  double d[2] = {0, 0};
  double acc = -INFINITY, ss = 0.0;
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    const double R = V.lrow[g];
    d[0] += b_rho_log(V.rt[g], V.lrt[g], logaddexp(R, V.ug[g]));
    lse_add(R, acc, ss);
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    d[1] += b_rho_log(V.ct[g], V.lct[g], logaddexp(V.lcol[g], V.vg[g]));
  }
  tm.template sums<2>(d);
  const double lt = tm.lse(acc > -INFINITY ? acc + log(ss) : POT_NEG_BIG, acc > -INFINITY);
  const int k = b_pick(d[0], d[1], b_rho_log(I.s, I.log_s, lt));
  double v[2] = {0, 0};
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    const double ug = V.ug[g];
    if (k == 0) {
      const double uh = V.lrt[g] - softplus(V.lrow[g] - ug);
      V.uh[g] = uh;
      v[0] += -uh * V.rt[g];
    } else {
      V.uh[g] = ug;
      v[0] += sexp(ug) - ug * V.rt[g];
    }
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    const double vg = V.vg[g];
    if (k == 1) {
      const double vh = V.lct[g] - softplus(V.lcol[g] - vg);
      V.vh[g] = vh;
      v[1] += -vh * V.ct[g];
    } else {
      V.vh[g] = vg;
      v[1] += sexp(vg) - vg * V.ct[g];
    }
  }
  tm.template sums<2>(v);
  if (threadIdx.x == 0) {
    double wh = I.w_grave, base;
    if (k == 0) base = I.sum_rt;
    else if (k == 1) base = I.sum_ct;
    else { wh = I.w_grave + I.log_s - lt; base = I.s; }
    I.kg = k;
    I.w_hat = wh;
    const double ph = base + v[0] + v[1] - wh * I.s;
    I.phi_hat = ph;
    const int take = ph < I.phi_check;
    I.take_hat = take;
    I.phi_z = take ? ph : I.phi_check;
    I.w_z = take ? wh : I.w_check;
  }
}

// After the two-sided pass at z^t: E_t, the block k2 with the largest
// decrease at z^t, z_check^{t+1} = Greenkhorn_{k2}(z^t) and its closed-form
// phi, theta update and the stop test.
template <class T>
static __device__ void b_greedy_final_body(const BVecs& V, int inst, T& tm) {
  BInst& I = tm.inst(V, inst);
  if (I.done) return;
  const int take = I.take_hat;
  // E parts, |B|_1, D_u, D_v, phi parts: rows stepped / kept, columns stepped / kept, nonfinite
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double acc = -INFINITY, ss = 0.0;
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    const double uz = take ? V.uh[g] : V.uc[g];
    const double R = V.lrow[g], a = V.rt[g];
    const double rB = sexp(R), eu = sexp(uz);
    v[0] += fabs(rB + eu - a);
    v[1] += rB;
    v[2] += b_rho_log(a, V.lrt[g], logaddexp(R, uz));
    v[4] += -(V.lrt[g] - softplus(R - uz)) * a;
    v[5] += eu - uz * a;
    I.pu[i] = uz;
    V.uo[g] = uz;
    if (!isfinite(R) && R != POT_NEG_BIG) v[8] = 1.0;
    lse_add(R, acc, ss);
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    const double vz = take ? V.vh[g] : V.vc[g];
    const double Cc = V.lcol[g], c = V.ct[g];
    const double cB = sexp(Cc), ev = sexp(vz);
    v[0] += fabs(cB + ev - c);
    v[3] += b_rho_log(c, V.lct[g], logaddexp(Cc, vz));
    v[6] += -(V.lct[g] - softplus(Cc - vz)) * c;
    v[7] += ev - vz * c;
    I.pv[j] = vz;
    V.vo[g] = vz;
    if (!isfinite(Cc) && Cc != POT_NEG_BIG) v[8] = 1.0;
  }
  tm.template sums<9>(v);
  const double lt = tm.lse(acc > -INFINITY ? acc + log(ss) : POT_NEG_BIG, acc > -INFINITY);
  const double s = I.s;
  const int k2 = b_pick(v[2], v[3], b_rho_log(s, I.log_s, lt));
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    const double uz = V.uo[g];
    V.uc[g] = (k2 == 0) ? V.lrt[g] - softplus(V.lrow[g] - uz) : uz;
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    const double vz = V.vo[g];
    V.vc[g] = (k2 == 1) ? V.lct[g] - softplus(V.lcol[g] - vz) : vz;
  }
  if (threadIdx.x == 0) {
    const double E = fabs(v[1] - s) + v[0];
    const double wz = I.w_z;
    I.w_out = wz;
    double wc = wz, ph;
    if (k2 == 0) ph = I.sum_rt + v[4] + v[7] - wz * s;
    else if (k2 == 1) ph = I.sum_ct + v[5] + v[6] - wz * s;
    else { wc = wz + I.log_s - lt; ph = s + v[5] + v[7] - wc * s; }
    I.w_check = wc;
    I.phi_check = ph;
    I.E = E;
    I.tot = v[1];
    if (V.trace && tm.writer() && I.t < kBTrace) V.trace[(int64_t)inst * kBTrace + I.t] = (unsigned char)(take + 2 * I.kg + 8 * k2);
    if (V.trace4 && tm.writer()) {
      double* tr = V.trace4 + (int64_t)(I.t & 4095) * 4;
      tr[0] = E; tr[1] = I.phi_z; tr[2] = ph; tr[3] = (double)(take + 2 * I.kg + 8 * k2);
    }
    const double th = I.theta;
    I.theta = th * (sqrt(th * th + 4.0) - th) / 2.0;
    I.t = I.t + 1;
    if (v[8] != 0.0 || !isfinite(E)) I.nonfinite = 1;
    if (E <= I.thr || I.t >= I.max_iter || I.nonfinite) {
      I.done = 1;
      if (tm.writer()) atomicAdd(V.ndone, 1);
    }
  }
}

enum { E_GRAD = 0, E_GK = 1, E_FINAL = 2, E_GGK = 3, E_GFINAL = 4 };

// FP64 log-sums of one instance's rows and / or columns from the pass
// partials (only its own column / row blocks; they are all written by every
// pass, so nothing needs clearing).  Partials come from other SMs: L1 bypass.
template <class T>
static __device__ void b_combine_body(const BatchPass& B, const BVecs& V, const BInst& I, bool rows, bool cols,
                                      T& tm) {
  double* lrow = const_cast<double*>(V.lrow);
  double* lcol = const_cast<double*>(V.lcol);
  if (rows) {
    const int64_t ncb = (I.m + B.W - 1) / B.W;
    for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
      const int64_t g = I.row0 + i;
      float M = -INFINITY;
      for (int64_t b = 0; b < ncb; ++b) {
        const float2 p = __ldcg(B.row_part + b * B.Ntot + g);
        if (p.y > 0.f) M = fmaxf(M, p.x);
      }
      float St = 0.f, comp = 0.f;
      if (M > -INFINITY)
        for (int64_t b = 0; b < ncb; ++b) {
          const float2 p = __ldcg(B.row_part + b * B.Ntot + g);
          if (p.y > 0.f) {
            const float y = p.y * ex2(p.x - M) - comp;
            const float t = St + y;
            comp = (t - St) - y;
            St = t;
          }
        }
      lrow[g] = St > 0.f ? log_shifted_sum(M, St) : POT_NEG_BIG;
    }
  }
  if (cols) {
    const int64_t nrb = (I.n + B.H - 1) / B.H;
    for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
      const int64_t g = I.col0 + j;
      float M = -INFINITY;
      for (int64_t b = 0; b < nrb; ++b) {
        const float2 p = __ldcg(B.col_part + b * B.Mtot + g);
        if (p.y > 0.f) M = fmaxf(M, p.x);
      }
      float St = 0.f, comp = 0.f;
      if (M > -INFINITY)
        for (int64_t b = 0; b < nrb; ++b) {
          const float2 p = __ldcg(B.col_part + b * B.Mtot + g);
          if (p.y > 0.f) {
            const float y = p.y * ex2(p.x - M) - comp;
            const float t = St + y;
            comp = (t - St) - y;
            St = t;
          }
        }
      lcol[g] = St > 0.f ? log_shifted_sum(M, St) : POT_NEG_BIG;
    }
  }
  __syncthreads();
}

// Per-pass FP32 (hi, lo) terms of one instance for the next pass (the
// batched prep kernel's arithmetic), potentials (arow, bcol) and the scalar
// w given explicitly.
template <class T>
static __device__ void b_prep_body(const BatchPass& B, const BInst& I, const double* arow, const double* bcol, double w,
                                   T& tm) {
  for (int64_t i = tm.first(); i < I.n; i += tm.step()) {
    const int64_t g = I.row0 + i;
    const float xn = B.xn[g];
    HiLo hl = split_hilo((arow[g] + w - I.gC * (double)xn) * kL2E);
    B.rowA[g] = make_float4(hl.hi, hl.lo, xn, 0.f);
  }
  for (int64_t j = tm.first(); j < I.m; j += tm.step()) {
    const int64_t g = I.col0 + j;
    const float yn = B.yn[g];
    HiLo hl = split_hilo((bcol[g] - I.gC * (double)yn) * kL2E);
    B.colA[g] = make_float2(hl.hi, hl.lo);
    B.colB[g] = make_float2(yn, 0.f);
  }
}

template <class T>
static __device__ void b_epilogue(const BatchPass& B, const BVecs& V, int inst, int epi, int k, T& tm) {
  BInst& I = tm.inst(V, inst);
  switch (epi) {
    case E_GRAD:       // after P1 at z_bar: step and coupling; next: P2 at z_grave
      b_combine_body(B, V, I, true, true, tm);
      b_after_grad_body(V, inst, tm);
      __syncthreads();
      b_prep_body(B, I, V.ug, V.vg, I.w_grave, tm);
      break;
    case E_GK: {       // after P2: Greenkhorn step k, argmin; next: P3 at z^t
      b_combine_body(B, V, I, k != 1, k == 1, tm);
      b_after_greenkhorn_body(V, inst, k, tm);
      __syncthreads();
      const bool hat = I.take_hat;
      b_prep_body(B, I, hat ? (k == 0 ? V.uh : V.ug) : V.uc, hat ? (k == 1 ? V.vh : V.vg) : V.vc,
                  hat ? I.w_hat : I.w_check, tm);
      break;
    }
    case E_GGK: {      // greedy rule after P2 (two-sided)
      b_combine_body(B, V, I, true, true, tm);
      b_greedy_greenkhorn_body(V, inst, tm);
      __syncthreads();
      const bool hat = I.take_hat;
      b_prep_body(B, I, hat ? V.uh : V.uc, hat ? V.vh : V.vc, hat ? I.w_hat : I.w_check, tm);
      break;
    }
    default:           // after P3 at z^t: E_t, z_check^{t+1}, theta, stop; next: P1 at z_bar^{t+1}
      b_combine_body(B, V, I, true, true, tm);
      if (epi == E_FINAL) b_after_final_body(V, inst, k, tm);
      else b_greedy_final_body(V, inst, tm);
      __syncthreads();
      if (!I.done) {
        b_extrap_body(V, inst, tm);
        __syncthreads();
        b_prep_body(B, I, V.ub, V.vb, I.w_bar, tm);
      }
      break;
  }
}

}  // namespace inst
}  // namespace pot
