// Shared device helpers of the ASPOT / feasible-Sinkhorn CUDA library.
//
// Numerics of every pass (the O(nm) reductions of the method):
//   logit_ij = a_i + b_j - gC * cost_ij          (log of an entry of B(z))
// where a_i collects the row potential (u_i + w, or u_i for the extended
// Sinkhorn kernel) and b_j the column potential.  Potentials are FP64
// masters; a pass receives them as FP32 (hi, lo) pairs, with hi rounded to a
// multiple of 2^-10 so that hi_a + hi_b is exact in FP32 for |a|,|b| < 2^13.
// The logit is then fma(-gC, cost, hi_a + hi_b) + (lo_a + lo_b): one rounding
// relative to the (small) logit instead of one relative to |u|+|v|+|w|.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define POT_NEG_BIG (-1.0e30)      // stands for log 0 in FP64 potentials
#define POT_NEG_BIGF (-1.0e30f)

namespace pot {

struct HiLo { float hi, lo; };

__device__ __forceinline__ HiLo split_hilo(double x) {
  HiLo r;
  if (!(x > -1.0e29)) { r.hi = POT_NEG_BIGF; r.lo = 0.f; return r; }   // log 0 (also NaN -> -big)
  double h = nearbyint(x * 1024.0) * (1.0 / 1024.0);
  r.hi = (float)h;
  r.lo = (float)(x - (double)r.hi);
  return r;
}

// 2^x with the hardware approximation (flushes denormal results to 0).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Programmatic dependent launch.  A kernel that a solver loop launches with
// the programmatic-serialisation attribute may be scheduled while its
// predecessor in the stream still runs: pdl_wait() returns once that
// predecessor has completed and its writes are visible (at once for a kernel
// launched without the attribute), and pdl_release() lets the successor's
// blocks be scheduled.  Such a kernel calls pdl_wait() before its first access
// to device memory, so every kernel of the chain still sees all earlier ones
// complete; only the launch latency overlaps.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() { pdl_wait(); pdl_release(); }

// Maxima that keep a NaN (fmaxf / fmax drop it): a NaN anywhere in the cost
// must reach the prologue's finiteness check through the max-cost pass.
__device__ __forceinline__ float nanmaxf(float a, float b) { return (a > b || a != a) ? a : b; }
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// log-sum-exp accumulator in FP64: value = m + log(s)
struct Lse {
  double m, s;
  __device__ __forceinline__ void init() { m = -INFINITY; s = 0.0; }
  // add a partial (shift k, sum t) meaning log(t) + k, all in the natural log
  __device__ __forceinline__ void add(double k, double t) {
    if (!(t > 0.0)) return;
    if (k > m) { s = s * exp(m - k) + t; m = k; }
    else { s += t * exp(k - m); }
  }
  __device__ __forceinline__ double value() const { return s > 0.0 ? m + log(s) : POT_NEG_BIG; }
};

// e^R of a log-sum R that comes from FP32 pass partials (whose own error is
// ~1e-7 relative and more): FP32 accuracy (~2^-22 relative) over the FP64
// range in a handful of FP64 operations instead of a full FP64 exponential,
// which costs dozens of instructions on this GPU's narrow FP64 pipe.  With
// y = R log2 e = k + f (k = floor y, f in [0, 1)): e^R = 2^k 2^f, 2^f from the
// FP32 hardware ex2, 2^k written into the exponent field.  R <= -700 and NaN
// give 0 (the log-domain convention for log 0, as for an FP64 exp below it).
__device__ __forceinline__ double exp_sum(double R) {
  if (!(R > -700.0)) return 0.0;
  if (R > 709.7) return INFINITY;
  const double y = R * 1.4426950408889634;
  const double k = floor(y);
  const float p = ex2((float)(y - k));                 // in [1, 2)
  return (double)p * __hiloint2double(((int)k + 1023) << 20, 0);
}

__device__ __forceinline__ double softplus(double x) {   // log(1 + e^x)
  return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}
__device__ __forceinline__ double logaddexp(double a, double b) {
  double mx = fmax(a, b);
  if (mx <= POT_NEG_BIG) return POT_NEG_BIG;
  return mx + log1p(exp(-fabs(a - b)));
}

// Natural log of 2^M * S (M in log2 units, S > 0 an FP32 sum): the exponent
// of S is split off exactly (frexpf), so the FP32 log2 acts on a mantissa in
// [0.5, 1) and its absolute error stays near 1e-7; M, the exponent and that
// logarithm are added in FP64.  FP64 logarithms would dominate the combine of
// pass partials on this GPU (FP64 runs at a small fraction of the FP32 rate).
__device__ __forceinline__ double log_shifted_sum(float M, float S) {
  int ex;
  const float mant = frexpf(S, &ex);
  return ((double)M + (double)ex + (double)log2f(mant)) * 0.6931471805599453;
}

}  // namespace pot
