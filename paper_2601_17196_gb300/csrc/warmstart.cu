// Learned warm start (include/warmstart.h): features, forward, backward and
// Adam kernels of the per-point network with a mean-pooled context, and the
// host side that forms batches of 128-point tiles.
//
// A tile holds up to 128 consecutive points of ONE instance, so every
// per-instance quantity (the context, its gradient) is a sum over whole
// tiles.  All sums over points or tiles run in a fixed order: results do not
// depend on scheduling.
//
// FP32 mode, per tile (one persistent CTA of 256 threads per SM):
//   H1 = GELU(X W1^T + b1)                (128 x 128, shared memory)
//   A2 = H1 W2^T + q + b2, y = w3 . GELU(A2) + b3
// and for gradients additionally
//   D2 = dL/dA2 = dy w3 GELU'(A2)          (128 x 128, shared memory)
//   dW2 += D2^T H1                         (register accumulators per CTA)
//   dH1 = D2 W2                            (the context term is added per
//                                           instance afterwards, see below)
// Thread (ty, tx) of the 16 x 16 grid owns rows ty + 16 i and columns
// tx + 16 j (i, j < 8) of each 128 x 128 product; rows of the shared arrays
// are padded to 129 floats so both orientations read without bank conflicts.
//
// The context gradient: dL/dctx_k = (U^T dq_k)[:H] with dq_k the sum of D2
// over instance k, and it reaches every point of k as dctx_k / n_k.  Its
// share of dW1 and db1 is dctx_k / n_k (.) [sum over points of
// GELU'(a1) x^T] (and of GELU'(a1)), so the tile kernel accumulates those
// per-tile sums and a per-instance kernel adds the product once dq_k is known.
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>
#include <string.h>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/warmstart.h"
#include "common.cuh"
#include "ws_common.cuh"

namespace pot {
pot_status set_last_error(pot_status s, const char* msg);
}

using namespace pot::ws;

namespace {

pot_status wfail(pot_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return pot::set_last_error(s, buf);
}

#define WCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return wfail(POT_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define WCKL()                                                                             \
  do {                                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                   \
    if (e_ != cudaSuccess) return wfail(POT_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

// ------------------------------------------------------------ kernels ---

__global__ void ws_init_kernel(float* P, Offs o, uint64_t seed) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= o.total) return;
  float sd = 0.f;
  if (e < o.b1) sd = rsqrtf((float)o.F);
  else if (e >= o.W2 && e < o.U) sd = rsqrtf((float)H);
  else if (e >= o.U && e < o.b2) sd = rsqrtf((float)(H + 2));
  else if (e >= o.w3 && e < o.b3) sd = rsqrtf((float)H);
  float x = 0.f;
  if (sd > 0.f) {
    // two SplitMix64 outputs of the counter 2e, 2e + 1 -> Box-Muller
    const uint64_t a = splitmix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * e + 1));
    const uint64_t b = splitmix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * e + 2));
    const double u1 = ((double)(a >> 11) + 1.0) * (1.0 / 9007199254740992.0);   // (0, 1]
    const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);
    x = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2)) * sd;
  }
  P[e] = x;
}

__device__ __forceinline__ float load_coord(int kind, const void* base, int64_t ld, int64_t i, int k) {
  const int64_t a = i * ld + k;
  if (kind == POT_COST_SQEUCLID_BF16) {
    const uint16_t b = static_cast<const uint16_t*>(base)[a];
    return __uint_as_float((uint32_t)b << 16);
  }
  if (kind == POT_COST_SQEUCLID_F16) return __half2float(static_cast<const __half*>(base)[a]);
  return static_cast<const float*>(base)[a];
}

// One block: coordinate sums over both clouds and the two masses (FP64).
__global__ void ws_stats_kernel(int kind, const void* X, const void* Y, int64_t ldx, int64_t ldy, int d,
                                int64_t n, int64_t m, const double* r, const double* c, double* out) {
  __shared__ double sh[32][POT_WS_MAX_D + 2];
  double acc[POT_WS_MAX_D + 2];
#pragma unroll
  for (int k = 0; k < POT_WS_MAX_D + 2; ++k) acc[k] = 0.0;
  for (int64_t i = threadIdx.x; i < n + m; i += blockDim.x) {
    const bool row = i < n;
    const int64_t q = row ? i : i - n;
#pragma unroll
    for (int k = 0; k < POT_WS_MAX_D; ++k)
      if (k < d) acc[k] += (double)load_coord(kind, row ? X : Y, row ? ldx : ldy, q, k);
    if (row) acc[POT_WS_MAX_D] += r[q]; else acc[POT_WS_MAX_D + 1] += c[q];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < POT_WS_MAX_D + 2; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < POT_WS_MAX_D + 2) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
    out[threadIdx.x] = v;
  }
}

// Per point: centred, scaled coordinates, mass ratio, side, and the soft
// minima T_t (lrow_t,i - lu_i) from the passes at (lu, lv) = normalised
// log-masses and temperatures T_t = gamma 4^t (lrow, lcol hold POT_WS_TEMPS
// consecutive vectors).
__global__ void ws_feat_kernel(int kind, const void* X, const void* Y, int64_t ldx, int64_t ldy, int d,
                               int64_t n, int64_t m, const double* r, const double* c, double s, double sqcs,
                               double gamma, const double* stats, const double* lu, const double* lv,
                               const double* lrow, const double* lcol, float* feats, float* extra) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int F = d + POT_WS_EXTRA;
  const double inv_pts = 1.0 / (double)(n + m);
  const double sr = stats[POT_WS_MAX_D], sc = stats[POT_WS_MAX_D + 1];
  if (i < n + m) {
    const bool row = i < n;
    const int64_t q = row ? i : i - n;
    for (int k = 0; k < d; ++k) {
      const double x = (double)load_coord(kind, row ? X : Y, row ? ldx : ldy, q, k);
      feats[i * F + k] = (float)((x - stats[k] * inv_pts) * sqcs);
    }
    feats[i * F + d] = row ? (float)((double)n * r[q] / sr) : (float)((double)m * c[q] / sc);
    feats[i * F + d + 1] = row ? 1.f : -1.f;
    double T = gamma;
    for (int t = 0; t < POT_WS_TEMPS; ++t, T *= 4.0)
      feats[i * F + d + 2 + t] = (float)(T * (row ? lrow[t * n + q] - lu[q] : lcol[t * m + q] - lv[q]));
  }
  if (i == 0) {
    extra[0] = (float)(sr / s);
    extra[1] = (float)(sc / s);
  }
}

// lu_i = log(r_i / |r|_1), lv_j = log(c_j / |c|_1), masses floored at 1e-12 of their mean.
__global__ void ws_logmass_kernel(int64_t n, int64_t m, const double* r, const double* c, const double* stats,
                                  double* lu, double* lv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double sr = stats[POT_WS_MAX_D], sc = stats[POT_WS_MAX_D + 1];
  if (i < n) lu[i] = log(fmax(r[i], 1e-12 * sr / (double)n) / sr);
  else if (i < n + m) lv[i - n] = log(fmax(c[i - n], 1e-12 * sc / (double)m) / sc);
}

// log r_i (rows) or log c_j (columns), masses below 1e-12 times their mean
// floored there.
__device__ __forceinline__ double ws_base(const double* r, const double* stats, int slot, int64_t cnt, int64_t i) {
  const double floor_ = 1e-12 * stats[slot] / (double)cnt;
  return log(fmax(r[i], floor_));
}

// target = gamma log K: gamma (lrow_i - u_i) for rows, gamma (lcol_j - v_j) for
// columns, with lrow, lcol the log-sums of B(u, v, w); weight = sigmoid(log K)^2
__global__ void ws_targets_kernel(int64_t n, int64_t m, double gamma, const double* lrow, const double* lcol,
                                  const double* u, const double* v, float* t, float* wt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n + m) return;
  const double lk = (i < n) ? lrow[i] - u[i] : lcol[i - n] - v[i - n];
  t[i] = (float)(gamma * lk);
  if (wt) {
    const double sg = lk >= 0.0 ? 1.0 / (1.0 + exp(-lk)) : exp(lk) / (1.0 + exp(lk));
    wt[i] = (float)(sg * sg);
  }
}

// u_i = log r_i - softplus(y_i / gamma), v_j = log c_j - softplus(y_j / gamma)
__global__ void ws_to_duals_kernel(int64_t n, int64_t m, double inv_gamma, const double* r, const double* c,
                                   const double* stats, const float* y, double* u, double* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] = ws_base(r, stats, POT_WS_MAX_D, n, i) - pot::softplus((double)y[i] * inv_gamma);
  else if (i < n + m) v[i - n] = ws_base(c, stats, POT_WS_MAX_D + 1, m, i - n) - pot::softplus((double)y[i] * inv_gamma);
}

// Shift step of the warm start (one block): exact minimiser of
// phi(u + a 1, v + b 1, w + c) over (a, b, c), from |B(u, v, 0)|_1 = tot and the
// log-sums LU = log sum e^{u_i}, LV = log sum e^{v_j}:
//   e^a = (|r| - s) / e^LU,  e^b = (|c| - s) / e^LV,  e^(a + b + c) = s / tot
// (a = 0 when |r| = s, b = 0 when |c| = s).  Writes a, b, w = c into out[0..2].
__global__ void ws_shift_kernel(int64_t n, int64_t m, const double* u, const double* v, const double* stats,
                                double s, const double* tot, double* out) {
  __shared__ double sh[4][32];
  double mu = -INFINITY, mv = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mu = fmax(mu, u[i]);
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) mv = fmax(mv, v[j]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
    mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
  }
  if (lane == 0) { sh[0][warp] = mu; sh[1][warp] = mv; }
  __syncthreads();
  mu = sh[0][0]; mv = sh[1][0];
  for (int w = 1; w < nw; ++w) { mu = fmax(mu, sh[0][w]); mv = fmax(mv, sh[1][w]); }
  double su = 0.0, sv = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) su += exp(u[i] - mu);
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) sv += exp(v[j] - mv);
  for (int o = 16; o > 0; o >>= 1) {
    su += __shfl_xor_sync(0xffffffffu, su, o);
    sv += __shfl_xor_sync(0xffffffffu, sv, o);
  }
  __syncthreads();
  if (lane == 0) { sh[2][warp] = su; sh[3][warp] = sv; }
  __syncthreads();
  if (threadIdx.x == 0) {
    su = 0.0; sv = 0.0;
    for (int w = 0; w < nw; ++w) { su += sh[2][w]; sv += sh[3][w]; }
    const double LU = mu + log(su), LV = mv + log(sv);
    const double sr = stats[POT_WS_MAX_D], sc = stats[POT_WS_MAX_D + 1];
    const double a = sr > s ? log(sr - s) - LU : 0.0;
    const double b = sc > s ? log(sc - s) - LV : 0.0;
    out[0] = a;
    out[1] = b;
    out[2] = log(s) - log(*tot) - a - b;
  }
}

__global__ void ws_apply_shift_kernel(int64_t n, int64_t m, const double* sh, double* u, double* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] += sh[0];
  else if (i < n + m) v[i - n] += sh[1];
}

// Mass sums |r|_1, |c|_1 into stats[MAX_D], stats[MAX_D + 1] (one block).
__global__ void ws_mass_kernel(int64_t n, int64_t m, const double* r, const double* c, double* stats) {
  __shared__ double sh[2][32];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += r[i];
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) b += c[j];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    stats[POT_WS_MAX_D + threadIdx.x] = v;
  }
}

// Per tile: column sums of H1 = GELU(X W1^T + b1) (the context numerator).
__global__ void __launch_bounds__(H) ws_ctx_kernel(WsArgs A) {
  __shared__ float xs[kTile * FMAX];
  const WsTile tl = A.tiles[blockIdx.x];
  const int F = A.F, k = threadIdx.x;
  for (int e = k; e < tl.count * FMAX; e += H) {
    const int p = e / FMAX, f = e % FMAX;
    xs[e] = f < F ? A.feats[(tl.start + p) * F + f] : 0.f;    // padding slots must be 0, not stale
  }
  __syncthreads();
  float w[FMAX];
#pragma unroll
  for (int f = 0; f < FMAX; ++f) w[f] = f < F ? A.P[A.o.W1 + k * F + f] : 0.f;
  const float b = A.P[A.o.b1 + k];
  float s = 0.f;
  for (int p = 0; p < tl.count; ++p) {
    float a = b;
#pragma unroll
    for (int f = 0; f < FMAX; ++f) a = fmaf(w[f], xs[p * FMAX + f], a);
    s += gelu(a);
  }
  A.ctxp[(int64_t)blockIdx.x * H + k] = s;
}

// Per instance of the batch: ctx = mean of H1, cin = [ctx; extra], q = U cin.
__global__ void __launch_bounds__(H) ws_q_kernel(WsArgs A) {
  __shared__ float cin[H + 2];
  const int b = blockIdx.x, k = threadIdx.x;
  const WsInst I = A.binfo[b];
  float s = 0.f;
  for (int t = I.tile0; t < I.tile0 + I.ntiles; ++t) s += A.ctxp[(int64_t)t * H + k];
  cin[k] = s / I.npts;
  if (k < 2) cin[H + k] = A.extra[I.inst * 2 + k];
  __syncthreads();
  float acc = 0.f;
  const float* Ur = A.P + A.o.U + (int64_t)k * (H + 2);
  for (int j = 0; j < H + 2; ++j) acc = fmaf(Ur[j], cin[j], acc);
  A.q[(int64_t)b * H + k] = acc;
  A.cin[(int64_t)b * (H + 2) + k] = cin[k];
  if (k < 2) A.cin[(int64_t)b * (H + 2) + H + k] = cin[H + k];
}

template <bool TRAIN>
__global__ void __launch_bounds__(256, 1) ws_main_kernel(WsArgs A) {
  extern __shared__ __align__(16) float sm[];
  float* W2s = sm;                                   // [H][LDS]
  float* H1s = W2s + H * kLds;                       // [kTile][LDS]
  float* D2s = H1s + kTile * kLds;                   // [kTile][LDS]   (TRAIN)
  float* red = D2s + (TRAIN ? kTile * kLds : 0);     // [2][16][H]     (TRAIN)
  float* xs = red + (TRAIN ? 2 * 16 * H : 0);        // [kTile][FMAX]
  float* W1s = xs + kTile * FMAX;                    // [H][FMAX]
  float* b1s = W1s + H * FMAX;
  float* b2q = b1s + H;
  float* w3s = b2q + H;
  float* dys = w3s + H;                              // [kTile]
  float* ls = dys + kTile;                           // [kTile]

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int F = A.F;
  const Offs o = A.o;
  for (int e = tid; e < H * H; e += 256) W2s[(e >> 7) * kLds + (e & (H - 1))] = A.P[o.W2 + e];
  for (int e = tid; e < H * FMAX; e += 256) {
    const int k = e / FMAX, f = e % FMAX;
    W1s[e] = f < F ? A.P[o.W1 + k * F + f] : 0.f;
  }
  if (tid < H) { b1s[tid] = A.P[o.b1 + tid]; w3s[tid] = A.P[o.w3 + tid]; }
  const float b3 = A.P[o.b3];

  float gacc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) gacc[i][j] = 0.f;

  for (int t = blockIdx.x; t < A.T; t += gridDim.x) {
    const WsTile tl = A.tiles[t];
    const int cnt = tl.count;
    __syncthreads();                                 // the previous tile is done with shared memory
    for (int e = tid; e < kTile * FMAX; e += 256) {
      const int p = e / FMAX, f = e % FMAX;
      xs[e] = (p < cnt && f < F) ? A.feats[(tl.start + p) * F + f] : 0.f;
    }
    if (tid < H) b2q[tid] = A.P[o.b2 + tid] + A.q[(int64_t)tl.b * H + tid];
    __syncthreads();
    // H1
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int p = ty + 16 * i;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = tx + 16 * j;
        float a = b1s[k];
#pragma unroll
        for (int f = 0; f < FMAX; ++f) a = fmaf(W1s[k * FMAX + f], xs[p * FMAX + f], a);
        H1s[p * kLds + k] = p < cnt ? gelu(a) : 0.f;
      }
    }
    __syncthreads();
    // A2 = H1 W2^T
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 2
    for (int k = 0; k < H; ++k) {
      float a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = H1s[(ty + 16 * i) * kLds + k];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = W2s[(tx + 16 * j) * kLds + k];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    float yp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      yp[i] = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int oc = tx + 16 * j;
        const float a2 = acc[i][j] + b2q[oc];
        acc[i][j] = a2;
        yp[i] = fmaf(w3s[oc], gelu(a2), yp[i]);
      }
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) yp[i] += __shfl_xor_sync(0xffffffffu, yp[i], off);
    }
    if constexpr (!TRAIN) {
      if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int p = ty + 16 * i;
          if (p < cnt) A.y[tl.ybase + p] = yp[i] + b3;
        }
      }
    } else {
    // ---- gradients ----
    float dy[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int p = ty + 16 * i;
      float dd = 0.f, wt = 0.f;
      if (p < cnt) {
        dd = yp[i] + b3 - A.target[tl.start + p];
        wt = A.weight ? A.weight[tl.start + p] : 1.f;
      }
      dy[i] = 2.f * wt * dd * A.invN;
      if (tx == 0) { dys[p] = dy[i]; ls[p] = wt * dd * dd * A.invN; }
    }
    float pw3[8], pdq[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { pw3[j] = 0.f; pdq[j] = 0.f; }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int oc = tx + 16 * j;
        const float a2 = acc[i][j];
        const float d2 = dy[i] * w3s[oc] * gelu_grad(a2);
        D2s[(ty + 16 * i) * kLds + oc] = d2;
        pw3[j] = fmaf(dy[i], gelu(a2), pw3[j]);
        pdq[j] += d2;
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      red[ty * H + tx + 16 * j] = pw3[j];
      red[(16 + ty) * H + tx + 16 * j] = pdq[j];
    }
    __syncthreads();
    if (tid < H) {
      float s = 0.f;
      for (int yy = 0; yy < 16; ++yy) s += red[yy * H + tid];
      A.gw3p[(int64_t)t * H + tid] = s;
    } else {
      const int k = tid - H;
      float s = 0.f;
      for (int yy = 0; yy < 16; ++yy) s += red[(16 + yy) * H + k];
      A.dqp[(int64_t)t * H + k] = s;
    }
    if (tid == 0) {
      float s = 0.f, l = 0.f;
      for (int p = 0; p < cnt; ++p) { s += dys[p]; l += ls[p]; }
      A.gb3p[t] = s;
      A.lossp[t] = l;
    }
    // dW2 += D2^T H1   (rows = output unit ty + 16 i, columns = input unit tx + 16 j)
    for (int p = 0; p < cnt; ++p) {
      float a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = D2s[p * kLds + ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = H1s[p * kLds + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) gacc[i][j] = fmaf(a[i], b[j], gacc[i][j]);
    }
    // dH1 = D2 W2   (rows = point ty + 16 i, columns = input unit tx + 16 j)
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 2
    for (int oc = 0; oc < H; ++oc) {
      float a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = D2s[(ty + 16 * i) * kLds + oc];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = W2s[oc * kLds + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();                                 // every read of H1s and red is done
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) H1s[(ty + 16 * i) * kLds + tx + 16 * j] = acc[i][j];
    __syncthreads();
    // per input unit k: sums over the tile's points (two halves of 64 points)
    {
      const int k = tid & (H - 1), half = tid >> 7;
      float gw[FMAX], mm[FMAX], wk[FMAX];
      float gb = 0.f, ss = 0.f;
#pragma unroll
      for (int f = 0; f < FMAX; ++f) { gw[f] = 0.f; mm[f] = 0.f; wk[f] = W1s[k * FMAX + f]; }
      const int p1 = min(cnt, half * 64 + 64);
      for (int p = half * 64; p < p1; ++p) {
        float a = b1s[k];
#pragma unroll
        for (int f = 0; f < FMAX; ++f) a = fmaf(wk[f], xs[p * FMAX + f], a);
        const float g = gelu_grad(a);
        const float da1 = H1s[p * kLds + k] * g;
#pragma unroll
        for (int f = 0; f < FMAX; ++f) {
          gw[f] = fmaf(da1, xs[p * FMAX + f], gw[f]);
          mm[f] = fmaf(g, xs[p * FMAX + f], mm[f]);
        }
        gb += da1;
        ss += g;
      }
      float* rk = red + k * (2 * FMAX + 2);
      if (half == 1) {
#pragma unroll
        for (int f = 0; f < FMAX; ++f) { rk[f] = gw[f]; rk[FMAX + f] = mm[f]; }
        rk[2 * FMAX] = gb;
        rk[2 * FMAX + 1] = ss;
      }
      __syncthreads();
      if (half == 0) {
        const int64_t base = (int64_t)t * H + k;
        for (int f = 0; f < F; ++f) {
          A.gW1p[base * F + f] = gw[f] + rk[f];
          A.Mp[base * F + f] = mm[f] + rk[FMAX + f];
        }
        A.gb1p[base] = gb + rk[2 * FMAX];
        A.Sp[base] = ss + rk[2 * FMAX + 1];
      }
    }
    }  // TRAIN
  }
  if (TRAIN) {
    float* out = A.gW2p + (int64_t)blockIdx.x * H * H;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) out[(ty + 16 * i) * H + tx + 16 * j] = gacc[i][j];
  }
}

// Per instance of the batch: dq = sum of D2 over its tiles, dctx = (U^T dq)[:H] / n_k,
// and the context share of dW1, db1.
__global__ void __launch_bounds__(H) ws_inst_grad_kernel(WsArgs A) {
  __shared__ float dqs[H];
  const int b = blockIdx.x, k = threadIdx.x;
  const WsInst I = A.binfo[b];
  const int F = A.F;
  float s = 0.f;
  for (int t = I.tile0; t < I.tile0 + I.ntiles; ++t) s += A.dqp[(int64_t)t * H + k];
  dqs[k] = s;
  A.dq[(int64_t)b * H + k] = s;
  __syncthreads();
  float dc = 0.f;
  for (int oc = 0; oc < H; ++oc) dc = fmaf(A.P[A.o.U + (int64_t)oc * (H + 2) + k], dqs[oc], dc);
  dc /= I.npts;
  float S = 0.f, M[FMAX];
#pragma unroll
  for (int f = 0; f < FMAX; ++f) M[f] = 0.f;
  for (int t = I.tile0; t < I.tile0 + I.ntiles; ++t) {
    const int64_t base = (int64_t)t * H + k;
    S += A.Sp[base];
    for (int f = 0; f < F; ++f) M[f] += A.Mp[base * F + f];
  }
  A.cb1[(int64_t)b * H + k] = dc * S;
  for (int f = 0; f < F; ++f) A.cW1[((int64_t)b * H + k) * F + f] = dc * M[f];
}

struct AdamK { float lr, b1, b2, eps, c1, c2; };

// One thread per parameter: the full gradient from the partials (fixed
// order), then either stored or applied with Adam.  Thread 0 also sums the
// loss.
template <bool ADAM>
__global__ void ws_final_kernel(WsArgs A, float* grad, float* P, float* m, float* v, AdamK ak, float* loss) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Offs o = A.o;
  const int F = A.F;
  const bool bad = *A.err != 0;          // a tensor-core wait gave up: no update, NaN loss
  if (e == 0 && loss) {
    float l = 0.f;
    for (int t = 0; t < A.T; ++t) l += A.lossp[t];
    *loss = bad ? __int_as_float(0x7fc00000) : l;
  }
  if (e >= o.total) return;
  float g = 0.f;
  if (e < o.b1) {
    const int64_t k = e / F, f = e % F;
    for (int t = 0; t < A.n_w1p; ++t) g += A.gW1p[((int64_t)t * H + k) * F + f];
    for (int b = 0; b < A.n_cw; ++b) g += A.cW1[((int64_t)b * H + k) * F + f];
  } else if (e < o.W2) {
    const int64_t k = e - o.b1;
    for (int t = 0; t < A.n_w1p; ++t) g += A.gb1p[(int64_t)t * H + k];
    for (int b = 0; b < A.n_cw; ++b) g += A.cb1[(int64_t)b * H + k];
  } else if (e < o.U) {
    const int64_t q = e - o.W2;
    for (int c = 0; c < A.G; ++c) g += A.gW2p[(int64_t)c * H * H + q];
  } else if (e < o.b2) {
    const int64_t q = e - o.U, k = q / (H + 2), j = q % (H + 2);
    for (int b = 0; b < A.B; ++b) g = fmaf(A.dq[(int64_t)b * H + k], A.cin[(int64_t)b * (H + 2) + j], g);
  } else if (e < o.w3) {
    const int64_t k = e - o.b2;
    for (int b = 0; b < A.B; ++b) g += A.dq[(int64_t)b * H + k];
  } else if (e < o.b3) {
    const int64_t k = e - o.w3;
    for (int t = 0; t < A.n_w3p; ++t) g += A.gw3p[(int64_t)t * H + k];
  } else {
    for (int t = 0; t < A.T; ++t) g += A.gb3p[t];
  }
  if (!ADAM) {
    grad[e] = bad ? __int_as_float(0x7fc00000) : g;
  } else if (!bad) {
    const float mm = ak.b1 * m[e] + (1.f - ak.b1) * g;
    const float vv = ak.b2 * v[e] + (1.f - ak.b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    P[e] -= ak.lr * (mm * ak.c1) / (sqrtf(vv * ak.c2) + ak.eps);
  }
}

// ---------------------------------------------------------- host side ---

constexpr size_t kAlign = 256;
size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    sms = 152;
  }
  return sms;
}

struct WsLayout {
  int64_t T = 0, B = 0, G = 0;
  int F = 0;
  size_t o_tiles = 0, o_binfo = 0, o_ctxp = 0, o_cin = 0, o_q = 0, o_gW1p = 0, o_Mp = 0, o_gb1p = 0, o_Sp = 0;
  size_t o_gw3p = 0, o_dqp = 0, o_lossp = 0, o_gb3p = 0, o_dq = 0, o_cW1 = 0, o_cb1 = 0, o_gW2p = 0;
  size_t o_dctx = 0, o_err = 0;
  size_t total = 0;
};

WsLayout ws_layout(int64_t T, int64_t B, int F) {
  WsLayout L;
  L.T = T; L.B = B; L.F = F;
  L.G = std::max<int64_t>(1, std::min<int64_t>(T, device_sms()));
  size_t x = 0;
  auto take = [&](size_t bytes) { const size_t r = x; x = al(x + bytes); return r; };
  L.o_tiles = take(sizeof(WsTile) * T);
  L.o_binfo = take(sizeof(WsInst) * B);
  L.o_ctxp = take(sizeof(float) * T * H);
  L.o_cin = take(sizeof(float) * B * (H + 2));
  L.o_q = take(sizeof(float) * B * H);
  L.o_gW1p = take(sizeof(float) * T * H * F);
  L.o_Mp = take(sizeof(float) * T * H * F);
  L.o_gb1p = take(sizeof(float) * T * H);
  L.o_Sp = take(sizeof(float) * T * H);
  L.o_gw3p = take(sizeof(float) * T * H);
  L.o_dqp = take(sizeof(float) * T * H);
  L.o_lossp = take(sizeof(float) * T);
  L.o_gb3p = take(sizeof(float) * T);
  L.o_dq = take(sizeof(float) * B * H);
  L.o_cW1 = take(sizeof(float) * B * H * F);
  L.o_cb1 = take(sizeof(float) * B * H);
  L.o_gW2p = take(sizeof(float) * L.G * H * H);
  L.o_dctx = take(sizeof(float) * B * H);
  L.o_err = take(sizeof(int));
  L.total = x;
  return L;
}

pot_status check_set(const pot_ws_set* S, bool need_target) {
  if (!S) return wfail(POT_EINVAL, "set is NULL");
  if (S->count < 1) return wfail(POT_EINVAL, "set->count must be >= 1");
  if (S->d < 1 || S->d > POT_WS_MAX_D) return wfail(POT_EINVAL, "set->d must be in [1, %d]", POT_WS_MAX_D);
  if (!S->off || !S->feats || !S->extra) return wfail(POT_EINVAL, "set->off, feats and extra must be non-NULL");
  if (need_target && !S->target) return wfail(POT_EINVAL, "set->target is NULL");
  if (S->off[0] != 0) return wfail(POT_EINVAL, "set->off[0] must be 0");
  for (int64_t k = 0; k < S->count; ++k)
    if (S->off[k + 1] <= S->off[k]) return wfail(POT_EINVAL, "instance %lld has no points", (long long)k);
  return POT_OK;
}

int64_t tiles_of(int64_t npts) { return (npts + kTile - 1) / kTile; }

pot_status check_mode(int32_t mode) {
  if (mode != POT_WS_FP32 && mode != POT_WS_BF16) return wfail(POT_EINVAL, "mode must be POT_WS_FP32 or POT_WS_BF16");
  return POT_OK;
}

size_t main_smem(bool train) {
  size_t f = (size_t)H * kLds + (size_t)kTile * kLds;
  if (train) f += (size_t)kTile * kLds + 2 * 16 * H;
  f += (size_t)kTile * FMAX + (size_t)H * FMAX + 3 * H + 2 * kTile;
  return f * sizeof(float);
}

enum What { kForward = 0, kGradient = 1, kAdam = 2 };

pot_status run_batch(const pot_ws_set* S, const int32_t* idx, int32_t nb, const float* params, int32_t mode,
                     What what, float* y, float* grad, float* loss, float* pm, float* pv, const pot_ws_adam* opt,
                     int64_t step, void* ws, size_t ws_bytes, cudaStream_t st) {
  pot_status s;
  if ((s = check_set(S, what != kForward)) != POT_OK) return s;
  if ((s = check_mode(mode)) != POT_OK) return s;
  if (!idx || nb < 1) return wfail(POT_EINVAL, "idx must hold nb >= 1 indices");
  if (!params) return wfail(POT_EINVAL, "params is NULL");
  if (what == kForward && !y) return wfail(POT_EINVAL, "y is NULL");
  if (what == kGradient && !grad) return wfail(POT_EINVAL, "grad is NULL");
  if (what == kAdam) {
    if (!pm || !pv || !opt) return wfail(POT_EINVAL, "adam_m, adam_v and opt must be non-NULL");
    if (step < 1) return wfail(POT_EINVAL, "step must be >= 1");
    if (!(opt->lr > 0.f) || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) || !(opt->beta2 >= 0.f && opt->beta2 < 1.f) ||
        !(opt->eps > 0.f))
      return wfail(POT_EINVAL, "Adam needs lr > 0, 0 <= beta < 1, eps > 0");
  }
  if (!ws) return wfail(POT_EINVAL, "workspace is NULL");
  const int F = S->d + POT_WS_EXTRA;
  std::vector<WsTile> tiles;
  std::vector<WsInst> binfo(nb);
  int64_t ybase = 0;
  for (int b = 0; b < nb; ++b) {
    const int32_t k = idx[b];
    if (k < 0 || k >= S->count) return wfail(POT_EINVAL, "idx[%d] = %d out of range", b, k);
    const int64_t n0 = S->off[k], npts = S->off[k + 1] - n0;
    if (npts > (int64_t(1) << 30)) return wfail(POT_EINVAL, "instance %d too large", k);
    binfo[b].inst = k;
    binfo[b].tile0 = (int32_t)tiles.size();
    binfo[b].ntiles = (int32_t)tiles_of(npts);
    binfo[b].npts = (float)npts;
    for (int64_t q = 0; q < npts; q += kTile) {
      WsTile t;
      t.start = n0 + q;
      t.ybase = ybase + q;
      t.b = b;
      t.count = (int32_t)std::min<int64_t>(kTile, npts - q);
      tiles.push_back(t);
    }
    ybase += npts;
  }
  const int64_t T = (int64_t)tiles.size();
  if (T > (int64_t(1) << 30)) return wfail(POT_EINVAL, "batch too large");
  const WsLayout L = ws_layout(T, nb, F);
  if (ws_bytes < L.total)
    return wfail(POT_ENOMEM, "workspace too small: %zu bytes, this batch needs %zu", ws_bytes, L.total);
  char* base = static_cast<char*>(ws);
  if (((uintptr_t)base & 255) != 0) return wfail(POT_EINVAL, "workspace must be 256-byte aligned");
  WCK(cudaMemcpyAsync(base + L.o_tiles, tiles.data(), sizeof(WsTile) * T, cudaMemcpyHostToDevice, st));
  WCK(cudaMemcpyAsync(base + L.o_binfo, binfo.data(), sizeof(WsInst) * nb, cudaMemcpyHostToDevice, st));

  WsArgs A{};
  A.F = F; A.T = (int)T; A.B = nb; A.G = (int)L.G;
  A.o = offsets(S->d);
  A.tiles = reinterpret_cast<const WsTile*>(base + L.o_tiles);
  A.binfo = reinterpret_cast<const WsInst*>(base + L.o_binfo);
  A.feats = S->feats; A.extra = S->extra; A.target = S->target; A.weight = S->weight; A.P = params;
  A.ctxp = reinterpret_cast<float*>(base + L.o_ctxp);
  A.cin = reinterpret_cast<float*>(base + L.o_cin);
  A.q = reinterpret_cast<float*>(base + L.o_q);
  A.y = y;
  A.invN = (float)(1.0 / (double)ybase);
  A.gW1p = reinterpret_cast<float*>(base + L.o_gW1p);
  A.Mp = reinterpret_cast<float*>(base + L.o_Mp);
  A.gb1p = reinterpret_cast<float*>(base + L.o_gb1p);
  A.Sp = reinterpret_cast<float*>(base + L.o_Sp);
  A.gw3p = reinterpret_cast<float*>(base + L.o_gw3p);
  A.dqp = reinterpret_cast<float*>(base + L.o_dqp);
  A.lossp = reinterpret_cast<float*>(base + L.o_lossp);
  A.gb3p = reinterpret_cast<float*>(base + L.o_gb3p);
  A.dq = reinterpret_cast<float*>(base + L.o_dq);
  A.cW1 = reinterpret_cast<float*>(base + L.o_cW1);
  A.cb1 = reinterpret_cast<float*>(base + L.o_cb1);
  A.gW2p = reinterpret_cast<float*>(base + L.o_gW2p);
  A.dctx = reinterpret_cast<float*>(base + L.o_dctx);
  A.err = reinterpret_cast<int*>(base + L.o_err);
  const bool tc = mode == POT_WS_BF16;
  A.n_w1p = tc ? (int)L.G : (int)T;
  A.n_cw = tc ? 0 : nb;
  A.n_w3p = tc ? (int)L.G : (int)T;

  ws_ctx_kernel<<<(unsigned)T, H, 0, st>>>(A);
  ws_q_kernel<<<(unsigned)nb, H, 0, st>>>(A);
  WCKL();
  const bool train = what != kForward;
  if (mode == POT_WS_BF16) {
    if ((s = launch_ws_main_tc(A, train, st)) != POT_OK) return s;
  } else {
    const size_t smem = main_smem(train);
    if (train) {
      WCK(cudaFuncSetAttribute(ws_main_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      ws_main_kernel<true><<<(unsigned)L.G, 256, smem, st>>>(A);
    } else {
      WCK(cudaFuncSetAttribute(ws_main_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      ws_main_kernel<false><<<(unsigned)L.G, 256, smem, st>>>(A);
    }
    WCKL();
  }
  if (!train) return POT_OK;
  if (!tc) {
    WCK(cudaMemsetAsync(A.err, 0, sizeof(int), st));
    ws_inst_grad_kernel<<<(unsigned)nb, H, 0, st>>>(A);
  }
  const unsigned fb = (unsigned)((A.o.total + 255) / 256);
  AdamK ak{};
  if (what == kAdam) {
    ak.lr = opt->lr; ak.b1 = opt->beta1; ak.b2 = opt->beta2; ak.eps = opt->eps;
    ak.c1 = (float)(1.0 / (1.0 - pow((double)opt->beta1, (double)step)));
    ak.c2 = (float)(1.0 / (1.0 - pow((double)opt->beta2, (double)step)));
    ws_final_kernel<true><<<fb, 256, 0, st>>>(A, nullptr, const_cast<float*>(params), pm, pv, ak, loss);
  } else {
    ws_final_kernel<false><<<fb, 256, 0, st>>>(A, grad, nullptr, nullptr, nullptr, ak, loss);
  }
  WCKL();
  return POT_OK;
}

bool is_points(const pot_problem* p) {
  return p->kind == POT_COST_SQEUCLID_BF16 || p->kind == POT_COST_SQEUCLID_F16 || p->kind == POT_COST_SQEUCLID_F32;
}

pot_status check_points_problem(const pot_problem* prob) {
  if (!prob) return wfail(POT_EINVAL, "problem is NULL");
  if (!is_points(prob)) return wfail(POT_EINVAL, "the warm start needs a squared-Euclidean point problem");
  if (prob->d < 1 || prob->d > POT_WS_MAX_D) return wfail(POT_EINVAL, "d must be in [1, %d]", POT_WS_MAX_D);
  return POT_OK;
}

}  // namespace

extern "C" {

POT_API pot_status pot_ws_param_count(int32_t d, int64_t* count) {
  if (d < 1 || d > POT_WS_MAX_D) return wfail(POT_EINVAL, "d must be in [1, %d]", POT_WS_MAX_D);
  if (!count) return wfail(POT_EINVAL, "count is NULL");
  *count = offsets(d).total;
  return POT_OK;
}

POT_API pot_status pot_ws_init(float* params, int32_t d, uint64_t seed, void* stream) {
  if (d < 1 || d > POT_WS_MAX_D) return wfail(POT_EINVAL, "d must be in [1, %d]", POT_WS_MAX_D);
  if (!params) return wfail(POT_EINVAL, "params is NULL");
  const Offs o = offsets(d);
  ws_init_kernel<<<(unsigned)((o.total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, o, seed);
  WCKL();
  return POT_OK;
}

// Features workspace: [solver scratch][stats 16][lu n][lv m][lrow TEMPS n][lcol TEMPS m]
static pot_status feat_layout(const pot_problem* prob, size_t* o_stats, size_t* o_lu, size_t* o_lv, size_t* o_lrow,
                              size_t* o_lcol, size_t* total) {
  pot_status s;
  size_t solver = 0;
  if ((s = pot_workspace_size(prob, nullptr, &solver)) != POT_OK) return s;
  size_t x = al(solver);
  *o_stats = x; x = al(x + sizeof(double) * 16);
  *o_lu = x; x = al(x + sizeof(double) * prob->n);
  *o_lv = x; x = al(x + sizeof(double) * prob->m);
  *o_lrow = x; x = al(x + sizeof(double) * prob->n * POT_WS_TEMPS);
  *o_lcol = x; x = al(x + sizeof(double) * prob->m * POT_WS_TEMPS);
  *total = x;
  return POT_OK;
}

POT_API pot_status pot_ws_features_workspace_size(const pot_problem* prob, size_t* bytes) {
  pot_status s;
  if ((s = check_points_problem(prob)) != POT_OK) return s;
  if (!bytes) return wfail(POT_EINVAL, "bytes is NULL");
  size_t a, b, c, d, e;
  return feat_layout(prob, &a, &b, &c, &d, &e, bytes);
}

POT_API pot_status pot_ws_features(const pot_problem* prob, double gamma, void* workspace, size_t ws_bytes,
                                   float* feats, float* extra, void* stream) {
  pot_status s;
  if ((s = check_points_problem(prob)) != POT_OK) return s;
  if (!(gamma > 0.0) || !isfinite(gamma)) return wfail(POT_EINVAL, "gamma must be finite and > 0");
  if (!feats || !extra) return wfail(POT_EINVAL, "feats and extra must be non-NULL");
  size_t o_stats, o_lu, o_lv, o_lrow, o_lcol, need;
  if ((s = feat_layout(prob, &o_stats, &o_lu, &o_lv, &o_lrow, &o_lcol, &need)) != POT_OK) return s;
  if (!workspace || ws_bytes < need) return wfail(POT_ENOMEM, "workspace too small (%zu < %zu)", ws_bytes, need);
  char* base = static_cast<char*>(workspace);
  if (((uintptr_t)base & 255) != 0) return wfail(POT_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  pot_problem q = *prob;
  if (!(q.cost_scale > 0.0)) {
    double mx = 0.0;
    if ((s = pot_cost_max(prob, base, o_stats, &mx, stream)) != POT_OK) return s;
    q.cost_scale = mx > 0.0 ? 1.0 / mx : 1.0;
  }
  double* stats = reinterpret_cast<double*>(base + o_stats);
  double* lu = reinterpret_cast<double*>(base + o_lu);
  double* lv = reinterpret_cast<double*>(base + o_lv);
  double* lrow = reinterpret_cast<double*>(base + o_lrow);
  double* lcol = reinterpret_cast<double*>(base + o_lcol);
  const int64_t N = q.n + q.m;
  ws_stats_kernel<<<1, 1024, 0, st>>>(q.kind, q.X, q.Y, q.ldx, q.ldy, q.d, q.n, q.m, q.r, q.c, stats);
  ws_logmass_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(q.n, q.m, q.r, q.c, stats, lu, lv);
  WCKL();
  double T = gamma;
  for (int t = 0; t < POT_WS_TEMPS; ++t, T *= 4.0)
    if ((s = pot_marginals(&q, T, lu, lv, 0.0, base, o_stats, lrow + t * q.n, lcol + t * q.m, nullptr, stream)) != POT_OK)
      return s;
  ws_feat_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(q.kind, q.X, q.Y, q.ldx, q.ldy, q.d, q.n, q.m, q.r,
                                                               q.c, q.s, sqrt(q.cost_scale), gamma, stats, lu, lv,
                                                               lrow, lcol, feats, extra);
  WCKL();
  return POT_OK;
}

POT_API pot_status pot_ws_targets(const pot_problem* prob, double gamma, const double* u, const double* v, double w,
                                  float* target, float* weight, void* workspace, size_t ws_bytes, void* stream) {
  pot_status s;
  if ((s = check_points_problem(prob)) != POT_OK) return s;
  if (!(gamma > 0.0) || !isfinite(gamma)) return wfail(POT_EINVAL, "gamma must be finite and > 0");
  if (!isfinite(w)) return wfail(POT_EINVAL, "w must be finite");
  if (!u || !v || !target) return wfail(POT_EINVAL, "u, v and target must be non-NULL");
  size_t o_stats, o_lu, o_lv, o_lrow, o_lcol, need;
  if ((s = feat_layout(prob, &o_stats, &o_lu, &o_lv, &o_lrow, &o_lcol, &need)) != POT_OK) return s;
  if (!workspace || ws_bytes < need) return wfail(POT_ENOMEM, "workspace too small (%zu < %zu)", ws_bytes, need);
  char* base = static_cast<char*>(workspace);
  if (((uintptr_t)base & 255) != 0) return wfail(POT_EINVAL, "workspace must be 256-byte aligned");
  pot_problem q = *prob;
  if (!(q.cost_scale > 0.0)) {
    double mx = 0.0;
    if ((s = pot_cost_max(prob, base, o_stats, &mx, stream)) != POT_OK) return s;
    q.cost_scale = mx > 0.0 ? 1.0 / mx : 1.0;
  }
  double* lrow = reinterpret_cast<double*>(base + o_lrow);
  double* lcol = reinterpret_cast<double*>(base + o_lcol);
  if ((s = pot_marginals(&q, gamma, u, v, w, base, o_stats, lrow, lcol, nullptr, stream)) != POT_OK) return s;
  const int64_t n = q.n, m = q.m;
  ws_targets_kernel<<<(unsigned)((n + m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, m, gamma, lrow, lcol, u,
                                                                                        v, target, weight);
  WCKL();
  return POT_OK;
}

POT_API pot_status pot_ws_workspace_size(const pot_ws_set* set, int32_t max_batch, size_t* bytes) {
  pot_status s;
  if ((s = check_set(set, false)) != POT_OK) return s;
  if (max_batch < 1) return wfail(POT_EINVAL, "max_batch must be >= 1");
  if (!bytes) return wfail(POT_EINVAL, "bytes is NULL");
  std::vector<int64_t> t(set->count);
  for (int64_t k = 0; k < set->count; ++k) t[k] = tiles_of(set->off[k + 1] - set->off[k]);
  std::sort(t.begin(), t.end(), std::greater<int64_t>());
  int64_t T = 0;
  const int64_t B = std::min<int64_t>(max_batch, set->count);
  for (int64_t k = 0; k < B; ++k) T += t[k];
  *bytes = ws_layout(T, std::max<int64_t>(B, max_batch), set->d + POT_WS_EXTRA).total;
  return POT_OK;
}

POT_API pot_status pot_ws_forward(const pot_ws_set* set, const int32_t* idx, int32_t nb, const float* params,
                                  int32_t mode, float* y, void* workspace, size_t ws_bytes, void* stream) {
  return run_batch(set, idx, nb, params, mode, kForward, y, nullptr, nullptr, nullptr, nullptr, nullptr, 0, workspace,
                   ws_bytes, (cudaStream_t)stream);
}

POT_API pot_status pot_ws_gradient(const pot_ws_set* set, const int32_t* idx, int32_t nb, const float* params,
                                   int32_t mode, float* grad, float* loss, void* workspace, size_t ws_bytes,
                                   void* stream) {
  return run_batch(set, idx, nb, params, mode, kGradient, nullptr, grad, loss, nullptr, nullptr, nullptr, 0,
                   workspace, ws_bytes, (cudaStream_t)stream);
}

POT_API pot_status pot_ws_train_step(const pot_ws_set* set, const int32_t* idx, int32_t nb, float* params,
                                     float* adam_m, float* adam_v, const pot_ws_adam* opt, int64_t step,
                                     int32_t mode, float* loss, void* workspace, size_t ws_bytes, void* stream) {
  return run_batch(set, idx, nb, params, mode, kAdam, nullptr, nullptr, loss, adam_m, adam_v, opt, step, workspace,
                   ws_bytes, (cudaStream_t)stream);
}

// Warm-start workspace: [features scratch (solver scratch first)][feats][extra][y][network scratch][tot]
static pot_status warm_layout(const pot_problem* prob, size_t* o_feat, size_t* o_extra, size_t* o_y, size_t* o_net,
                              size_t* o_tot, size_t* total) {
  pot_status s;
  size_t a, b, c, d, e, fws = 0;
  if ((s = feat_layout(prob, &a, &b, &c, &d, &e, &fws)) != POT_OK) return s;
  const int64_t N = prob->n + prob->m;
  const int F = prob->d + POT_WS_EXTRA;
  size_t x = al(fws);
  *o_feat = x; x = al(x + sizeof(float) * N * F);
  *o_extra = x; x = al(x + sizeof(float) * 2);
  *o_y = x; x = al(x + sizeof(float) * N);
  *o_net = x; x = al(x + ws_layout(tiles_of(N), 1, F).total);
  *o_tot = x; x = al(x + 4 * sizeof(double));
  *total = x;
  return POT_OK;
}

POT_API pot_status pot_ws_warm_workspace_size(const pot_problem* prob, size_t* bytes) {
  pot_status s;
  if ((s = check_points_problem(prob)) != POT_OK) return s;
  if (!bytes) return wfail(POT_EINVAL, "bytes is NULL");
  size_t a, b, c, d, e;
  return warm_layout(prob, &a, &b, &c, &d, &e, bytes);
}

POT_API pot_status pot_ws_warm_start(const pot_problem* prob, double gamma, const float* params, int32_t d,
                                     int32_t mode, double* u0, double* v0, double* w0, void* workspace,
                                     size_t ws_bytes, void* stream) {
  pot_status s;
  if ((s = check_points_problem(prob)) != POT_OK) return s;
  if ((s = check_mode(mode)) != POT_OK) return s;
  if (prob->d != d) return wfail(POT_EINVAL, "network dimension %d differs from the problem's d = %d", d, prob->d);
  if (!(gamma > 0.0) || !isfinite(gamma)) return wfail(POT_EINVAL, "gamma must be finite and > 0");
  if (!params || !u0 || !v0 || !w0) return wfail(POT_EINVAL, "params, u0, v0 and w0 must be non-NULL");
  if (!workspace) return wfail(POT_EINVAL, "workspace is NULL");
  size_t o_feat, o_extra, o_y, o_net, o_tot, total;
  if ((s = warm_layout(prob, &o_feat, &o_extra, &o_y, &o_net, &o_tot, &total)) != POT_OK) return s;
  if (ws_bytes < total) return wfail(POT_ENOMEM, "workspace too small (%zu < %zu)", ws_bytes, total);
  char* base = static_cast<char*>(workspace);
  if (((uintptr_t)base & 255) != 0) return wfail(POT_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  float* feats = reinterpret_cast<float*>(base + o_feat);
  float* extra = reinterpret_cast<float*>(base + o_extra);
  float* y = reinterpret_cast<float*>(base + o_y);
  double* tot = reinterpret_cast<double*>(base + o_tot);
  // the effective cost scale, as the solver's prologue computes it
  pot_problem q = *prob;
  if (!(q.cost_scale > 0.0)) {
    double mx = 0.0;
    if ((s = pot_cost_max(prob, base, o_feat, &mx, stream)) != POT_OK) return s;
    q.cost_scale = mx > 0.0 ? 1.0 / mx : 1.0;
  }
  prob = &q;
  if ((s = pot_ws_features(prob, gamma, base, o_feat, feats, extra, stream)) != POT_OK) return s;
  size_t f_stats, f_lu, f_lv, f_lrow, f_lcol, f_total;
  if ((s = feat_layout(prob, &f_stats, &f_lu, &f_lv, &f_lrow, &f_lcol, &f_total)) != POT_OK) return s;
  const double* stats = reinterpret_cast<const double*>(base + f_stats);   // masses, from the features call
  const int64_t N = prob->n + prob->m;
  const int64_t off[2] = {0, N};
  pot_ws_set set{};
  set.count = 1; set.d = d; set.off = off; set.feats = feats; set.extra = extra; set.target = nullptr;
  const int32_t idx = 0;
  if ((s = pot_ws_forward(&set, &idx, 1, params, mode, y, base + o_net, total - o_net, stream)) != POT_OK) return s;
  ws_to_duals_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(prob->n, prob->m, 1.0 / gamma, prob->r, prob->c,
                                                                   stats, y, u0, v0);
  WCKL();
  if ((s = pot_marginals(prob, gamma, u0, v0, 0.0, base, f_stats, nullptr, nullptr, tot, stream)) != POT_OK) return s;
  double* shift = tot + 1;
  ws_shift_kernel<<<1, 1024, 0, st>>>(prob->n, prob->m, u0, v0, stats, prob->s, tot, shift);
  ws_apply_shift_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(prob->n, prob->m, shift, u0, v0);
  WCKL();
  double h[4] = {0, 0, 0, 0};
  WCK(cudaMemcpyAsync(h, tot, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WCK(cudaStreamSynchronize(st));
  if (!(h[0] > 0.0) || !isfinite(h[0])) return wfail(POT_ENONFINITE, "|B(u0, v0, 0)|_1 = %g is not a positive number", h[0]);
  if (!isfinite(h[1]) || !isfinite(h[2]) || !isfinite(h[3])) return wfail(POT_ENONFINITE, "non-finite warm-start shift");
  *w0 = h[3];
  return POT_OK;
}

}  // extern "C"
