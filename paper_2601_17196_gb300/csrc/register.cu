// Rigid registration steps (include/registration.h): the moments of each
// instance's rounded plan, the weighted Procrustes fit by a one-sided Jacobi
// SVD, and the motion applied to the source cloud.
//
// pot_rigid_fit: one CTA per instance.  Threads own rows i of the plan; the
// columns are staged through shared memory 512 at a time (current source
// point, original source point, g_j) and every thread sums
//   w_ij = exp(f_i + g_j - cost_scale |x_i - y_j|^2 / gamma)
// and w_ij y0_j over j in FP32 (entries of a feasible plan are <= 1, so no
// shift is needed); the rank-one part kappa p_i q_j adds kappa p_i (|q|_1,
// sum_j q_j y0_j).  The 16 moments |pi|, sum a_i x_i, sum_ij pi_ij y0_j and
// sum_i x_i (sum_j pi_ij y0_j)^T are reduced over the CTA in FP64, and thread
// 0 finishes the fit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <vector>

#include "../../include/registration.h"
#include "common.cuh"

namespace pot {
pot_status set_last_error(pot_status s, const char* msg);
}

namespace {

constexpr int kRT = 256;
constexpr int kRChunk = 512;
constexpr double kLog2e = 1.4426950408889634;

struct RgInst {
  int64_t n, m;
  const float* X;
  float* Y;
  const float* Y0;
  const double *f, *g, *p, *q, *kappa;
  double gC2;        // cost_scale / gamma * log2(e)
};

pot_status rfail(pot_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return pot::set_last_error(s, buf);
}

// Sum of v[0..NV) over the CTA; the totals land in out[] (shared) for all threads.
template <int NV>
__device__ void cta_sums(double (&v)[NV], double* sh /* [NV][kRT/32] */, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k * (kRT / 32) + warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double a = 0.0;
    for (int w = 0; w < kRT / 32; ++w) a += sh[threadIdx.x * (kRT / 32) + w];
    out[threadIdx.x] = a;
  }
  __syncthreads();
}

// Weighted Procrustes from M = U S V^T (one-sided Jacobi on the columns of M):
// R = U diag(..., det(U V^T) at the smallest singular value, ...) V^T.
__device__ void jacobi_fit(const double (&M)[9], double (&R)[9], double* dsign, double* sweeps) {
  double A[3][3], V[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) { A[r][c] = M[3 * r + c]; V[r][c] = (r == c) ? 1.0 : 0.0; }
  int sw = 0;
  for (; sw < 40; ++sw) {
    bool rotated = false;
    for (int pair = 0; pair < 3; ++pair) {
      const int p = pair == 2 ? 1 : 0, q = pair == 0 ? 1 : 2;
      double al = 0, be = 0, ga = 0;
      for (int k = 0; k < 3; ++k) { al += A[k][p] * A[k][p]; be += A[k][q] * A[k][q]; ga += A[k][p] * A[k][q]; }
      if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
      rotated = true;
      const double ze = (be - al) / (2.0 * ga);
      const double t = (ze >= 0.0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(1.0 + ze * ze));
      const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
      for (int k = 0; k < 3; ++k) {
        const double ap = A[k][p], aq = A[k][q];
        A[k][p] = cs * ap - sn * aq;
        A[k][q] = sn * ap + cs * aq;
        const double vp = V[k][p], vq = V[k][q];
        V[k][p] = cs * vp - sn * vq;
        V[k][q] = sn * vp + cs * vq;
      }
    }
    if (!rotated) break;
  }
  double sig[3], U[3][3];
  for (int c = 0; c < 3; ++c) sig[c] = sqrt(A[0][c] * A[0][c] + A[1][c] * A[1][c] + A[2][c] * A[2][c]);
  int kmin = 0;
  for (int c = 1; c < 3; ++c) if (sig[c] < sig[kmin]) kmin = c;
  const double smax = fmax(sig[0], fmax(sig[1], sig[2]));
  for (int c = 0; c < 3; ++c)
    for (int r = 0; r < 3; ++r) U[r][c] = (c != kmin && sig[c] > 0.0) ? A[r][c] / sig[c] : 0.0;
  const int k1 = (kmin + 1) % 3, k2 = (kmin + 2) % 3;
  if (!(smax > 0.0)) {                       // no correlation at all (e.g. one target point): no rotation
    for (int k = 0; k < 9; ++k) R[k] = (k % 4 == 0) ? 1.0 : 0.0;
    *dsign = 1.0;
    *sweeps = sw;
    return;
  }
  if (sig[kmin] > 1e-12 * smax) {
    for (int r = 0; r < 3; ++r) U[r][kmin] = A[r][kmin] / sig[kmin];
  } else {                                   // rank-deficient: complete U to an orthonormal basis
    int kmid = sig[k1] < sig[k2] ? k1 : k2, kbig = sig[k1] < sig[k2] ? k2 : k1;
    if (!(sig[kmid] > 1e-12 * smax)) {
      // rank one: any unit vector orthogonal to the one valid column, by the
      // cross product with the coordinate axis it is least aligned with
      int ax = 0;
      for (int r = 1; r < 3; ++r) if (fabs(U[r][kbig]) < fabs(U[ax][kbig])) ax = r;
      double e[3] = {0.0, 0.0, 0.0};
      e[ax] = 1.0;
      double w[3] = {U[1][kbig] * e[2] - U[2][kbig] * e[1], U[2][kbig] * e[0] - U[0][kbig] * e[2],
                     U[0][kbig] * e[1] - U[1][kbig] * e[0]};
      const double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
      for (int r = 0; r < 3; ++r) U[r][kmid] = w[r] / nw;
    }
    U[0][kmin] = U[1][k1] * U[2][k2] - U[2][k1] * U[1][k2];
    U[1][kmin] = U[2][k1] * U[0][k2] - U[0][k1] * U[2][k2];
    U[2][kmin] = U[0][k1] * U[1][k2] - U[1][k1] * U[0][k2];
  }
  auto det3 = [](const double (&B)[3][3]) {
    return B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) - B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
           B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
  };
  const double d = (det3(U) * det3(V) < 0.0) ? -1.0 : 1.0;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += U[r][k] * (k == kmin ? d : 1.0) * V[c][k];
      R[3 * r + c] = a;
    }
  *dsign = d;
  *sweeps = sw;
}

__global__ void __launch_bounds__(kRT) rigid_fit_kernel(const RgInst* insts, double* fit) {
  const RgInst I = insts[blockIdx.x];
  __shared__ float sY[kRChunk * 3], sY0[kRChunk * 3], sG[kRChunk];
  __shared__ double sh[16 * (kRT / 32)];
  __shared__ double tot[16];
  const int tid = threadIdx.x;
  // rank-one column sums |q|_1, sum_j q_j y0_j
  {
    double v[4] = {0, 0, 0, 0};
    for (int64_t j = tid; j < I.m; j += kRT) {
      const double qj = I.q[j];
      v[0] += qj;
      v[1] += qj * I.Y0[3 * j];
      v[2] += qj * I.Y0[3 * j + 1];
      v[3] += qj * I.Y0[3 * j + 2];
    }
    cta_sums<4>(v, sh, tot);
  }
  const double Q0 = tot[0], Q1 = tot[1], Q2 = tot[2], Q3 = tot[3];
  const double kap = *I.kappa;
  const float gC2 = (float)I.gC2;
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  const int64_t rounds = (I.n + kRT - 1) / kRT;
  for (int64_t it = 0; it < rounds; ++it) {
    const int64_t i = it * kRT + tid;
    const bool live = i < I.n;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, fi = 0.f;
    if (live) {
      x0 = I.X[3 * i]; x1 = I.X[3 * i + 1]; x2 = I.X[3 * i + 2];
      fi = (float)(I.f[i] * kLog2e);
    }
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int64_t j0 = 0; j0 < I.m; j0 += kRChunk) {
      const int cnt = (int)((I.m - j0) < kRChunk ? (I.m - j0) : kRChunk);
      __syncthreads();
      for (int e = tid; e < cnt; e += kRT) {
        const int64_t j = j0 + e;
        sY[3 * e] = I.Y[3 * j]; sY[3 * e + 1] = I.Y[3 * j + 1]; sY[3 * e + 2] = I.Y[3 * j + 2];
        sY0[3 * e] = I.Y0[3 * j]; sY0[3 * e + 1] = I.Y0[3 * j + 1]; sY0[3 * e + 2] = I.Y0[3 * j + 2];
        sG[e] = (float)(I.g[j] * kLog2e);
      }
      __syncthreads();
      if (live) {
        for (int e = 0; e < cnt; ++e) {
          const float d0 = x0 - sY[3 * e], d1 = x1 - sY[3 * e + 1], d2 = x2 - sY[3 * e + 2];
          const float c = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
          const float w = pot::ex2(fmaf(-gC2, c, fi + sG[e]));
          s0 += w;
          s1 = fmaf(w, sY0[3 * e], s1);
          s2 = fmaf(w, sY0[3 * e + 1], s2);
          s3 = fmaf(w, sY0[3 * e + 2], s3);
        }
      }
    }
    if (live) {
      const double pk = kap * I.p[i];
      const double a = (double)s0 + pk * Q0;
      const double w0 = (double)s1 + pk * Q1, w1 = (double)s2 + pk * Q2, w2 = (double)s3 + pk * Q3;
      const double xs[3] = {x0, x1, x2}, ws[3] = {w0, w1, w2};
      acc[0] += a;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        acc[1 + r] += a * xs[r];
        acc[4 + r] += ws[r];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[7 + 3 * r + c] += xs[r] * ws[c];
      }
    }
  }
  cta_sums<16>(acc, sh, tot);
  if (tid == 0) {
    double* out = fit + (int64_t)blockIdx.x * POT_RIGID_FIT_STRIDE;
    const double mass = tot[0];
    double ux[3], uy[3], M[9], R[9], d = 1.0, sw = 0.0;
    for (int r = 0; r < 3; ++r) { ux[r] = tot[1 + r] / mass; uy[r] = tot[4 + r] / mass; }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[3 * r + c] = tot[7 + 3 * r + c] - mass * ux[r] * uy[c];
    jacobi_fit(M, R, &d, &sw);
    for (int k = 0; k < 9; ++k) out[k] = R[k];
    for (int r = 0; r < 3; ++r) out[9 + r] = ux[r] - (R[3 * r] * uy[0] + R[3 * r + 1] * uy[1] + R[3 * r + 2] * uy[2]);
    out[12] = mass;
    out[13] = d;
    out[14] = sw;
    out[15] = 0.0;
  }
}

__global__ void rigid_apply_kernel(const RgInst* insts, const double* fit) {
  const RgInst I = insts[blockIdx.y];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= I.m) return;
  const double* F = fit + (int64_t)blockIdx.y * POT_RIGID_FIT_STRIDE;
  const double y0[3] = {I.Y0[3 * j], I.Y0[3 * j + 1], I.Y0[3 * j + 2]};
  for (int r = 0; r < 3; ++r)
    I.Y[3 * j + r] = (float)(F[3 * r] * y0[0] + F[3 * r + 1] * y0[1] + F[3 * r + 2] * y0[2] + F[9 + r]);
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

pot_status build(const pot_problem* probs, int32_t count, const pot_plan* plans, double gamma,
                 const float* const* y0, void* ws, size_t ws_bytes, cudaStream_t st, int64_t* max_m,
                 RgInst** dev) {
  if (!probs || count < 1) return rfail(POT_EINVAL, "probs must hold count >= 1 problems");
  if (!y0) return rfail(POT_EINVAL, "y0 is NULL");
  const size_t need = al256(sizeof(RgInst) * (size_t)count);
  if (!ws || ws_bytes < need) return rfail(POT_ENOMEM, "workspace too small (%zu < %zu)", ws_bytes, need);
  if (((uintptr_t)ws & 255) != 0) return rfail(POT_EINVAL, "workspace must be 256-byte aligned");
  std::vector<RgInst> h(count);
  *max_m = 0;
  for (int32_t k = 0; k < count; ++k) {
    const pot_problem& P = probs[k];
    if (P.kind != POT_COST_SQEUCLID_F32 || P.d != 3 || P.ldx != 3 || P.ldy != 3)
      return rfail(POT_EINVAL, "instance %d: registration needs FP32 points with d = ldx = ldy = 3", k);
    if (P.n < 1 || P.m < 1 || !P.X || !P.Y || !y0[k]) return rfail(POT_EINVAL, "instance %d: bad sizes or points", k);
    if (!(P.cost_scale > 0.0) || !isfinite(P.cost_scale))
      return rfail(POT_EINVAL, "instance %d: registration needs an explicit cost_scale > 0", k);
    RgInst& I = h[k];
    I.n = P.n; I.m = P.m;
    I.X = static_cast<const float*>(P.X);
    I.Y = const_cast<float*>(static_cast<const float*>(P.Y));
    I.Y0 = y0[k];
    if (plans) {
      const pot_plan& L = plans[k];
      if (!L.f || !L.g || !L.p || !L.q || !L.kappa) return rfail(POT_EINVAL, "instance %d: plan pointers are NULL", k);
      I.f = L.f; I.g = L.g; I.p = L.p; I.q = L.q; I.kappa = L.kappa;
      I.gC2 = P.cost_scale / gamma * kLog2e;
    }
    if (P.m > *max_m) *max_m = P.m;
  }
  RgInst* d = static_cast<RgInst*>(ws);
  if (cudaMemcpyAsync(d, h.data(), sizeof(RgInst) * (size_t)count, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return rfail(POT_ECUDA, "copy of the instance table failed");
  *dev = d;
  return POT_OK;
}

}  // namespace

extern "C" {

POT_API pot_status pot_rigid_workspace_size(int32_t count, size_t* bytes) {
  if (count < 1) return rfail(POT_EINVAL, "count must be >= 1");
  if (!bytes) return rfail(POT_EINVAL, "bytes is NULL");
  *bytes = al256(sizeof(RgInst) * (size_t)count);
  return POT_OK;
}

POT_API pot_status pot_rigid_fit(const pot_problem* probs, int32_t count, const pot_plan* plans, double gamma,
                                 const float* const* y0, double* fit, void* workspace, size_t ws_bytes,
                                 void* stream) {
  if (!plans) return rfail(POT_EINVAL, "plans is NULL");
  if (!fit) return rfail(POT_EINVAL, "fit is NULL");
  if (!(gamma > 0.0) || !isfinite(gamma)) return rfail(POT_EINVAL, "gamma must be finite and > 0");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t max_m = 0;
  RgInst* d = nullptr;
  pot_status s = build(probs, count, plans, gamma, y0, workspace, ws_bytes, st, &max_m, &d);
  if (s != POT_OK) return s;
  rigid_fit_kernel<<<(unsigned)count, kRT, 0, st>>>(d, fit);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rfail(POT_ECUDA, "rigid_fit_kernel: %s", cudaGetErrorString(e));
  return POT_OK;
}

POT_API pot_status pot_rigid_apply(const pot_problem* probs, int32_t count, const float* const* y0,
                                   const double* fit, void* workspace, size_t ws_bytes, void* stream) {
  if (!fit) return rfail(POT_EINVAL, "fit is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t max_m = 0;
  RgInst* d = nullptr;
  pot_status s = build(probs, count, nullptr, 1.0, y0, workspace, ws_bytes, st, &max_m, &d);
  if (s != POT_OK) return s;
  dim3 grid((unsigned)((max_m + 255) / 256), (unsigned)count);
  rigid_apply_kernel<<<grid, 256, 0, st>>>(d, fit);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rfail(POT_ECUDA, "rigid_apply_kernel: %s", cudaGetErrorString(e));
  return POT_OK;
}

}  // extern "C"
