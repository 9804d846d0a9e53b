// CUDA-core passes over the Gibbs matrix B(z) of entropic POT.
//
// Used for the dense FP32 cost (HBM-bound: 4 bytes of C per entry) and for
// squared-Euclidean costs of low-dimensional points (d <= 4, where the cost
// is a handful of FMAs and tensor cores do not apply).  A generic loop over d
// serves any other point dimension.
//
// Tile = H rows x W = 128*V columns.  Lane l of every warp owns columns
// col0 + 128k + 4l + e (k < V, e < 4), so one warp reads a row segment with
// coalesced 128-bit loads; warp w takes rows row0 + w, row0 + w + 8, ...
//   * row side: exact per-row max over the W columns (warp shuffle), then
//     sum_j 2^(logit - max); one (max, sum) partial per row and column block.
//   * column side: every lane keeps an exact running (max, sum) for each of
//     its 4V columns; rows come in chunks of four, so a column costs one
//     rescale per chunk plus one ex2 per entry.  The eight warps' columns
//     are merged in shared memory into one (max, sum) partial per column and
//     row block.  (An entry thus costs about 2.25 exponentials when both
//     sides are wanted, well inside the MUFU budget of an HBM-bound pass.)
// All logits are kept in log2 units (potentials are pre-multiplied by
// log2 e in FP64 before the hi/lo split).
#include "common.cuh"
#include "pass.h"
#include "kernels.h"

namespace pot {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = 8;
constexpr double kL2E = 1.4426950408889634;

template <int KIND>
__device__ __forceinline__ float load_pt(const void* base, int64_t idx) {
  if (KIND == COST_SQEUCLID_BF16) {
    unsigned short b = reinterpret_cast<const unsigned short*>(base)[idx];
    return __uint_as_float(((unsigned)b) << 16);
  } else if (KIND == COST_SQEUCLID_F16) {
    return __half2float(reinterpret_cast<const __half*>(base)[idx]);
  } else {
    return reinterpret_cast<const float*>(base)[idx];
  }
}

// DMAX > 0: the lane's point coordinates live in registers (d <= DMAX).
// DMAX == 0: generic loop over d (slow; any d).
template <int KIND, int V, int DMAX, bool VEC>
__global__ void __launch_bounds__(kThreads) pass_simt_kernel(PassDesc P, int H) {
  if (P.done && *P.done) return;
  constexpr int NC = 4 * V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col0 = (int64_t)blockIdx.x * (128 * V);
  const int64_t row0 = (int64_t)blockIdx.y * H;
  const bool use1 = P.sel && *P.sel;
  const double* arow = use1 ? P.arow1 : P.arow0;
  const double* bcol = use1 ? P.bcol1 : P.bcol0;
  const double* aoffp = use1 ? P.aoff1 : P.aoff0;
  const double aoff = (aoffp && (P.mode & (PASS_ROWS | PASS_COLS | PASS_OBJ))) ? *aoffp : 0.0;
  const bool want_rows = P.mode & PASS_ROWS, want_cols = P.mode & PASS_COLS;
  const bool want_obj = P.mode & PASS_OBJ, want_max = P.mode & PASS_MAXCOST;
  const bool need_pot = P.mode & (PASS_ROWS | PASS_COLS | PASS_OBJ);
  const float g2 = (float)(P.gC * kL2E);
  const bool sq = KIND != COST_DENSE_F32;

  __shared__ float sS[kWarps][NC * 32];
  __shared__ float sM[kWarps][NC * 32];
  __shared__ double sRed[kWarps];

  float bh[NC], bl[NC], colS[NC];
  float yv[DMAX > 0 ? NC * DMAX : 1];
  double qv[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const int k = q >> 2, e = q & 3;
    const int64_t j = col0 + 128 * k + 4 * lane + e;
    const bool ok = j < P.m;
    double b = POT_NEG_BIG;
    if (ok && need_pot) {
      b = bcol[j];
      if (sq) b -= P.gC * (double)P.yn[j];
    }
    HiLo h = split_hilo(ok ? b * kL2E : POT_NEG_BIG);
    bh[q] = h.hi; bl[q] = h.lo;
    colS[q] = 0.f;
    qv[q] = (want_obj && ok) ? P.q[j] : 0.0;
    if (DMAX > 0) {
#pragma unroll
      for (int t = 0; t < (DMAX > 0 ? DMAX : 1); ++t)
        yv[q * (DMAX > 0 ? DMAX : 1) + t] = (ok && t < P.d) ? load_pt<KIND>(P.Y, j * P.ldy + t) : 0.f;
    }
  }
  float colM[NC];                     // exact running column max (log2 units)
#pragma unroll
  for (int q = 0; q < NC; ++q) colM[q] = POT_NEG_BIGF;
  double objacc = 0.0;
  float maxc = 0.f;
  const double kap = want_obj ? *P.kappa : 0.0;

  const int64_t rend = (row0 + H < P.n) ? row0 + H : P.n;
  // rows of this warp: row0 + warp + 8 t; processed in chunks of R rows
  constexpr int R = 4;
  for (int64_t ib = row0 + warp; ib < rend; ib += (int64_t)kWarps * R) {
    float lg[R][NC];
    float cost[R][NC];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int64_t i = ib + (int64_t)kWarps * rr;
      const bool rowv = i < rend;
      double a = (need_pot && rowv) ? arow[i] + aoff : POT_NEG_BIG;
      if (sq && rowv) a -= P.gC * (double)P.xn[i];
      HiLo ah = split_hilo(rowv ? a * kL2E : POT_NEG_BIG);
      if (!need_pot && rowv) { ah.hi = 0.f; ah.lo = 0.f; }
      if (KIND == COST_DENSE_F32) {
        const float* crow = P.C + (rowv ? i : 0) * P.ldc;
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const int64_t j0 = col0 + 128 * k + 4 * lane;
          if (rowv && VEC && j0 + 3 < P.m) {
            float4 c4 = __ldg(reinterpret_cast<const float4*>(crow + j0));
            cost[rr][4 * k] = c4.x; cost[rr][4 * k + 1] = c4.y; cost[rr][4 * k + 2] = c4.z; cost[rr][4 * k + 3] = c4.w;
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) cost[rr][4 * k + e] = (rowv && j0 + e < P.m) ? __ldg(crow + j0 + e) : 0.f;
          }
        }
      } else {
        // dot products x_i . y_j (the logit uses them directly; the cost
        // |x|^2 + |y|^2 - 2 x.y is only formed for the objective / max)
#pragma unroll
        for (int q = 0; q < NC; ++q) cost[rr][q] = 0.f;
        if (rowv) {
          if (DMAX > 0) {
#pragma unroll
            for (int t = 0; t < (DMAX > 0 ? DMAX : 1); ++t) {
              if (t < P.d) {
                const float xt = load_pt<KIND>(P.X, i * P.ldx + t);
#pragma unroll
                for (int q = 0; q < NC; ++q) cost[rr][q] = fmaf(xt, yv[q * (DMAX > 0 ? DMAX : 1) + t], cost[rr][q]);
              }
            }
          } else {
            for (int t = 0; t < P.d; ++t) {
              const float xt = load_pt<KIND>(P.X, i * P.ldx + t);
#pragma unroll
              for (int q = 0; q < NC; ++q) {
                const int64_t j = col0 + 128 * (q >> 2) + 4 * lane + (q & 3);
                const float yt = j < P.m ? load_pt<KIND>(P.Y, j * P.ldy + t) : 0.f;
                cost[rr][q] = fmaf(xt, yt, cost[rr][q]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const float t0 = ah.hi + bh[q];
        float l = sq ? fmaf(2.f * g2, cost[rr][q], t0) : fmaf(-g2, cost[rr][q], t0);
        l += ah.lo + bl[q];
        if (!(t0 > -1.0e29f)) l = POT_NEG_BIGF;
        lg[rr][q] = l;
      }
    }

    if (want_obj || want_max) {
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int64_t i = ib + (int64_t)kWarps * rr;
        if (i >= rend) continue;
        const double pi = want_obj ? P.p[i] : 0.0;
        const float xn = sq ? P.xn[i] : 0.f;
        float rowacc = 0.f;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          const int64_t j = col0 + 128 * (q >> 2) + 4 * lane + (q & 3);
          if (j < P.m) {
            const float cst = sq ? fmaxf(xn + P.yn[j] - 2.f * cost[rr][q], 0.f) : cost[rr][q];
            maxc = fmaxf(maxc, cst);
            if (want_obj) {
              const float x = (lg[rr][q] > -1.0e29f ? ex2(lg[rr][q]) : 0.f) + (float)(kap * pi * qv[q]);
              rowacc = fmaf(cst, x, rowacc);
            }
          }
        }
        objacc += (double)rowacc;
      }
    }

    if (want_rows) {
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int64_t i = ib + (int64_t)kWarps * rr;
        float mx = POT_NEG_BIGF;
#pragma unroll
        for (int q = 0; q < NC; ++q) mx = fmaxf(mx, lg[rr][q]);
        const float m_i = warp_max(mx);
        float ssum = 0.f;
#pragma unroll
        for (int q = 0; q < NC; ++q) ssum += (lg[rr][q] > -1.0e29f) ? ex2(lg[rr][q] - m_i) : 0.f;
        ssum = warp_sum(ssum);
        if (lane == 0 && i < rend) P.row_part[(int64_t)blockIdx.x * P.n + i] = make_float2(m_i, ssum);
      }
    }
    if (want_cols) {
      // exact per-column log-sum-exp: one rescale per chunk, one ex2 per entry
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        float cmx = colM[q];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) cmx = fmaxf(cmx, lg[rr][q]);
        if (cmx > -1.0e29f) {
          if (cmx > colM[q]) {
            colS[q] = (colM[q] > -1.0e29f) ? colS[q] * ex2(colM[q] - cmx) : 0.f;
            colM[q] = cmx;
          }
#pragma unroll
          for (int rr = 0; rr < R; ++rr)
            if (lg[rr][q] > -1.0e29f) colS[q] += ex2(lg[rr][q] - cmx);
        }
      }
    }
  }

  if (want_cols) {
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      sS[warp][128 * (q >> 2) + 4 * lane + (q & 3)] = colS[q];
      sM[warp][128 * (q >> 2) + 4 * lane + (q & 3)] = colM[q];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NC * 32; t += kThreads) {
      const int64_t j = col0 + t;
      if (j >= P.m) continue;
      float Km = POT_NEG_BIGF;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) Km = fmaxf(Km, sM[w][t]);
      float S = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w)
        if (sM[w][t] > -1.0e29f) S = fmaf(sS[w][t], ex2(sM[w][t] - Km), S);
      P.col_part[(int64_t)blockIdx.y * P.m + j] = make_float2(Km, S);
    }
  }
  if (want_obj || want_max) {
    double v = want_obj ? objacc : (double)maxc;
    if (want_obj) v = warp_sum_d(v);
    else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    if (lane == 0) sRed[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = want_obj ? 0.0 : sRed[0];
      for (int w = 0; w < kWarps; ++w) acc = want_obj ? acc + sRed[w] : fmax(acc, sRed[w]);
      P.red_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
    }
  }
}

template <int KIND, int V, int DMAX>
void launch_v(const PassDesc& P, const SimtLayout& L, cudaStream_t st) {
  dim3 grid((unsigned)L.ncolblk, (unsigned)L.nrowblk);
  const bool vec = KIND == COST_DENSE_F32 && (P.ldc % 4 == 0) && ((uintptr_t)P.C % 16 == 0);
  if (vec) pass_simt_kernel<KIND, V, DMAX, true><<<grid, kThreads, 0, st>>>(P, L.H);
  else pass_simt_kernel<KIND, V, DMAX, false><<<grid, kThreads, 0, st>>>(P, L.H);
}

template <int KIND>
void launch_kind(const PassDesc& P, const SimtLayout& L, cudaStream_t st) {
  if (KIND == COST_DENSE_F32) {
    if (L.V == 1) launch_v<KIND, 1, 0>(P, L, st); else launch_v<KIND, 2, 0>(P, L, st);
  } else if (P.d <= 4) {
    if (L.V == 1) launch_v<KIND, 1, 4>(P, L, st); else launch_v<KIND, 2, 4>(P, L, st);
  } else {
    if (L.V == 1) launch_v<KIND, 1, 0>(P, L, st); else launch_v<KIND, 2, 0>(P, L, st);
  }
}

}  // namespace

SimtLayout simt_layout(int64_t n, int64_t m) {
  SimtLayout L;
  L.V = m > 256 ? 2 : 1;
  L.ncolblk = (m + 128 * L.V - 1) / (128 * L.V);
  int H = 128;
  while (H > 8 && L.ncolblk * ((n + H - 1) / H) < 1216) H >>= 1;
  L.H = H;
  L.nrowblk = (n + H - 1) / H;
  return L;
}

void launch_pass_simt(const PassDesc& P, const SimtLayout& L, cudaStream_t st) {
  switch (P.kind) {
    case COST_DENSE_F32: launch_kind<COST_DENSE_F32>(P, L, st); break;
    case COST_SQEUCLID_BF16: launch_kind<COST_SQEUCLID_BF16>(P, L, st); break;
    case COST_SQEUCLID_F16: launch_kind<COST_SQEUCLID_F16>(P, L, st); break;
    default: launch_kind<COST_SQEUCLID_F32>(P, L, st); break;
  }
}

// Squared norms of point rows (FP32 accumulation of exact products).
template <int KIND>
__global__ void sqnorm_kernel(const void* X, int64_t n, int d, int64_t ldx, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.f;
  for (int t = 0; t < d; ++t) {
    const float x = load_pt<KIND>(X, i * ldx + t);
    acc = fmaf(x, x, acc);
  }
  out[i] = acc;
}

void launch_sqnorm(int kind, const void* X, int64_t n, int d, int64_t ldx, float* out, cudaStream_t st) {
  const int b = 256;
  const unsigned g = (unsigned)((n + b - 1) / b);
  switch (kind) {
    case COST_SQEUCLID_BF16: sqnorm_kernel<COST_SQEUCLID_BF16><<<g, b, 0, st>>>(X, n, d, ldx, out); break;
    case COST_SQEUCLID_F16: sqnorm_kernel<COST_SQEUCLID_F16><<<g, b, 0, st>>>(X, n, d, ldx, out); break;
    default: sqnorm_kernel<COST_SQEUCLID_F32><<<g, b, 0, st>>>(X, n, d, ldx, out); break;
  }
}

}  // namespace pot
