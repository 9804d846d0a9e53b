// The CUDA-core tile body of the passes (one H x 128 V tile of the Gibbs
// matrix: row (max, sum) partials by a four-row transposing butterfly, exact
// running column (max, sum), objective / max-cost partials), shared by the
// single-instance passes (pass_simt.cu) and the fused batched sweep
// (batched.cu).  Device code only; each translation unit that includes it
// gets its own copy.
#pragma once
#include "common.cuh"
#include "pass.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace pot {
namespace simt {

using tcx::pk2; using tcx::upk2; using tcx::add2; using tcx::fma2; using tcx::max3f;

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

// v[0..3] (one value per row) reduced over the 32 lanes; lane 8r ends with
// row r's total in v[0].  IS_MAX selects max, else sum.
template <bool IS_MAX>
__device__ __forceinline__ void rows4_reduce(float (&v)[4], int lane) {
  const bool up16 = lane & 16, up8 = lane & 8;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = up16 ? v[k] : v[k + 2];
    const float keep = up16 ? v[k + 2] : v[k];
    const float got = __shfl_xor_sync(0xffffffffu, send, 16);
    v[k] = IS_MAX ? fmaxf(keep, got) : keep + got;
  }
  {
    const float send = up8 ? v[0] : v[1];
    const float keep = up8 ? v[1] : v[0];
    const float got = __shfl_xor_sync(0xffffffffu, send, 8);
    v[0] = IS_MAX ? fmaxf(keep, got) : keep + got;
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    const float got = __shfl_xor_sync(0xffffffffu, v[0], o);
    v[0] = IS_MAX ? fmaxf(v[0], got) : v[0] + got;
  }
}

// DMAX > 0: the lane's point coordinates live in registers (d <= DMAX).
// DMAX == 0: generic loop over d (slow; any d).
// One H x 128V tile (column block cb, row block rb) of the pass.  Partials
// go to row_part[cb * rstride + i] and col_part[rb * cstride + j]; objective /
// max-cost partials to red_part[red_idx].
// MT: 0 = the pass mode is read at run time (any mode, including the
// objective and max-cost passes); 1 / 2 / 3 = rows + columns / rows /
// columns fixed at compile time, which drops the other modes' registers.
// The per-pass terms (rowA, colA) are read through L2: the single-cluster
// loop writes them in the same kernel, on another SM, before a barrier.
template <int KIND, int V, int DMAX, bool VEC, int MT = 0>
__device__ __forceinline__ void simt_tile(const PassDesc& P, int H, int64_t cb, int64_t rb, int64_t rstride,
                                          int64_t cstride, int64_t red_idx) {
  constexpr int NC = 4 * V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col0 = cb * (128 * V);
  const int64_t row0 = rb * H;
const bool want_rows = MT == 0 ? (P.mode & PASS_ROWS) != 0 : (MT == 1 || MT == 2);
  const bool want_cols = MT == 0 ? (P.mode & PASS_COLS) != 0 : (MT == 1 || MT == 3);
  const bool want_obj = MT == 0 ? (P.mode & PASS_OBJ) != 0 : false;
  const bool want_max = MT == 0 ? (P.mode & PASS_MAXCOST) != 0 : false;
  const bool need_pot = MT == 0 ? (P.mode & (PASS_ROWS | PASS_COLS | PASS_OBJ)) != 0 : true;
  const float g2 = (float)(P.gC * kL2E);
  const bool sq = KIND != COST_DENSE_F32;

  __shared__ float sS[kWarps][NC * 32];
  __shared__ float sM[kWarps][NC * 32];
  __shared__ double sRed[kWarps];

  float bh[NC], bl[NC], colS[NC];
  float yv[DMAX > 0 ? NC * DMAX : 1];
  float qv[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const int k = q >> 2, e = q & 3;
    const int64_t j = col0 + 128 * k + 4 * lane + e;
    const bool ok = j < P.m;
    const float2 cb2 = (ok && need_pot) ? __ldcg(P.colA + j) : make_float2(POT_NEG_BIGF, 0.f);
    bh[q] = cb2.x; bl[q] = cb2.y;
    colS[q] = 0.f;
    qv[q] = (want_obj && ok) ? P.colB[j].y : 0.f;
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
      HiLo ah;
      if (rowv && need_pot) {
        const float4 ra = __ldcg(P.rowA + i);
        ah.hi = ra.x; ah.lo = ra.y;
      } else {
        ah.hi = rowv ? 0.f : POT_NEG_BIGF; ah.lo = 0.f;
      }
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
        const float kpi = want_obj ? (float)(kap * (double)P.rowA[i].w) : 0.f;
        const float xn = sq ? P.xn[i] : 0.f;
        float rowacc = 0.f;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          const int64_t j = col0 + 128 * (q >> 2) + 4 * lane + (q & 3);
          if (j < P.m) {
            const float cst = sq ? nanmaxf(xn + P.yn[j] - 2.f * cost[rr][q], 0.f) : cost[rr][q];
            maxc = nanmaxf(maxc, cst);
            if (want_obj) {
              const float x = (lg[rr][q] > -1.0e29f ? ex2(lg[rr][q]) : 0.f) + kpi * qv[q];
              rowacc = fmaf(cst, x, rowacc);
            }
          }
        }
        objacc += (double)rowacc;
      }
    }

    // Entries of log 0 carry logits near -1e30; shifted by a real maximum
    // their ex2 is 0, so the sums need no per-entry test; a row or column
    // whose entries are all log 0 is caught by its maximum.  Adjacent columns
    // q, q + 1 of a lane go through the shifts and sums as FP32x2 pairs.
    if (want_rows) {
      // the chunk's four rows reduced together by the transposing butterfly
      float mx[R], sm[R], rm[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        mx[rr] = POT_NEG_BIGF;
#pragma unroll
        for (int q = 0; q < NC; ++q) mx[rr] = fmaxf(mx[rr], lg[rr][q]);
      }
      rows4_reduce<true>(mx, lane);                 // lane 8r: row r's max in mx[0]
#pragma unroll
      for (int rr = 0; rr < R; ++rr) rm[rr] = __shfl_sync(0xffffffffu, mx[0], 8 * rr);
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const unsigned long long NM = pk2(-rm[rr], -rm[rr]);
        unsigned long long sp = 0ull;               // packed partial sums; bits 0 = 0.0f
#pragma unroll
        for (int q = 0; q < NC; q += 2) {
          float a, b;
          upk2(add2(pk2(lg[rr][q], lg[rr][q + 1]), NM), a, b);
          sp = add2(sp, pk2(ex2(a), ex2(b)));
        }
        float s0, s1;
        upk2(sp, s0, s1);
        sm[rr] = s0 + s1;
      }
      rows4_reduce<false>(sm, lane);                // lane 8r: row r's sum in sm[0]
      if ((lane & 7) == 0) {
        const int64_t i = ib + (int64_t)kWarps * (lane >> 3);
        if (i < rend) P.row_part[cb * rstride + i] = make_float2(mx[0], mx[0] > -1.0e29f ? sm[0] : 0.f);
      }
    }
    if (want_cols) {
      // exact per-column log-sum-exp: the running (max, sum) rescaled once per
      // chunk (by ex2(old max - new max): 0 from log 0, 1 when unchanged)
#pragma unroll
      for (int q = 0; q < NC; q += 2) {
        const float nm0 = max3f(max3f(lg[0][q], lg[1][q], lg[2][q]), lg[3][q], colM[q]);
        const float nm1 = max3f(max3f(lg[0][q + 1], lg[1][q + 1], lg[2][q + 1]), lg[3][q + 1], colM[q + 1]);
        const unsigned long long NMp = pk2(-nm0, -nm1);
        unsigned long long e[R];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
          float a, b;
          upk2(add2(pk2(lg[rr][q], lg[rr][q + 1]), NMp), a, b);
          e[rr] = pk2(ex2(a), ex2(b));
        }
        const unsigned long long sum = add2(add2(e[0], e[1]), add2(e[2], e[3]));
        float n0, n1;
        upk2(fma2(pk2(colS[q], colS[q + 1]), pk2(ex2(colM[q] - nm0), ex2(colM[q + 1] - nm1)), sum), n0, n1);
        if (nm0 > -1.0e29f) { colS[q] = n0; colM[q] = nm0; }
        if (nm1 > -1.0e29f) { colS[q + 1] = n1; colM[q + 1] = nm1; }
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
      P.col_part[rb * cstride + j] = make_float2(Km, S);
    }
  }
  if (want_obj || want_max) {
    double v = want_obj ? objacc : (double)maxc;
    if (want_obj) v = warp_sum_d(v);
    else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    if (lane == 0) sRed[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = want_obj ? 0.0 : sRed[0];
      for (int w = 0; w < kWarps; ++w) acc = want_obj ? acc + sRed[w] : nanmax(acc, sRed[w]);
      P.red_part[red_idx] = acc;
    }
  }
}

}  // namespace simt
}  // namespace pot
