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
//   * row side: exact per-row max over the W columns, then
//     sum_j 2^(logit - max), the four rows of a chunk reduced over the warp
//     together by a transposing butterfly; one (max, sum) partial per row and
//     column block.
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
#include "tc_common.cuh"
#include "simt_tile.cuh"

namespace pot {

using namespace simt;

namespace {

// Per-pass row / column terms of the logit, formed once per pass in FP64 and
// handed to the pass kernels as FP32 (hi, lo) pairs in log2 units:
//   rowA[i] = (hi, lo of (a_i + aoff - gC |x_i|^2) log2 e, |x_i|^2, p_i)
//   colA[j] = (hi, lo of (b_j - gC |y_j|^2) log2 e),  colB[j] = (|y_j|^2, q_j)
// (no norm terms for a dense cost).  Entries past n / m (padding) are log 0.
// In max-cost mode the tensor-core pass reads the norms through the same slots.
__global__ void prep_kernel(PassDesc P, int64_t n_pad, int64_t m_pad, int release_first) {
  // release_first: the pass that follows is scheduled while this kernel still
  // waits for the loop kernel before it.  Not before the persistent dense
  // pass, whose fixed share of the work per CTA wants every CTA placed at once
  // (CTAs that found an SM still held by the loop kernel would start late).
  if (release_first) pdl_release();
  pdl_wait();
  if (!release_first) pdl_release();
  if (pass_off(P)) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool use1 = P.sel && *P.sel;
  const double* arow = use1 ? P.arow1 : P.arow0;
  const double* bcol = use1 ? P.bcol1 : P.bcol0;
  const double* aoffp = use1 ? P.aoff1 : P.aoff0;
  const bool maxmode = P.mode & PASS_MAXCOST;
  const bool sq = P.kind != COST_DENSE_F32;
  if (t < n_pad) {
    float4 o = make_float4(POT_NEG_BIGF, 0.f, 0.f, 0.f);
    if (t < P.n) {
      const float xn = sq ? P.xn[t] : 0.f;
      if (maxmode) {
        o = make_float4(xn, 0.f, xn, 0.f);
      } else {
        const double a = (arow[t] + (aoffp ? *aoffp : 0.0) - P.gC * (double)xn) * kL2E;
        HiLo hl = split_hilo(a);
        o = make_float4(hl.hi, hl.lo, xn, (P.mode & PASS_OBJ) ? (float)P.p[t] : 0.f);
      }
    }
    P.rowA[t] = o;
  } else if (t < n_pad + m_pad) {
    const int64_t j = t - n_pad;
    float2 A = make_float2(POT_NEG_BIGF, 0.f), Bv = make_float2(0.f, 0.f);
    if (j < P.m) {
      const float yn = sq ? P.yn[j] : 0.f;
      if (maxmode) {
        A = make_float2(yn, 0.f);
      } else {
        const double b = ((double)bcol[j] - P.gC * (double)yn) * kL2E;
        HiLo hl = split_hilo(b);
        A = make_float2(hl.hi, hl.lo);
        Bv = make_float2(yn, (P.mode & PASS_OBJ) ? (float)P.q[j] : 0.f);
      }
    }
    P.colA[j] = A;
    P.colB[j] = Bv;
  }
}

// ------------------------------------------------------------------------
// Dense FP32 cost, rows / columns / both: the HBM-bound hot pass.
// Tile = H rows x 256 columns, 8 warps; lane l owns columns 4l..4l+3 and
// 128+4l..128+4l+3 (two coalesced float4 per row); warp w takes chunks of 4
// consecutive rows (row0 + 32k + 4w + r).  The next chunk's cost is loaded
// while the current one is reduced (register double buffer).
//   rows: the 4 rows' maxima and sums are reduced over the warp together by a
//         transposing butterfly (10 shuffles for 4 rows instead of 40);
//   columns: exact running (max, sum) per column, one rescale per chunk.
// Requires m % 4 == 0, ldc % 4 == 0 and a 16-byte aligned C.

using tcx::pk2; using tcx::upk2; using tcx::add2; using tcx::fma2; using tcx::max3f;

__host__ __device__ __forceinline__ int64_t dense_owner(int64_t u, int64_t G, int64_t U) { return ((u + 1) * G - 1) / U; }

// Per-warp shared-memory ring of cost chunks filled with cp.async (16 bytes
// per lane and copy); kDStages chunks of 4 rows x 256 columns per warp, so
// kDStages - 1 loads are in flight while one chunk is reduced.  Each lane
// reads back exactly the 16-byte slots it copied.  Beside it, the chunk's four
// row terms (hi, lo), copied by lanes 0..3 in the same group and read by the
// whole warp, so the warp synchronises after the wait and before a stage is
// refilled.  (Loaded from global memory at their use, the row terms were the
// pass's main long-scoreboard stall.)  2 CTAs per SM: 2 x (16 KB static +
// 96.75 KB ring + 1 KB reserved) fits the 228 KB of an SM.
constexpr int kDStages = 3;
constexpr size_t kDenseCostRingBytes = (size_t)kWarps * kDStages * 4 * 256 * sizeof(float);
constexpr size_t kDenseRingBytes = kDenseCostRingBytes + (size_t)kWarps * kDStages * 4 * sizeof(float2);

__device__ __forceinline__ void cp_async16s(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_ring() { asm volatile("cp.async.wait_group %0;" ::"n"(kDStages - 1) : "memory"); }

template <int MODE>   // 0: rows + columns, 1: rows, 2: columns
__global__ void __launch_bounds__(kThreads, 2) dense_pass_kernel(PassDesc P, SimtLayout DL) {
  // no early release: the loop kernel that follows spreads its FP64 work one block
  // per SM, which holds only for blocks placed on an idle GPU, not on the few
  // SMs a draining pass frees first
  pdl_wait();
  if (pass_off(P)) return;
  constexpr bool ROWS = MODE != 2, COLS = MODE != 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ float sS[kWarps][256];
  __shared__ float sM[kWarps][256];
  extern __shared__ float4 dring[];                      // [kWarps][kDStages][4 rows][64], then row terms
  float4* ring = dring + (size_t)warp * kDStages * 4 * 64;
  float2* aring = reinterpret_cast<float2*>(dring + (size_t)kWarps * kDStages * 4 * 64) + warp * kDStages * 4;
  const float g2 = (float)(P.gC * kL2E);
  const unsigned long long NG = pk2(-g2, -g2);
  // persistent: CTA c owns units [c U / G, (c+1) U / G) of the panel-major
  // list of (256-column panel, 32-row unit); a run of units of one panel is a
  // segment with its own column partial slot
  const int64_t c = blockIdx.x;
  const int64_t u_end = (c + 1) * DL.U / DL.G;
  for (int64_t u = c * DL.U / DL.G; u < u_end;) {
  const int64_t panel = u / DL.nrg;
  const int64_t seg_end = ((panel + 1) * DL.nrg < u_end) ? (panel + 1) * DL.nrg : u_end;
  const int64_t slot = c - dense_owner(panel * DL.nrg, DL.G, DL.U);
  const int64_t col0 = panel * 256;
  const int64_t row0 = (u - panel * DL.nrg) * 32;
  const int64_t rlim = (seg_end - panel * DL.nrg) * 32;
  const int64_t rend = (rlim < P.n) ? rlim : P.n;
  u = seg_end;

  // column terms (pairs) and validity of the two float4 groups
  unsigned long long BH[4], BL[4];
  bool gv[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int64_t j0 = col0 + 128 * k + 4 * lane;
    gv[k] = j0 < P.m;
    float2 c0 = make_float2(POT_NEG_BIGF, 0.f), c1 = c0, c2 = c0, c3 = c0;
    if (gv[k]) { c0 = P.colA[j0]; c1 = P.colA[j0 + 1]; c2 = P.colA[j0 + 2]; c3 = P.colA[j0 + 3]; }
    BH[2 * k] = pk2(c0.x, c1.x); BH[2 * k + 1] = pk2(c2.x, c3.x);
    BL[2 * k] = pk2(c0.y, c1.y); BL[2 * k + 1] = pk2(c2.y, c3.y);
  }
  float cM[8], cS[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) { cM[q] = POT_NEG_BIGF; cS[q] = 0.f; }

  // chunk ci of this warp: rows row0 + 4 warp + 32 ci + r, in ring stage ci % kDStages
  // one running row pointer and 32-bit shared addresses per chunk
  const float* const cbase = P.C + col0 + 4 * lane;
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring + lane);
  auto issue = [&](int64_t b, int st) {
    const float* src = cbase + b * P.ldc;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const bool rv = b + r < rend;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int slot = (st * 4 + r) * 64 + k * 32;          // in float4, before the lane
        if (rv && gv[k]) cp_async16s(ring_s + (uint32_t)slot * 16u, src + 128 * k);
        else ring[slot + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      src += P.ldc;
    }
    if (lane < 4) {                                      // the row terms (hi, lo) of the chunk
      float2* dst = aring + st * 4 + lane;
      if (b + lane < rend) cp_async8(dst, P.rowA + b + lane);
      else *dst = make_float2(POT_NEG_BIGF, 0.f);
    }
    cp_commit();
  };
  const int64_t first = row0 + 4 * warp;
  const int64_t nchunks = first < rend ? (rend - first + 31) / 32 : 0;
#pragma unroll
  for (int st = 0; st < kDStages - 1; ++st) {
    if (st < nchunks) issue(first + 32 * st, st);
    else cp_commit();
  }
  for (int64_t ci = 0; ci < nchunks; ++ci) {
    const int64_t base = first + 32 * ci;
    const int64_t nci = ci + kDStages - 1;
    __syncwarp();                                        // every lane is done with the stage refilled now
    if (nci < nchunks) issue(first + 32 * nci, (int)(nci % kDStages));
    else cp_commit();
    cp_wait_ring();                                      // chunk ci has landed
    __syncwarp();                                        // and its row terms, copied by lanes 0..3
    float4 cur[4][2];
    {
      const int st = (int)(ci % kDStages);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 2; ++k) cur[r][k] = ring[(st * 4 + r) * 64 + k * 32 + lane];
    }
    // logits of the 4 x 8 entries
    float lg[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float2 ra = aring[(int)(ci % kDStages) * 4 + r];
      const unsigned long long AH = pk2(ra.x, ra.x), AL = pk2(ra.y, ra.y);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float4 c = cur[r][k];
        const unsigned long long t0 = add2(fma2(NG, pk2(c.x, c.y), add2(AH, BH[2 * k])), add2(AL, BL[2 * k]));
        const unsigned long long t1 = add2(fma2(NG, pk2(c.z, c.w), add2(AH, BH[2 * k + 1])), add2(AL, BL[2 * k + 1]));
        upk2(t0, lg[r][4 * k], lg[r][4 * k + 1]);
        upk2(t1, lg[r][4 * k + 2], lg[r][4 * k + 3]);
      }
    }
    if (ROWS) {
      float mx[4], sm[4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        mx[r] = fmaxf(max3f(lg[r][0], lg[r][1], lg[r][2]), max3f(max3f(lg[r][3], lg[r][4], lg[r][5]), lg[r][6], lg[r][7]));
      rows4_reduce<true>(mx, lane);
      float rm[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) rm[r] = __shfl_sync(0xffffffffu, mx[0], 8 * r);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const bool ok = rm[r] > -1.0e29f;
        const unsigned long long NM = pk2(ok ? -rm[r] : 0.f, ok ? -rm[r] : 0.f);
        unsigned long long sp = 0ull;                    // packed (even, odd) partial sums; bits 0 = 0.0f
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          float a, b;
          upk2(add2(pk2(lg[r][2 * p], lg[r][2 * p + 1]), NM), a, b);
          sp = add2(sp, pk2(ex2(a), ex2(b)));
        }
        float s0, s1;
        upk2(sp, s0, s1);
        sm[r] = s0 + s1;
      }
      rows4_reduce<false>(sm, lane);
      if ((lane & 7) == 0) {
        const int r = lane >> 3;
        const int64_t i = base + r;
        if (i < rend) P.row_part[panel * P.n + i] = make_float2(rm[r], rm[r] > -1.0e29f ? sm[0] : 0.f);
      }
    }
    if (COLS) {
      // columns q, q + 1 of the lane as FP32x2 pairs (as the logits were
      // formed): shift, sum over the chunk's 4 rows, rescale of the running sum.
      // A running max of log 0 (-big) rescales by ex2(-huge) = 0; a column whose
      // entries are all log 0 keeps its state (ok).
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int q0 = 2 * p, q1 = 2 * p + 1;
        const float nm0 = max3f(max3f(lg[0][q0], lg[1][q0], lg[2][q0]), lg[3][q0], cM[q0]);
        const float nm1 = max3f(max3f(lg[0][q1], lg[1][q1], lg[2][q1]), lg[3][q1], cM[q1]);
        const unsigned long long NMp = pk2(-nm0, -nm1);
        unsigned long long e[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float a, b;
          upk2(add2(pk2(lg[r][q0], lg[r][q1]), NMp), a, b);
          e[r] = pk2(ex2(a), ex2(b));
        }
        const unsigned long long sum = add2(add2(e[0], e[1]), add2(e[2], e[3]));
        float n0, n1;
        upk2(fma2(pk2(cS[q0], cS[q1]), pk2(ex2(cM[q0] - nm0), ex2(cM[q1] - nm1)), sum), n0, n1);
        if (nm0 > -1.0e29f) { cS[q0] = n0; cM[q0] = nm0; }
        if (nm1 > -1.0e29f) { cS[q1] = n1; cM[q1] = nm1; }
      }
    }
  }
  if (COLS) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = 128 * (q >> 2) + 4 * lane + (q & 3);
      sS[warp][c] = cS[q];
      sM[warp][c] = cM[q];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += kThreads) {
      const int64_t j = col0 + t;
      if (j >= P.m) continue;
      float Km = POT_NEG_BIGF;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) Km = fmaxf(Km, sM[w][t]);
      float S = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w)
        if (sM[w][t] > -1.0e29f) S = fmaf(sS[w][t], ex2(sM[w][t] - Km), S);
      P.col_part[slot * P.m + j] = make_float2(Km, S);
      // the panel's last segment marks the slots no segment of it writes empty
      if (seg_end == (panel + 1) * DL.nrg)
        for (int64_t e = slot + 1; e < DL.nslots; ++e) P.col_part[e * P.m + j] = make_float2(POT_NEG_BIGF, 0.f);
    }
    __syncthreads();            // shared memory is reused by the next segment
  }
  }
}

template <int KIND, int V, int DMAX, bool VEC>
__global__ void __launch_bounds__(kThreads) pass_simt_kernel(PassDesc P, int H) {
  // no early release: the loop kernel that follows spreads its FP64 work one block
  // per SM, which holds only for blocks placed on an idle GPU, not on the few
  // SMs a draining pass frees first
  pdl_wait();
  if (pass_off(P)) return;
  simt_tile<KIND, V, DMAX, VEC>(P, H, blockIdx.x, blockIdx.y, P.n, P.m, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
}

template <int KIND, int V, int DMAX>
void launch_v(const PassDesc& P, const SimtLayout& L, cudaStream_t st) {
  dim3 grid((unsigned)L.ncolblk, (unsigned)L.nrowblk);
  const bool vec = KIND == COST_DENSE_F32 && (P.ldc % 4 == 0) && ((uintptr_t)P.C % 16 == 0);
  launch_k(vec ? pass_simt_kernel<KIND, V, DMAX, true> : pass_simt_kernel<KIND, V, DMAX, false>, grid, dim3(kThreads), 0,
           st, P, L.H);
}

template <int KIND>
void launch_kind(const PassDesc& P, const SimtLayout& L, cudaStream_t st) {
  const bool hot = (P.mode & (PASS_ROWS | PASS_COLS)) && !(P.mode & (PASS_OBJ | PASS_MAXCOST));
  if (KIND == COST_DENSE_F32 && hot && L.dense_fast) {
    const unsigned grid = (unsigned)L.G;
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(dense_pass_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseRingBytes);
      cudaFuncSetAttribute(dense_pass_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseRingBytes);
      cudaFuncSetAttribute(dense_pass_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseRingBytes);
      cudaFuncSetAttribute(dense_pass_kernel<0>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(dense_pass_kernel<1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(dense_pass_kernel<2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      attr_set = true;
    }
    const int mode = ((P.mode & PASS_ROWS) && (P.mode & PASS_COLS)) ? 0 : ((P.mode & PASS_ROWS) ? 1 : 2);
    launch_k(mode == 0 ? dense_pass_kernel<0> : (mode == 1 ? dense_pass_kernel<1> : dense_pass_kernel<2>), dim3(grid),
             dim3(kThreads), kDenseRingBytes, st, P, L);
    return;
  }
  if (KIND == COST_DENSE_F32) {
    if (L.V == 1) launch_v<KIND, 1, 0>(P, L, st); else launch_v<KIND, 2, 0>(P, L, st);
  } else if (P.d <= 4) {
    if (L.V == 1) launch_v<KIND, 1, 4>(P, L, st); else launch_v<KIND, 2, 4>(P, L, st);
  } else {
    if (L.V == 1) launch_v<KIND, 1, 0>(P, L, st); else launch_v<KIND, 2, 0>(P, L, st);
  }
}

// Batched pass: one CTA per tile of the work list (H rows x 128 V columns);
// the tile's instance supplies sizes, points, offsets and its scalar
// potentials.
template <int KIND, int V, int MT>
__global__ void __launch_bounds__(kThreads, MT == 0 ? 1 : (V == 1 ? 3 : 2)) pass_simt_batched_kernel(BatchPass B) {
  const BTile tl = B.tiles[blockIdx.x];
  BInst* I = B.inst + tl.inst;
  if (B.check_done && I->done) return;
  PassDesc P{};
  P.n = I->n; P.m = I->m; P.kind = KIND;
  P.X = I->X; P.Y = I->Y; P.d = I->d; P.ldx = I->ldx; P.ldy = I->ldy;
  P.xn = B.xn + I->row0; P.yn = B.yn + I->col0;
  P.gC = I->gC;
  const char* base = reinterpret_cast<const char*>(I);
  P.arow0 = B.arow0 ? B.arow0 + I->row0 : nullptr;
  P.bcol0 = B.bcol0 ? B.bcol0 + I->col0 : nullptr;
  P.aoff0 = B.aoff0 >= 0 ? reinterpret_cast<const double*>(base + B.aoff0) : nullptr;
  P.arow1 = B.arow1 ? B.arow1 + I->row0 : nullptr;
  P.bcol1 = B.bcol1 ? B.bcol1 + I->col0 : nullptr;
  P.aoff1 = B.aoff1 >= 0 ? reinterpret_cast<const double*>(base + B.aoff1) : nullptr;
  P.sel = B.use_sel ? &I->take_hat : nullptr;
  P.mode = B.mode;
  P.row_part = B.row_part + I->row0;
  P.col_part = B.col_part + I->col0;
  P.red_part = B.red_part;
  P.p = B.p ? B.p + I->row0 : nullptr;
  P.q = B.q ? B.q + I->col0 : nullptr;
  P.kappa = &I->kappa;
  P.rowA = B.rowA + I->row0;
  P.colA = B.colA + I->col0;
  P.colB = B.colB + I->col0;
  simt_tile<KIND, V, 4, false, MT>(P, B.H, tl.cb, tl.rb, B.Ntot, B.Mtot, blockIdx.x);
}

// Batched counterpart of prep_kernel: one CTA per instance.
__global__ void prep_batched_kernel(BatchPass B) {
  BInst* I = B.inst + blockIdx.x;
  if (B.check_done && I->done) return;
  const bool use1 = B.use_sel && I->take_hat;
  const double* arow = use1 ? B.arow1 : B.arow0;
  const double* bcol = use1 ? B.bcol1 : B.bcol0;
  const int aoffb = use1 ? B.aoff1 : B.aoff0;
  const double aoff = aoffb >= 0 ? *reinterpret_cast<const double*>(reinterpret_cast<const char*>(I) + aoffb) : 0.0;
  const bool obj = B.mode & PASS_OBJ;
  for (int64_t i = threadIdx.x; i < I->n; i += blockDim.x) {
    const int64_t g = I->row0 + i;
    const float xn = B.xn[g];
    HiLo hl = split_hilo((arow[g] + aoff - I->gC * (double)xn) * kL2E);
    B.rowA[g] = make_float4(hl.hi, hl.lo, xn, obj ? (float)B.p[g] : 0.f);
  }
  for (int64_t j = threadIdx.x; j < I->m; j += blockDim.x) {
    const int64_t g = I->col0 + j;
    const float yn = B.yn[g];
    HiLo hl = split_hilo((bcol[g] - I->gC * (double)yn) * kL2E);
    B.colA[g] = make_float2(hl.hi, hl.lo);
    B.colB[g] = make_float2(yn, obj ? (float)B.q[g] : 0.f);
  }
}

}  // namespace

void launch_prep_batched(const BatchPass& B, cudaStream_t st) {
  prep_batched_kernel<<<(unsigned)B.count, 512, 0, st>>>(B);
}

template <int V, int MT>
void launch_batched_vm(const BatchPass& B, cudaStream_t st) {
  const unsigned g = (unsigned)B.ntiles;
  switch (B.kind) {
    case COST_SQEUCLID_BF16: pass_simt_batched_kernel<COST_SQEUCLID_BF16, V, MT><<<g, kThreads, 0, st>>>(B); break;
    case COST_SQEUCLID_F16: pass_simt_batched_kernel<COST_SQEUCLID_F16, V, MT><<<g, kThreads, 0, st>>>(B); break;
    default: pass_simt_batched_kernel<COST_SQEUCLID_F32, V, MT><<<g, kThreads, 0, st>>>(B); break;
  }
}

template <int V>
void launch_batched_v(const BatchPass& B, cudaStream_t st) {
  if (B.mode == (PASS_ROWS | PASS_COLS)) launch_batched_vm<V, 1>(B, st);
  else if (B.mode == PASS_ROWS) launch_batched_vm<V, 2>(B, st);
  else if (B.mode == PASS_COLS) launch_batched_vm<V, 3>(B, st);
  else launch_batched_vm<V, 0>(B, st);
}

void launch_pass_simt_batched(const BatchPass& B, cudaStream_t st) {
  if (B.W == 128) launch_batched_v<1>(B, st);
  else launch_batched_v<2>(B, st);
}

SimtLayout simt_layout(int64_t n, int64_t m) {
  // About four CTAs per SM in total, each streaming as many rows as that
  // leaves (a multiple of 32: eight warps x chunks of four rows), so the
  // per-CTA set-up and the column partials are amortised over many rows.
  SimtLayout L;
  L.V = m > 256 ? 2 : 1;
  L.ncolblk = (m + 128 * L.V - 1) / (128 * L.V);
  const int64_t target = 4 * 152;
  int64_t groups = target / L.ncolblk;
  if (groups < 1) groups = 1;
  int64_t H = (n + groups - 1) / groups;
  H = ((H + 31) / 32) * 32;
  if (H < 32) H = 32;
  L.H = (int)H;
  L.nrowblk = (n + H - 1) / H;
  L.dense_fast = 0;
  L.G = L.nrg = L.U = 0;
  L.nslots = 0;
  return L;
}

void simt_dense_layout(SimtLayout& L, int64_t n, int64_t m, int num_sms) {
  L.dense_fast = (L.V == 2) ? 1 : 0;
  if (!L.dense_fast) return;
  L.nrg = (n + 31) / 32;
  L.U = L.ncolblk * L.nrg;
  L.G = 2 * (int64_t)num_sms;
  if (L.G > L.U) L.G = L.U;
  int64_t slots = 1;
  for (int64_t p = 0; p < L.ncolblk; ++p) {
    const int64_t a = dense_owner(p * L.nrg, L.G, L.U), b = dense_owner((p + 1) * L.nrg - 1, L.G, L.U);
    if (b - a + 1 > slots) slots = b - a + 1;
  }
  L.nslots = slots;
}

void launch_prep(const PassDesc& P, int64_t n_pad, int64_t m_pad, cudaStream_t st) {
  const int64_t tot = n_pad + m_pad;
  const bool dense_next = P.kind == COST_DENSE_F32 && (P.mode & (PASS_ROWS | PASS_COLS)) &&
                          !(P.mode & (PASS_OBJ | PASS_MAXCOST));
  launch_k(prep_kernel, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st, P, n_pad, m_pad, dense_next ? 0 : 1);
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
