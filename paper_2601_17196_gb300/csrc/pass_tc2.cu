// tcgen05 on-the-fly squared-Euclidean pass for the solver's hot loop
// (BF16 points, d = 64 or 128; rows, columns or both).
//
// Differences from the general version in pass_tc.cu, all aimed at the
// epilogue, which bounds the pass (per cost entry: one ex2 and a handful of
// FP32 operations, against 2 d tensor FLOP):
//  * persistent CTAs, one per SM; CTA c owns the contiguous range
//    [c T / G, (c+1) T / G) of the T = ceil(n/256) x ceil(m/96) tiles taken
//    in row-block-major order, so work is balanced to one tile;
//  * 256-row tiles: two M = 128 MMAs (two TMEM accumulators) share each
//    Y tile, and every epilogue thread owns one row of each accumulator, so
//    the column reduction handles two rows per shuffle;
//  * 12 epilogue warps (4 TMEM lane quadrants x 3 groups of 32 columns of a
//    96-column tile); with the TMA and MMA warps that is 14 warps, at most 4
//    on each SM sub-partition, which leaves 128 registers per thread;
//  * the per-column terms of each tile are staged in shared memory by the TMA
//    warp behind their own mbarrier ring;
//  * packed FP32x2 arithmetic (add/mul/fma.rn.f32x2), 3-input max and
//    independent partial sums.
// Row partials: one (max, sum) per row for every CTA that touches its row
// block (slot = CTA - first CTA of the block, at most a few); column partials:
// one (shift, sum) per column and 256-row block.
#include "common.cuh"
#include "pass.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace pot {

namespace {

using namespace tcx;

constexpr int NGRP = 3;                           // groups of 32 columns per tile
constexpr int BM2 = 256, BN2 = 32 * NGRP;
constexpr int NEPI = 4 * NGRP;                    // epilogue warps (4 TMEM lane quadrants per group)
constexpr int NTHREADS2 = 64 + 32 * NEPI;         // + TMA warp + MMA warp
constexpr uint32_t TMEM2_COLS = 512;              // 2 buffers x 2 accumulators, each at a 128-column boundary
constexpr int NCA = 8;                            // column-term ring depth
constexpr int kMaxStages = 8;                     // Y ring depth bound (barrier slots)
constexpr int kBarSlots = 2 + 2 * kMaxStages + 4 + 2 * NCA + 1;
constexpr double kL2E2 = 1.4426950408889634;

enum { V_RC = 0, V_R = 1, V_C = 2 };

struct Tc2Smem {
  uint32_t a_off, b_off, b_stage, ca_off, cs_off, cm_off, rb_off, bar_off, misc_off, total;
  int nst;
};

__host__ __device__ inline Tc2Smem tc2_smem(int d) {
  Tc2Smem L;
  const uint32_t kb = (uint32_t)(d / 64);
  L.nst = (d <= 64) ? 4 : 3;
  L.a_off = 0;                                   // [kb][half][128 rows][128 B]
  L.b_off = kb * 2 * 128 * 128;
  L.b_stage = kb * BN2 * 128;                    // [kb][128 rows][128 B]
  uint32_t o = L.b_off + (uint32_t)L.nst * L.b_stage;
  L.ca_off = o; o += NCA * (BN2 / 2) * 16;       // [NCA][BN2/2 column pairs] float4
  L.cs_off = o; o += 2 * NGRP * 4 * 32 * 4;      // [buf][group][quad][32] float
  L.cm_off = o; o += 2 * NGRP * 4 * 4;           // [buf][group][quad] float
  L.rb_off = o; o += NGRP * 256 * 8;             // [group][256 rows] float2
  L.bar_off = (o + 7) & ~7u; o = L.bar_off + kBarSlots * 8;
  L.misc_off = o; o += 16;
  L.total = o;
  return L;
}

__host__ __device__ __forceinline__ int64_t owner_cta(int64_t tau, int64_t G, int64_t T) { return ((tau + 1) * G - 1) / T; }

template <int MODE>
__global__ void __maxnreg__(128)
tc2_pass_kernel(PassDesc P, TcLayout TL, const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const Tc2Smem SL = tc2_smem(P.d);
  const int kblocks = P.d / 64;
  const int nst = SL.nst;
  uint64_t* bars = (uint64_t*)(smem + SL.bar_off);
  uint64_t* fullA = bars + 0;
  uint64_t* aempty = bars + 1;
  uint64_t* fullB = bars + 2;                  // [nst <= kMaxStages]
  uint64_t* emptyB = bars + 2 + kMaxStages;    // [nst]
  uint64_t* tfull = bars + 2 + 2 * kMaxStages; // [2]
  uint64_t* tempty = tfull + 2;                // [2]
  uint64_t* cfull = tfull + 4;                 // [NCA]
  uint64_t* cempty = cfull + NCA;              // [NCA]
  uint64_t* spare = cempty + NCA;              // stall test hook: receives the withheld hand-off
  uint32_t* s_tmem = (uint32_t*)(smem + SL.misc_off);
  volatile int* s_abort = (volatile int*)(smem + SL.misc_off + 4);
  float4* sCA = (float4*)(smem + SL.ca_off);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (pass_off(P)) return;

  const int64_t G = TL.G, T = TL.T, ntiles = TL.ntiles2;
  const int64_t c = blockIdx.x;
  const int64_t t_start = c * T / G, t_end = (c + 1) * T / G;
  const int nt = (int)(t_end - t_start);

  if (threadIdx.x == 0) {
    mbar_init(fullA, 1);
    mbar_init(aempty, 1);
    for (int s = 0; s < nst; ++s) { mbar_init(fullB + s, 1); mbar_init(emptyB + s, 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(tfull + b, 1); mbar_init(tempty + b, NEPI); }
    for (int k = 0; k < NCA; ++k) { mbar_init(cfull + k, 32); mbar_init(cempty + k, NEPI); }
    mbar_init(spare, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(TMEM2_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0) {
    // ------------------------------------------- TMA + column-term staging
    int a_idx = 0, issued = 0;
    int64_t cur_rb = -1;
    for (int li = 0; li < nt; ++li) {
      const int64_t tau = t_start + li, rb = tau / ntiles, ct = tau % ntiles;
      if (rb != cur_rb) {
        if (a_idx > 0 && !mbar_wait(aempty, (a_idx - 1) & 1, s_abort, P.wait_ns)) break;
        if (lane == 0) {
          mbar_expect_tx(fullA, (uint32_t)(kblocks * 2 * 128 * 128));
          for (int kb = 0; kb < kblocks; ++kb)
            for (int hh = 0; hh < 2; ++hh)
              tma_load_2d(smem + SL.a_off + (kb * 2 + hh) * 128 * 128, &tmX, fullA, kb * 64, (int)(rb * BM2 + hh * 128));
        }
        ++a_idx;
        cur_rb = rb;
      }
      const int s = li % nst;
      if (li >= nst && !mbar_wait(emptyB + s, ((li / nst) - 1) & 1, s_abort, P.wait_ns)) break;
      if (lane == 0) {
        unsigned char* sB = smem + SL.b_off + s * SL.b_stage;
        mbar_expect_tx(fullB + s, SL.b_stage);
        for (int kb = 0; kb < kblocks; ++kb) tma_load_2d(sB + kb * BN2 * 128, &tmY, fullB + s, kb * 64, (int)(ct * BN2));
      }
      issued = li + 1;
      const int cs = li % NCA;
      if (li >= NCA && !mbar_wait(cempty + cs, ((li / NCA) - 1) & 1, s_abort, P.wait_ns)) break;
      {
        // lane l < BN2/4 stages columns 4l .. 4l+3 as pairs (bhi_j, bhi_j+1, blo_j, blo_j+1)
        if (lane < BN2 / 4) {
          const float4* src = reinterpret_cast<const float4*>(P.colA + ct * BN2 + 4 * lane);
          const float4 x = __ldg(src), y = __ldg(src + 1);   // (hi0, lo0, hi1, lo1), (hi2, lo2, hi3, lo3)
          sCA[cs * (BN2 / 2) + 2 * lane] = make_float4(x.x, x.z, x.y, x.w);
          sCA[cs * (BN2 / 2) + 2 * lane + 1] = make_float4(y.x, y.z, y.y, y.w);
        }
        mbar_arrive(cfull + cs);
      }
    }
    __syncwarp();
    if (lane == 0) {
      // our own loads still in flight must land before the CTA may exit
      for (int li = (issued > nst ? issued - nst : 0); li < issued; ++li) mbar_drain(fullB + li % nst, (li / nst) & 1);
      if (a_idx > 0) mbar_drain(fullA, (a_idx - 1) & 1);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, BN2);
      const uint32_t a_base = smem_u32(smem + SL.a_off);
      int a_idx = 0, last = -1;
      int64_t cur_rb = -1;
      for (int li = 0; li < nt; ++li) {
        const int64_t tau = t_start + li, rb = tau / ntiles;
        if (rb != cur_rb) {
          if (!mbar_wait(fullA, a_idx & 1, s_abort, P.wait_ns)) break;
          ++a_idx;
          cur_rb = rb;
        }
        const int b = li & 1, s = li % nst;
        if (li >= 2 && !mbar_wait(tempty + b, ((li >> 1) - 1) & 1, s_abort, P.wait_ns)) break;
        if (!mbar_wait(fullB + s, (li / nst) & 1, s_abort, P.wait_ns)) break;
        tc_fence_after();
        const uint32_t b_base = smem_u32(smem + SL.b_off + s * SL.b_stage);
        for (int kb = 0; kb < kblocks; ++kb) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t bd = sdesc(b_base + kb * BN2 * 128 + kk * 32);
            const uint64_t ad0 = sdesc(a_base + (kb * 2 + 0) * 128 * 128 + kk * 32);
            const uint64_t ad1 = sdesc(a_base + (kb * 2 + 1) * 128 * 128 + kk * 32);
            const uint32_t acc = (kb | kk) != 0;
            umma_bf16(tmem + (uint32_t)(b * 256), ad0, bd, idesc, acc);
            umma_bf16(tmem + (uint32_t)(b * 256 + 128), ad1, bd, idesc, acc);   // second 128 rows
          }
        }
        umma_commit(emptyB + s);
        // test hook (P.stall): the first tile's hand-off goes to a spare barrier, so the
        // epilogue's wait for it runs out and the pass reports the stall
        umma_commit((P.stall && li == 0) ? spare : tfull + b);
        const bool rb_ends = (li + 1 == nt) || ((t_start + li + 1) / ntiles != rb);
        if (rb_ends) umma_commit(aempty);
        last = li;
      }
      // the MMAs of the last committed tile (and all before it) must be complete before TMEM is freed
      if (last >= 0) mbar_drain((P.stall && last == 0) ? spare : tfull + (last & 1), (last >> 1) & 1);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int e = warp - 2;
    const int q = warp & 3;                   // TMEM lane quadrant
    const int g = e >> 2;                     // group of 32 columns (warps 4g+2 .. 4g+5)
    const int r0 = q * 32 + lane;             // row in accumulator 0; + 128 in accumulator 1
    float* csum = (float*)(smem + SL.cs_off);
    float* cmax = (float*)(smem + SL.cm_off);
    float2* rbuf = (float2*)(smem + SL.rb_off);
    const unsigned long long K2 = pk2((float)(2.0 * P.gC * kL2E2), (float)(2.0 * P.gC * kL2E2));
    int64_t cur_rb = -1, slot = 0;
    float ahi0 = 0.f, alo0 = 0.f, ahi1 = 0.f, alo1 = 0.f;
    float Mr0 = POT_NEG_BIGF, Sr0 = 0.f, Mr1 = POT_NEG_BIGF, Sr1 = 0.f;

    auto flush_rows = [&]() {
      if (MODE == V_C) return;
      rbuf[g * 256 + r0] = make_float2(Mr0, Sr0);
      rbuf[g * 256 + r0 + 128] = make_float2(Mr1, Sr1);
      named_bar(5, 32 * NEPI);
      if (g == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = r0 + 128 * h;
          const int64_t i = cur_rb * BM2 + r;
          float M = POT_NEG_BIGF, S = 0.f;
#pragma unroll
          for (int gg = 0; gg < NGRP; ++gg) M = fmaxf(M, rbuf[gg * 256 + r].x);
          if (M > -1.0e29f) {
#pragma unroll
            for (int gg = 0; gg < NGRP; ++gg) {
              const float2 o = rbuf[gg * 256 + r];
              if (o.x > -1.0e29f) S = fmaf(o.y, ex2(o.x - M), S);
            }
          }
          const float lo = h ? alo1 : alo0;
          if (i < P.n) P.row_part[slot * P.n + i] = make_float2(M > -1.0e29f ? lo + M : POT_NEG_BIGF, S);
        }
      }
      named_bar(5, 32 * NEPI);
    };

    for (int li = 0; li < nt; ++li) {
      const int64_t tau = t_start + li, rb = tau / ntiles, ct = tau % ntiles;
      if (rb != cur_rb) {
        if (cur_rb >= 0) flush_rows();
        cur_rb = rb;
        slot = c - owner_cta(rb * ntiles, G, T);
        const float4 ra0 = P.rowA[rb * BM2 + r0], ra1 = P.rowA[rb * BM2 + r0 + 128];
        ahi0 = ra0.x; alo0 = ra0.y; ahi1 = ra1.x; alo1 = ra1.y;
        Mr0 = POT_NEG_BIGF; Sr0 = 0.f; Mr1 = POT_NEG_BIGF; Sr1 = 0.f;
      }
      const int b = li & 1;
      float x0[32], x1[32];
      const bool ok = mbar_wait(tfull + b, (li >> 1) & 1, s_abort, P.wait_ns);
      if (ok) {
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256 + g * 32);
        tmem_ld32(ta, x0);
        tmem_ld32(ta + 128, x1);
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) { x0[k] = 0.f; x1[k] = 0.f; }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + b);

      // ---- logits (log2 units, row lo part applied per row)
      const int cslot = li % NCA;
      const bool okc = mbar_wait(cfull + cslot, (li / NCA) & 1, s_abort, P.wait_ns);
      const unsigned long long AH0 = pk2(ahi0, ahi0), AH1 = pk2(ahi1, ahi1);
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const float4 bb = okc ? sCA[cslot * (BN2 / 2) + g * 16 + p] : make_float4(POT_NEG_BIGF, POT_NEG_BIGF, 0.f, 0.f);
        const unsigned long long BH = pk2(bb.x, bb.y), BL = pk2(bb.z, bb.w);
        unsigned long long y0 = add2(fma2(K2, pk2(x0[2 * p], x0[2 * p + 1]), add2(AH0, BH)), BL);
        unsigned long long y1 = add2(fma2(K2, pk2(x1[2 * p], x1[2 * p + 1]), add2(AH1, BH)), BL);
        upk2(y0, x0[2 * p], x0[2 * p + 1]);
        upk2(y1, x1[2 * p], x1[2 * p + 1]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(cempty + cslot);

      // ---- row maxima (independent chains)
      float m0a = max3f(x0[0], x0[1], x0[2]), m0b = max3f(x0[3], x0[4], x0[5]);
      float m1a = max3f(x1[0], x1[1], x1[2]), m1b = max3f(x1[3], x1[4], x1[5]);
#pragma unroll
      for (int k = 6; k < 30; k += 6) {
        m0a = max3f(m0a, x0[k], x0[k + 1]); m0b = max3f(m0b, x0[k + 2], x0[k + 3]);
        m0a = max3f(m0a, x0[k + 4], x0[k + 5]);
        m1a = max3f(m1a, x1[k], x1[k + 1]); m1b = max3f(m1b, x1[k + 2], x1[k + 3]);
        m1a = max3f(m1a, x1[k + 4], x1[k + 5]);
      }
      const float m0 = max3f(m0a, m0b, fmaxf(x0[30], x0[31]));
      const float m1 = max3f(m1a, m1b, fmaxf(x1[30], x1[31]));
      const bool ok0 = m0 > -1.0e29f, ok1 = m1 > -1.0e29f;

      // ---- exponentials (a fully masked row gets 2^(-big) = 0)
      const unsigned long long NM0 = pk2(ok0 ? -m0 : 0.f, ok0 ? -m0 : 0.f);
      const unsigned long long NM1 = pk2(ok1 ? -m1 : 0.f, ok1 ? -m1 : 0.f);
      unsigned long long s0a = 0ull, s0b = 0ull, s1a = 0ull, s1b = 0ull;   // packed partial sums (bit pattern 0 = 0.0f)
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        float a, bq;
        upk2(add2(pk2(x0[2 * p], x0[2 * p + 1]), NM0), a, bq);
        x0[2 * p] = ex2(a); x0[2 * p + 1] = ex2(bq);
        upk2(add2(pk2(x1[2 * p], x1[2 * p + 1]), NM1), a, bq);
        x1[2 * p] = ex2(a); x1[2 * p + 1] = ex2(bq);
        if (MODE != V_C) {
          if (p & 1) {
            s0b = add2(s0b, pk2(x0[2 * p], x0[2 * p + 1]));
            s1b = add2(s1b, pk2(x1[2 * p], x1[2 * p + 1]));
          } else {
            s0a = add2(s0a, pk2(x0[2 * p], x0[2 * p + 1]));
            s1a = add2(s1a, pk2(x1[2 * p], x1[2 * p + 1]));
          }
        }
      }
      if (MODE != V_C) {
        float u0, u1, w0, w1;
        upk2(add2(s0a, s0b), u0, u1);
        upk2(add2(s1a, s1b), w0, w1);
        const float ss0 = u0 + u1, ss1 = w0 + w1;
        if (ok0) {
          if (m0 > Mr0) { Sr0 = (Mr0 > -1.0e29f ? Sr0 * ex2(Mr0 - m0) : 0.f) + ss0; Mr0 = m0; }
          else Sr0 = fmaf(ss0, ex2(m0 - Mr0), Sr0);
        }
        if (ok1) {
          if (m1 > Mr1) { Sr1 = (Mr1 > -1.0e29f ? Sr1 * ex2(Mr1 - m1) : 0.f) + ss1; Mr1 = m1; }
          else Sr1 = fmaf(ss1, ex2(m1 - Mr1), Sr1);
        }
      }

      // ---- column sums over the warp's 64 rows, merged over the 4 quadrants
      if (MODE != V_R) {
        const float cm0 = ok0 ? alo0 + m0 : POT_NEG_BIGF;
        const float cm1 = ok1 ? alo1 + m1 : POT_NEG_BIGF;
        float Mw = fmaxf(cm0, cm1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Mw = fmaxf(Mw, __shfl_xor_sync(0xffffffffu, Mw, o));
        float v = 0.f;
        if (Mw > -1.0e29f) {
          const float f0 = ok0 ? ex2(cm0 - Mw) : 0.f;
          const float f1 = ok1 ? ex2(cm1 - Mw) : 0.f;
          const unsigned long long F0 = pk2(f0, f0), F1 = pk2(f1, f1);
#pragma unroll
          for (int p = 0; p < 16; ++p) {
            const unsigned long long t = fma2(F0, pk2(x0[2 * p], x0[2 * p + 1]), mul2(F1, pk2(x1[2 * p], x1[2 * p + 1])));
            upk2(t, x0[2 * p], x0[2 * p + 1]);
          }
          v = transpose_reduce32(x0, lane);
        }
        const int buf = li & 1;
        csum[((buf * NGRP + g) * 4 + q) * 32 + lane] = v;
        if (lane == 0) cmax[(buf * NGRP + g) * 4 + q] = Mw;
        named_bar(1 + g, 128);
        if (q == 0) {
          const int64_t j = ct * BN2 + g * 32 + lane;
          float M = POT_NEG_BIGF;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) M = fmaxf(M, cmax[(buf * NGRP + g) * 4 + qq]);
          float S = 0.f;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float Mq = cmax[(buf * NGRP + g) * 4 + qq];
            if (Mq > -1.0e29f) S = fmaf(csum[((buf * NGRP + g) * 4 + qq) * 32 + lane], ex2(Mq - M), S);
          }
          if (j < P.m) P.col_part[rb * P.m + j] = make_float2(M, S);
        }
      }
    }
    if (nt > 0) flush_rows();
  }

  tc_fence_before();
  __syncthreads();
  if (*s_abort && threadIdx.x == 0 && P.err) atomicExch(P.err, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM2_COLS) : "memory");
  }
}

// empty row partials (-big, 0) for the slots no CTA writes
__global__ void tc2_clear_rows_kernel(float2* row_part, int64_t count) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) row_part[t] = make_float2(POT_NEG_BIGF, 0.f);
}

template <int MODE>
cudaError_t launch2(const PassDesc& P, const TcLayout& L, const CUtensorMap& mx, const CUtensorMap& my,
                    cudaStream_t st) {
  const Tc2Smem SL = tc2_smem(P.d);
  const int smem = (int)SL.total + 1024;
  static int configured = 0;
  if (configured < smem) {
    cudaError_t e = cudaFuncSetAttribute(tc2_pass_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  tc2_pass_kernel<MODE><<<(unsigned)L.G, NTHREADS2, smem, st>>>(P, L, mx, my);
  return cudaGetLastError();
}

}  // namespace

bool tc2_applicable(int d) { return d == 64 || d == 128; }
int tc2_tile_cols() { return BN2; }

void tc2_fill_layout(TcLayout& L, int64_t n, int64_t m, int num_sms) {
  L.nrb2 = (n + BM2 - 1) / BM2;
  L.ntiles2 = (m + BN2 - 1) / BN2;
  L.T = L.nrb2 * L.ntiles2;
  L.G = L.T < num_sms ? L.T : num_sms;
  int64_t slots = 1;
  for (int64_t rb = 0; rb < L.nrb2; ++rb) {
    const int64_t a = owner_cta(rb * L.ntiles2, L.G, L.T);
    const int64_t b = owner_cta((rb + 1) * L.ntiles2 - 1, L.G, L.T);
    if (b - a + 1 > slots) slots = b - a + 1;
  }
  L.nslots = slots;
  L.n_pad2 = L.nrb2 * BM2;
  if (L.ntiles2 * BN2 > L.m_pad) L.m_pad = L.ntiles2 * BN2;
}

cudaError_t launch_pass_tc2(const PassDesc& P, const TcLayout& L, const CUtensorMap& mx, const CUtensorMap& my,
                            cudaStream_t st) {
  if (P.mode & PASS_ROWS) {
    const int64_t cnt = L.nslots * P.n;
    tc2_clear_rows_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(P.row_part, cnt);
  }
  const int md = P.mode;
  if ((md & PASS_ROWS) && (md & PASS_COLS)) return launch2<V_RC>(P, L, mx, my, st);
  if (md & PASS_ROWS) return launch2<V_R>(P, L, mx, my, st);
  return launch2<V_C>(P, L, mx, my, st);
}

}  // namespace pot
