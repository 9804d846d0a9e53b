// tcgen05 on-the-fly squared-Euclidean pass for the solver's hot loop
// (BF16 points, d = 64 or 128; rows, columns or both).
//
// Tile geometry.  A row block is 256 rows held as two M = 128 accumulators
// in TMEM; a tile is that row block against 128 columns (one TMA-loaded Y
// tile shared by the two MMAs, N = 128 each).  Two buffers of 2 x 128
// columns fill the 512 TMEM columns, so the MMA warp computes tile t + 1
// while the epilogue reads tile t.  Persistent CTAs, one per SM; CTA c owns
// the contiguous range [c T / G, (c+1) T / G) of the T = ceil(n/256) x
// ceil(m/128) tiles in row-block-major order (the X block stays in shared
// memory while the CTA walks the columns of its row block).
//
// Warp roles (576 threads): warp 0 issues TMA (the X block once per row
// block, a ring of Y tiles) and stages each tile's column terms in shared
// memory; warp 1 allocates TMEM and issues the MMAs; warps 2..17 are the
// epilogue: 4 TMEM lane quadrants (warp % 4) x 4 groups of 32 columns, four
// epilogue warps on every SM sub-partition.  Every epilogue thread owns two
// rows (one lane of each accumulator) and 32 columns of a tile, so the
// column reduction across the warp (a transposing butterfly) is paid once
// per 2 x 32 entries.  (Measured against four rows per thread in 512 x 64
// tiles with eight epilogue warps: the extra warps hide more latency than the
// extra transposes cost, 0.555 against 0.585 ms per two-sided pass at
// n = 32768.)
//
// Numerics (log2 units, per entry):
//   z_ij  = fma(k2, acc_ij, bhi_j) + blo_j          k2 = 2 log2(e) cost_scale / gamma
//   logit = ahi_i + alo_i + z_ij                      (ahi_i + alo_i: row term, constant along the row)
// row side: exact per-tile maximum M_i of z over the 32 columns, one ex2 per
// entry, a running (max, sum) per row in z units (the row term is added once,
// when the row's partial is written); column side: the same exponentials
// scaled by 2^(ahi + alo + M_i - W), W the largest such value among the
// warp's 64 rows, summed over the thread's two rows, then over the warp's
// 32 lanes, then over the four quadrants: one (shift, sum) per column and
// 256-row block.  An entry smaller than 2^-126 times the largest entry of
// its 64-row warp stripe in the tile may be flushed (the same bound as the
// per-warp shift of the other passes).
#include "common.cuh"
#include "pass.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace pot {

namespace {

using namespace tcx;

constexpr int NACC = 2;                           // accumulators (128 rows each) per row block
constexpr int BM3 = 128 * NACC, BN3 = 128;
constexpr int NGRP3 = BN3 / 32;                   // groups of 32 columns
constexpr int NEPI3 = 4 * NGRP3;                  // epilogue warps
constexpr int NTHREADS3 = 64 + 32 * NEPI3;        // + TMA warp + MMA warp
constexpr uint32_t TMEM3_COLS = 512;              // 2 buffers x 2 accumulators x 128 columns
constexpr int NCA3 = 8;                           // column-term ring depth
constexpr int kMaxStages3 = 8;
constexpr int kBarSlots3 = 2 + 2 * kMaxStages3 + 4 + 2 * NCA3 + 1;
constexpr double kL2E3 = 1.4426950408889634;

enum { W_RC = 0, W_R = 1, W_C = 2 };

struct Tc3Smem {
  uint32_t a_off, b_off, b_stage, ca_off, cs_off, cm_off, rb_off, bar_off, misc_off, total;
  int nst;
};

__host__ __device__ inline Tc3Smem tc3_smem(int d) {
  Tc3Smem L;
  const uint32_t kb = (uint32_t)(d / 64);
  L.nst = (d <= 64) ? 6 : 4;
  L.a_off = 0;                                   // [kb][h < 4][128 rows][128 B]
  L.b_off = kb * NACC * 128 * 128;
  L.b_stage = kb * BN3 * 128;                    // [kb][64 rows][128 B]
  uint32_t o = L.b_off + (uint32_t)L.nst * L.b_stage;
  L.ca_off = o; o += NCA3 * (BN3 / 2) * 16;      // [NCA3][32 column pairs] float4
  L.cs_off = o; o += 2 * NGRP3 * 4 * 32 * 4;     // [buf][group][quad][32] float
  L.cm_off = o; o += 2 * NGRP3 * 4 * 4;          // [buf][group][quad] float
  L.rb_off = o; o += NGRP3 * BM3 * 8;            // [group][512 rows] float2
  L.bar_off = (o + 7) & ~7u; o = L.bar_off + kBarSlots3 * 8;
  L.misc_off = o; o += 16;
  L.total = o;
  return L;
}

__host__ __device__ __forceinline__ int64_t owner3(int64_t tau, int64_t G, int64_t T) { return ((tau + 1) * G - 1) / T; }

template <int MODE>
__global__ void __launch_bounds__(NTHREADS3, 1)
tc3_pass_kernel(PassDesc P, TcLayout TL, const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const Tc3Smem SL = tc3_smem(P.d);
  const int kblocks = P.d / 64;
  const int nst = SL.nst;
  uint64_t* bars = (uint64_t*)(smem + SL.bar_off);
  uint64_t* fullA = bars + 0;
  uint64_t* aempty = bars + 1;
  uint64_t* fullB = bars + 2;                   // [nst <= kMaxStages3]
  uint64_t* emptyB = bars + 2 + kMaxStages3;    // [nst]
  uint64_t* tfull = bars + 2 + 2 * kMaxStages3; // [2]
  uint64_t* tempty = tfull + 2;                 // [2]
  uint64_t* cfull = tfull + 4;                  // [NCA3]
  uint64_t* cempty = cfull + NCA3;              // [NCA3]
  uint64_t* spare = cempty + NCA3;              // stall test hook: receives the withheld hand-off
  uint32_t* s_tmem = (uint32_t*)(smem + SL.misc_off);
  volatile int* s_abort = (volatile int*)(smem + SL.misc_off + 4);
  float4* sCA = (float4*)(smem + SL.ca_off);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (pass_off(P)) return;

  const int64_t G = TL.G, T = TL.T, ntiles = TL.ntiles2;
  const int64_t c = blockIdx.x;
  const int64_t t_start = c * T / G, t_end = (c + 1) * T / G;
  const int nt = (int)(t_end - t_start);
  const int64_t rb_first = t_start / ntiles, ct_first = t_start % ntiles;

  if (threadIdx.x == 0) {
    mbar_init(fullA, 1);
    mbar_init(aempty, 1);
    for (int s = 0; s < nst; ++s) { mbar_init(fullB + s, 1); mbar_init(emptyB + s, 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(tfull + b, 1); mbar_init(tempty + b, NEPI3); }
    for (int k = 0; k < NCA3; ++k) { mbar_init(cfull + k, 32); mbar_init(cempty + k, NEPI3); }
    mbar_init(spare, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(TMEM3_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0) {
    // ------------------------------------------- TMA + column-term staging
    int a_idx = 0, issued = 0;
    int64_t rb = rb_first, ct = ct_first, cur_rb = -1;
    for (int li = 0; li < nt; ++li) {
      if (rb != cur_rb) {
        if (a_idx > 0 && !mbar_wait(aempty, (a_idx - 1) & 1, s_abort, P.wait_ns)) break;
        if (lane == 0) {
          mbar_expect_tx(fullA, (uint32_t)(kblocks * NACC * 128 * 128));
          for (int kb = 0; kb < kblocks; ++kb)
            for (int h = 0; h < NACC; ++h)
              tma_load_2d(smem + SL.a_off + (kb * NACC + h) * 128 * 128, &tmX, fullA, kb * 64, (int)(rb * BM3 + h * 128));
        }
        ++a_idx;
        cur_rb = rb;
      }
      const int s = li % nst;
      if (li >= nst && !mbar_wait(emptyB + s, ((li / nst) - 1) & 1, s_abort, P.wait_ns)) break;
      if (lane == 0) {
        unsigned char* sB = smem + SL.b_off + s * SL.b_stage;
        mbar_expect_tx(fullB + s, SL.b_stage);
        for (int kb = 0; kb < kblocks; ++kb) tma_load_2d(sB + kb * BN3 * 128, &tmY, fullB + s, kb * 64, (int)(ct * BN3));
      }
      issued = li + 1;
      const int cs = li % NCA3;
      if (li >= NCA3 && !mbar_wait(cempty + cs, ((li / NCA3) - 1) & 1, s_abort, P.wait_ns)) break;
      // lane l < 16 stages columns 4l .. 4l+3 as pairs (bhi_j, bhi_j+1, blo_j, blo_j+1)
      if (lane < BN3 / 4) {
        const float4* src = reinterpret_cast<const float4*>(P.colA + ct * BN3 + 4 * lane);
        const float4 x = __ldg(src), y = __ldg(src + 1);   // (hi0, lo0, hi1, lo1), (hi2, lo2, hi3, lo3)
        sCA[cs * (BN3 / 2) + 2 * lane] = make_float4(x.x, x.z, x.y, x.w);
        sCA[cs * (BN3 / 2) + 2 * lane + 1] = make_float4(y.x, y.z, y.y, y.w);
      }
      mbar_arrive(cfull + cs);
      if (++ct == ntiles) { ct = 0; ++rb; }
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
      const uint32_t idesc = idesc_bf16(128, BN3);
      const uint32_t a_base = smem_u32(smem + SL.a_off);
      int a_idx = 0, last = -1;
      int64_t rb = rb_first, ct = ct_first, cur_rb = -1;
      for (int li = 0; li < nt; ++li) {
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
            const uint64_t bd = sdesc(b_base + kb * BN3 * 128 + kk * 32);
            const uint32_t acc = (kb | kk) != 0;
#pragma unroll
            for (int h = 0; h < NACC; ++h)
              umma_bf16(tmem + (uint32_t)(b * 256 + h * BN3), sdesc(a_base + (kb * NACC + h) * 128 * 128 + kk * 32),
                        bd, idesc, acc);
          }
        }
        umma_commit(emptyB + s);
        // test hook (P.stall): the first tile's hand-off goes to a spare barrier, so the
        // epilogue's wait for it runs out and the pass reports the stall
        umma_commit((P.stall && li == 0) ? spare : tfull + b);
        if (++ct == ntiles) { ct = 0; ++rb; }
        if (li + 1 == nt || rb != cur_rb) umma_commit(aempty);
        last = li;
      }
      // the MMAs of the last committed tile (and all before it) must be complete before TMEM is freed
      if (last >= 0) mbar_drain((P.stall && last == 0) ? spare : tfull + (last & 1), (last >> 1) & 1);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;                   // TMEM lane quadrant of this warp
    const int g = (warp - 2) >> 2;            // group of 32 columns
    const int r0 = q * 32 + lane;             // row of accumulator h: r0 + 128 h
    float* csum = (float*)(smem + SL.cs_off);
    float* cmax = (float*)(smem + SL.cm_off);
    float2* rbuf = (float2*)(smem + SL.rb_off);
    const unsigned long long K2 = pk2((float)(2.0 * P.gC * kL2E3), (float)(2.0 * P.gC * kL2E3));
    // 32-bit tile indices (n / 512 and m / 64 fit easily) keep the loop state small
    int rb = (int)rb_first, ct = (int)ct_first, cur_rb = -1, slot = 0;
    const int ntl = (int)ntiles, pn = (int)P.n, pm = (int)P.m;
    float2* const rowp = P.row_part;
    float2* const colp = P.col_part;
    float arow[NACC], Mr[NACC], Sr[NACC];      // arow: ahi + alo of the thread's rows
#pragma unroll
    for (int h = 0; h < NACC; ++h) { arow[h] = POT_NEG_BIGF; Mr[h] = POT_NEG_BIGF; Sr[h] = 0.f; }

    auto flush_rows = [&]() {
      if (MODE == W_C) return;
#pragma unroll
      for (int h = 0; h < NACC; ++h) rbuf[g * BM3 + r0 + 128 * h] = make_float2(Mr[h], Sr[h]);
      named_bar(5, 32 * NEPI3);
      if (g == 0) {
#pragma unroll
        for (int h = 0; h < NACC; ++h) {
          const int r = r0 + 128 * h;
          const int i = cur_rb * BM3 + r;
          float M = POT_NEG_BIGF, S = 0.f;
#pragma unroll
          for (int gg = 0; gg < NGRP3; ++gg) M = fmaxf(M, rbuf[gg * BM3 + r].x);
          if (M > -1.0e29f) {
#pragma unroll
            for (int gg = 0; gg < NGRP3; ++gg) {
              const float2 o = rbuf[gg * BM3 + r];
              if (o.x > -1.0e29f) S = fmaf(o.y, ex2(o.x - M), S);
            }
          }
          const bool ok = M > -1.0e29f && arow[h] > -1.0e29f && S > 0.f;
          if (i < pn) rowp[(int64_t)slot * pn + i] = make_float2(ok ? arow[h] + M : POT_NEG_BIGF, ok ? S : 0.f);
        }
      }
      named_bar(5, 32 * NEPI3);
    };

    for (int li = 0; li < nt; ++li) {
      if (rb != cur_rb) {
        if (cur_rb >= 0) flush_rows();
        cur_rb = rb;
        slot = (int)(c - owner3((int64_t)rb * ntiles, G, T));
#pragma unroll
        for (int h = 0; h < NACC; ++h) {
          const float4 ra = P.rowA[(int64_t)rb * BM3 + r0 + 128 * h];
          arow[h] = ra.x > -1.0e29f ? ra.x + ra.y : POT_NEG_BIGF;
          Mr[h] = POT_NEG_BIGF; Sr[h] = 0.f;
        }
      }
      const int b = li & 1;
      float x[NACC][32];
      const bool ok = mbar_wait(tfull + b, (li >> 1) & 1, s_abort, P.wait_ns);
      if (ok) {
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256 + g * 32);
#pragma unroll
        for (int h = 0; h < NACC; ++h) tmem_ld32(ta + (uint32_t)(h * BN3), x[h]);
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int h = 0; h < NACC; ++h)
#pragma unroll
          for (int k = 0; k < 32; ++k) x[h][k] = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + b);

      // ---- z = k2 acc + bhi + blo (the row term is constant along the row)
      const int cslot = li % NCA3;
      const bool okc = mbar_wait(cfull + cslot, (li / NCA3) & 1, s_abort, P.wait_ns);
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const float4 bb = okc ? sCA[cslot * (BN3 / 2) + g * 16 + p] : make_float4(POT_NEG_BIGF, POT_NEG_BIGF, 0.f, 0.f);
        const unsigned long long BH = pk2(bb.x, bb.y), BL = pk2(bb.z, bb.w);
#pragma unroll
        for (int h = 0; h < NACC; ++h) {
          const unsigned long long z = add2(fma2(K2, pk2(x[h][2 * p], x[h][2 * p + 1]), BH), BL);
          upk2(z, x[h][2 * p], x[h][2 * p + 1]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(cempty + cslot);

      // ---- per-row maxima over the 32 columns (independent 3-input chains)
      float m[NACC];
#pragma unroll
      for (int h = 0; h < NACC; ++h) {
        float ma = max3f(x[h][0], x[h][1], x[h][2]), mb = max3f(x[h][3], x[h][4], x[h][5]);
#pragma unroll
        for (int k = 6; k < 30; k += 6) {
          ma = max3f(ma, x[h][k], x[h][k + 1]); mb = max3f(mb, x[h][k + 2], x[h][k + 3]);
          ma = max3f(ma, x[h][k + 4], x[h][k + 5]);
        }
        m[h] = max3f(ma, mb, fmaxf(x[h][30], x[h][31]));
      }
      bool okr[NACC];
#pragma unroll
      for (int h = 0; h < NACC; ++h) okr[h] = m[h] > -1.0e29f && arow[h] > -1.0e29f;

      // ---- exponentials relative to the row maxima, row sums
#pragma unroll
      for (int h = 0; h < NACC; ++h) {
        const unsigned long long NM = pk2(okr[h] ? -m[h] : POT_NEG_BIGF, okr[h] ? -m[h] : POT_NEG_BIGF);
        unsigned long long sa = 0ull, sb = 0ull;   // packed partial sums (bit pattern 0 = 0.0f)
#pragma unroll
        for (int p = 0; p < 16; ++p) {
          float a0, a1;
          upk2(add2(pk2(x[h][2 * p], x[h][2 * p + 1]), NM), a0, a1);
          x[h][2 * p] = ex2(a0); x[h][2 * p + 1] = ex2(a1);
          if (MODE != W_C) {
            if (p & 1) sb = add2(sb, pk2(x[h][2 * p], x[h][2 * p + 1]));
            else sa = add2(sa, pk2(x[h][2 * p], x[h][2 * p + 1]));
          }
        }
        if (MODE != W_C && okr[h]) {
          float u0, u1;
          upk2(add2(sa, sb), u0, u1);
          const float ss = u0 + u1;
          if (m[h] > Mr[h]) { Sr[h] = (Mr[h] > -1.0e29f ? Sr[h] * ex2(Mr[h] - m[h]) : 0.f) + ss; Mr[h] = m[h]; }
          else Sr[h] = fmaf(ss, ex2(m[h] - Mr[h]), Sr[h]);
        }
      }

      // ---- column sums over the thread's 4 rows, the warp's 32 lanes and the 4 quadrants
      if (MODE != W_R) {
        float cm[NACC];
        float Mw = POT_NEG_BIGF;
#pragma unroll
        for (int h = 0; h < NACC; ++h) {
          cm[h] = okr[h] ? arow[h] + m[h] : POT_NEG_BIGF;
          Mw = fmaxf(Mw, cm[h]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Mw = fmaxf(Mw, __shfl_xor_sync(0xffffffffu, Mw, o));
        float v = 0.f;
        if (Mw > -1.0e29f) {
          unsigned long long F[NACC];
#pragma unroll
          for (int h = 0; h < NACC; ++h) {
            const float f = okr[h] ? ex2(cm[h] - Mw) : 0.f;
            F[h] = pk2(f, f);
          }
#pragma unroll
          for (int p = 0; p < 16; ++p) {
            unsigned long long t = mul2(F[0], pk2(x[0][2 * p], x[0][2 * p + 1]));
#pragma unroll
            for (int h = 1; h < NACC; ++h) t = fma2(F[h], pk2(x[h][2 * p], x[h][2 * p + 1]), t);
            upk2(t, x[0][2 * p], x[0][2 * p + 1]);
          }
          v = transpose_reduce32(x[0], lane);
        }
        const int buf = li & 1;
        csum[((buf * NGRP3 + g) * 4 + q) * 32 + lane] = v;
        if (lane == 0) cmax[(buf * NGRP3 + g) * 4 + q] = Mw;
        named_bar(1 + g, 128);
        if (q == 0) {
          const int j = ct * BN3 + g * 32 + lane;
          float M = POT_NEG_BIGF;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) M = fmaxf(M, cmax[(buf * NGRP3 + g) * 4 + qq]);
          float S = 0.f;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float Mq = cmax[(buf * NGRP3 + g) * 4 + qq];
            if (Mq > -1.0e29f) S = fmaf(csum[((buf * NGRP3 + g) * 4 + qq) * 32 + lane], ex2(Mq - M), S);
          }
          if (j < pm) colp[(int64_t)rb * pm + j] = make_float2(M, S);
        }
      }
      if (++ct == ntl) { ct = 0; ++rb; }
    }
    if (nt > 0) flush_rows();
  }

  tc_fence_before();
  __syncthreads();
  if (*s_abort && threadIdx.x == 0 && P.err) atomicExch(P.err, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM3_COLS) : "memory");
  }
}

// empty row partials (-big, 0) for the slots no CTA writes (nothing when the
// pass is off: a skipped pass must leave the previous partials in place)
__global__ void tc3_clear_rows_kernel(PassDesc P, float2* row_part, int64_t count) {
  if (pass_off(P)) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) row_part[t] = make_float2(POT_NEG_BIGF, 0.f);
}

// Per-pass terms of the transposed problem (rows = the columns j, columns =
// the rows i), the arithmetic of prep_kernel with the two sides exchanged:
//   rowA[j] = (hi, lo of (b_j - gC |y_j|^2) log2 e, |y_j|^2, 0)
//   colA[i] = (hi, lo of (a_i + aoff - gC |x_i|^2) log2 e)
// padding entries are log 0.
__global__ void tc3_prep_swap_kernel(PassDesc P, int64_t rows_pad, int64_t cols_pad) {
  if (pass_off(P)) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool use1 = P.sel && *P.sel;
  const double* arow = use1 ? P.arow1 : P.arow0;
  const double* bcol = use1 ? P.bcol1 : P.bcol0;
  const double* aoffp = use1 ? P.aoff1 : P.aoff0;
  if (t < rows_pad) {
    float4 o = make_float4(POT_NEG_BIGF, 0.f, 0.f, 0.f);
    if (t < P.m) {
      const float yn = P.yn[t];
      HiLo hl = split_hilo(((double)bcol[t] - P.gC * (double)yn) * kL2E3);
      o = make_float4(hl.hi, hl.lo, yn, 0.f);
    }
    P.rowA[t] = o;
  } else if (t < rows_pad + cols_pad) {
    const int64_t i = t - rows_pad;
    float2 A = make_float2(POT_NEG_BIGF, 0.f);
    if (i < P.n) {
      const float xn = P.xn[i];
      HiLo hl = split_hilo((arow[i] + (aoffp ? *aoffp : 0.0) - P.gC * (double)xn) * kL2E3);
      A = make_float2(hl.hi, hl.lo);
    }
    P.colA[i] = A;
  }
}

template <int MODE>
cudaError_t launch3(const PassDesc& P, const TcLayout& L, const CUtensorMap& mx, const CUtensorMap& my,
                    cudaStream_t st) {
  const Tc3Smem SL = tc3_smem(P.d);
  const int smem = (int)SL.total + 1024;
  static int configured = 0;
  if (configured < smem) {
    cudaError_t e = cudaFuncSetAttribute(tc3_pass_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  tc3_pass_kernel<MODE><<<(unsigned)L.G, NTHREADS3, smem, st>>>(P, L, mx, my);
  return cudaGetLastError();
}

}  // namespace

bool tc3_applicable(int d) { return d == 64 || d == 128; }
int tc3_tile_cols() { return BN3; }

// The columns-only pass runs as the rows-only kernel on the transposed
// problem: a columns-only tile pays the per-tile transposing reduction across
// the warp, the quadrant merge and a partial per 256 rows, a rows-only tile
// reduces along its own registers and keeps running sums.  Its layout is the
// one of (m, n); each column then has sw_nslots partials (the CTAs sharing a
// row block of the transposed problem) instead of one per 256 rows, so only
// where the combine kernel reads them (more than 32 row blocks; the loop
// kernels' inline combine expects one per row block).
static void tc3_fill_swap(TcLayout& L, int64_t n, int64_t m, int num_sms) {
  TcLayout S{};
  S.m_pad = 0;
  tc3_fill_layout(S, m, n, num_sms);
  L.sw_G = S.G; L.sw_T = S.T; L.sw_ntiles2 = S.ntiles2; L.sw_nrb2 = S.nrb2; L.sw_nslots = S.nslots;
  L.sw_rows_pad = S.nrb2 * BM3;
  L.sw_cols_pad = S.ntiles2 * BN3;
  L.swap = L.nrb2 > 32 ? 1 : 0;
}

void tc3_fill_layout(TcLayout& L, int64_t n, int64_t m, int num_sms) {
  L.nrb2 = (n + BM3 - 1) / BM3;
  L.ntiles2 = (m + BN3 - 1) / BN3;
  L.T = L.nrb2 * L.ntiles2;
  L.G = L.T < num_sms ? L.T : num_sms;
  int64_t slots = 1;
  for (int64_t rb = 0; rb < L.nrb2; ++rb) {
    const int64_t a = owner3(rb * L.ntiles2, L.G, L.T);
    const int64_t b = owner3((rb + 1) * L.ntiles2 - 1, L.G, L.T);
    if (b - a + 1 > slots) slots = b - a + 1;
  }
  L.nslots = slots;
  L.n_pad2 = L.nrb2 * BM3;
  if (L.ntiles2 * BN3 > L.m_pad) L.m_pad = L.ntiles2 * BN3;
}

void tc3_fill_layout_swap(TcLayout& L, int64_t n, int64_t m, int num_sms) { tc3_fill_swap(L, n, m, num_sms); }

cudaError_t launch_pass_tc3_cols_swapped(const PassDesc& P, const TcLayout& L, const CUtensorMap& my_rows,
                                         const CUtensorMap& mx_cols, cudaStream_t st) {
  {
    const int64_t tot = L.sw_rows_pad + L.sw_cols_pad;
    tc3_prep_swap_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(P, L.sw_rows_pad, L.sw_cols_pad);
  }
  PassDesc Q = P;
  Q.n = P.m; Q.m = P.n;
  Q.X = P.Y; Q.Y = P.X; Q.ldx = P.ldy; Q.ldy = P.ldx; Q.xn = P.yn; Q.yn = P.xn;
  Q.mode = PASS_ROWS;
  Q.row_part = P.col_part;            // [sw_nslots][m]: the column partials
  Q.col_part = nullptr;
  TcLayout S = L;
  S.G = L.sw_G; S.T = L.sw_T; S.ntiles2 = L.sw_ntiles2; S.nrb2 = L.sw_nrb2; S.nslots = L.sw_nslots;
  const int64_t cnt = L.sw_nslots * Q.n;
  tc3_clear_rows_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Q, Q.row_part, cnt);
  return launch3<W_R>(Q, S, my_rows, mx_cols, st);
}

cudaError_t launch_pass_tc3(const PassDesc& P, const TcLayout& L, const CUtensorMap& mx, const CUtensorMap& my,
                            cudaStream_t st) {
  if (P.mode & PASS_ROWS) {
    const int64_t cnt = L.nslots * P.n;
    tc3_clear_rows_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(P, P.row_part, cnt);
  }
  const int md = P.mode;
  if ((md & PASS_ROWS) && (md & PASS_COLS)) return launch3<W_RC>(P, L, mx, my, st);
  if (md & PASS_ROWS) return launch3<W_R>(P, L, mx, my, st);
  return launch3<W_C>(P, L, mx, my, st);
}

}  // namespace pot
