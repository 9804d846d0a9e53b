// On-the-fly squared-Euclidean passes on the 5th-generation tensor cores
// (tcgen05, sm_103a) for BF16 point clouds.
//
// For a tile of 128 rows x 128 columns the dot products x_i . y_j are formed
// by tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 accumulator in TMEM) from
// TMA-loaded, 128B-swizzled shared-memory tiles; the cost
//   C_ij = cost_scale (|x_i|^2 + |y_j|^2 - 2 x_i . y_j)
// is never written anywhere.  The epilogue reads the accumulator with
// tcgen05.ld and fuses
//   logit2_ij = a_i + b_j + k2 * acc_ij        (log2 units, k2 = 2 log2(e) cost_scale / gamma)
// with the row and column log-sum-exp reductions of the pass:
//   * row side: each epilogue thread owns one row (one TMEM lane) and 64
//     columns of a tile; exact per-tile row max, one ex2 per entry;
//   * column side: the same exponentials are rescaled by a per-row factor
//     relative to the warp's largest row maximum and reduced over the 32 rows
//     of the warp with a transposing butterfly; four warps are merged in
//     shared memory into one (shift, sum) partial per column and 128 rows.
// The row potential enters as hi + lo where hi lies on a 2^-10 grid, so
// hi_a + hi_b is exact in FP32 and the FMA rounds once relative to the small
// result; lo_a is applied per row (it is constant along the row).
//
// Warp roles (320 threads): warp 0 issues TMA loads (X tile once per work
// unit, a 2-stage ring of Y tiles), warp 1 allocates TMEM (2 x 128 columns,
// double-buffered accumulator) and issues the MMAs, warps 2..9 are the
// epilogue (warps 2-5 take columns 0-63 of a tile, warps 6-9 columns 64-127).
// Every wait on an mbarrier is bounded by %globaltimer: after 2 s the kernel
// raises an error flag, stops issuing work and still frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include "common.cuh"
#include "pass.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace pot {

namespace {

constexpr int BM = 128, BN = 128;
constexpr int NSTAGE = 2;
constexpr int NTHREADS = 320;
constexpr uint32_t TMEM_COLS = 256;
constexpr double kL2E = 1.4426950408889634;

enum { M_RC = 0, M_R = 1, M_C = 2, M_MAX = 3, M_OBJ = 4 };

using namespace tcx;

struct TcSmemLayout {
  uint32_t a_off, b_off, b_stage, cs_off, cm_off, rs_off, red_off, bar_off, misc_off, total;
};

__host__ __device__ inline TcSmemLayout tc_smem_layout(int d) {
  TcSmemLayout L;
  const uint32_t kb = (uint32_t)(d / 64);
  L.a_off = 0;
  L.b_stage = kb * BN * 128;
  L.b_off = kb * BM * 128;
  uint32_t o = L.b_off + NSTAGE * L.b_stage;
  L.cs_off = o; o += 2 * 2 * 4 * 64 * 4;     // [buf][half][quad][64] floats
  L.cm_off = o; o += 2 * 2 * 4 * 4;          // [buf][half][quad]
  L.rs_off = o; o += 2 * 128 * 8;            // [half][row] float2
  L.red_off = o; o += 16 * 8;                // per-warp doubles
  L.bar_off = (o + 7) & ~7u; o = L.bar_off + 16 * 8;
  L.misc_off = o; o += 16;
  L.total = o;
  return L;
}

template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
tc_pass_kernel(PassDesc P, TcLayout TL, const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled operand tiles
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const TcSmemLayout SL = tc_smem_layout(P.d);
  const int kblocks = P.d / 64;
  uint64_t* bars = (uint64_t*)(smem + SL.bar_off);
  uint64_t* fullA = bars + 0;
  uint64_t* fullB = bars + 1;           // [NSTAGE]
  uint64_t* emptyB = bars + 1 + NSTAGE; // [NSTAGE]
  uint64_t* tfull = bars + 1 + 2 * NSTAGE;      // [2]
  uint64_t* tempty = bars + 3 + 2 * NSTAGE;     // [2]
  uint32_t* s_tmem = (uint32_t*)(smem + SL.misc_off);
  volatile int* s_abort = (volatile int*)(smem + SL.misc_off + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (pass_off(P)) return;

  const int64_t unit = blockIdx.x;
  const int64_t rb = unit / TL.nchunks, ch = unit % TL.nchunks;
  const int64_t ntiles = (P.m + BN - 1) / BN;
  const int64_t t_begin = ch * TL.tiles_per_chunk;
  const int64_t t_end = (t_begin + TL.tiles_per_chunk < ntiles) ? t_begin + TL.tiles_per_chunk : ntiles;
  const int nt = (int)(t_end - t_begin);

  if (threadIdx.x == 0) {
    mbar_init(fullA, 1);
    for (int s = 0; s < NSTAGE; ++s) { mbar_init(fullB + s, 1); mbar_init(emptyB + s, 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(tfull + b, 1); mbar_init(tempty + b, 8); }
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0 && nt > 0) {
      unsigned char* sA = smem + SL.a_off;
      mbar_expect_tx(fullA, (uint32_t)(kblocks * BM * 128));
      for (int kb = 0; kb < kblocks; ++kb)
        tma_load_2d(sA + kb * BM * 128, &tmX, fullA, kb * 64, (int)(rb * BM));
      int issued = 0;
      for (int li = 0; li < nt; ++li) {
        const int s = li % NSTAGE;
        if (li >= NSTAGE && !mbar_wait(emptyB + s, ((li / NSTAGE) - 1) & 1, s_abort, P.wait_ns)) break;
        unsigned char* sB = smem + SL.b_off + s * SL.b_stage;
        mbar_expect_tx(fullB + s, SL.b_stage);
        const int col = (int)((t_begin + li) * BN);
        for (int kb = 0; kb < kblocks; ++kb) tma_load_2d(sB + kb * BN * 128, &tmY, fullB + s, kb * 64, col);
        issued = li + 1;
      }
      // wait for our own loads still in flight before the CTA may exit
      for (int li = (issued > NSTAGE ? issued - NSTAGE : 0); li < issued; ++li) mbar_drain(fullB + li % NSTAGE, (li / NSTAGE) & 1);
      mbar_drain(fullA, 0);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0 && nt > 0) {
      const uint32_t idesc = idesc_bf16(BM, BN);
      const uint32_t a_base = smem_u32(smem + SL.a_off);
      int last = -1;
      if (mbar_wait(fullA, 0, s_abort, P.wait_ns)) {
        for (int li = 0; li < nt; ++li) {
          const int b = li & 1, s = li % NSTAGE;
          if (li >= 2 && !mbar_wait(tempty + b, ((li >> 1) - 1) & 1, s_abort, P.wait_ns)) break;
          if (!mbar_wait(fullB + s, (li / NSTAGE) & 1, s_abort, P.wait_ns)) break;
          tc_fence_after();
          const uint32_t b_base = smem_u32(smem + SL.b_off + s * SL.b_stage);
          for (int kb = 0; kb < kblocks; ++kb) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = sdesc(a_base + kb * BM * 128 + kk * 32);
              const uint64_t bd = sdesc(b_base + kb * BN * 128 + kk * 32);
              umma_bf16(tmem + (uint32_t)(b * BN), ad, bd, idesc, (kb | kk) != 0);
            }
          }
          umma_commit(emptyB + s);
          umma_commit(tfull + b);
          last = li;
        }
      }
      // the accumulator of the last issued tile must be complete before TMEM is freed
      if (last >= 0) mbar_drain(tfull + (last & 1), (last >> 1) & 1);
    }
  } else {
    // ----------------------------------------------------------- epilogue
    const int q = warp & 3;                  // TMEM lane quadrant of this warp
    const int h = (warp - 2) >> 2;           // column half of the tile
    const int r = q * 32 + lane;
    const int64_t i = rb * BM + r;
    const float4 ra = P.rowA[i];             // rows padded to a multiple of 128
    const float ahi = ra.x, alo = ra.y;
    const float k2 = (MODE == M_MAX) ? -2.0f : (float)(2.0 * P.gC * kL2E);
    float* cs = (float*)(smem + SL.cs_off);
    float* cm = (float*)(smem + SL.cm_off);
    float2* rs = (float2*)(smem + SL.rs_off);
    float Mr = POT_NEG_BIGF, Sr = 0.f;        // running row (max, sum) over this half's columns
    float maxc = POT_NEG_BIGF;
    double objacc = 0.0;
    const float kap = (MODE == M_OBJ) ? (float)*P.kappa : 0.f;
    const float4* colA4 = reinterpret_cast<const float4*>(P.colA);
    for (int li = 0; li < nt; ++li) {
      const int b = li & 1;
      const int64_t j0 = (t_begin + li) * BN + h * 64;
      float t[64];
      const bool ok = mbar_wait(tfull + b, (li >> 1) & 1, s_abort, P.wait_ns);
      if (ok) {
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + h * 64);
        tmem_ld32(ta, t);
        tmem_ld32(ta + 32, t + 32);
        tmem_wait_ld();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + b);
      if (!ok) {
#pragma unroll
        for (int k = 0; k < 64; ++k) t[k] = 0.f;
      }
      if (MODE == M_OBJ) {
        // <C, X> contribution: raw cost from the accumulator, plan entry from the logit
        const float2* colB2 = P.colB;
        float accf = 0.f;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const float4 bb = __ldg(colA4 + ((j0 >> 1) + c));
#pragma unroll
          for (int e2 = 0; e2 < 2; ++e2) {
            const int k = 2 * c + e2;
            const float2 yq = __ldg(colB2 + j0 + k);
            const float bh = e2 ? bb.z : bb.x, bl = e2 ? bb.w : bb.y;
            const float lg = fmaf(k2, t[k], ahi + bh) + bl + alo;
            const float x = ex2(lg) + kap * ra.w * yq.y;
            const float cst = fmaxf(fmaf(-2.f, t[k], ra.z + yq.x), 0.f);
            accf = fmaf(cst, x, accf);
          }
        }
        objacc += (double)accf;
        continue;
      }
      // logits (log2 units, without the per-row lo part)
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float4 bb = __ldg(colA4 + ((j0 >> 1) + c));
        t[2 * c] = fmaf(k2, t[2 * c], ahi + bb.x) + bb.y;
        t[2 * c + 1] = fmaf(k2, t[2 * c + 1], ahi + bb.z) + bb.w;
      }
      if (MODE == M_MAX) {          // NaN-keeping max: a NaN coordinate must reach the finiteness check
#pragma unroll
        for (int k = 0; k < 64; ++k) maxc = nanmaxf(maxc, t[k]);
        continue;
      }
      float mx = t[0];
#pragma unroll
      for (int k = 1; k < 64; ++k) mx = fmaxf(mx, t[k]);
      const bool rowok = mx > -1.0e29f;
      float ssum = 0.f;
#pragma unroll
      for (int k = 0; k < 64; ++k) {
        const float e = rowok ? ex2(t[k] - mx) : 0.f;
        t[k] = e;
        ssum += e;
      }
      if (MODE == M_RC || MODE == M_R) {
        if (rowok) {
          if (mx > Mr) { Sr = Sr * ex2(Mr - mx) + ssum; Mr = mx; }
          else Sr = fmaf(ssum, ex2(mx - Mr), Sr);
        }
      }
      if (MODE == M_RC || MODE == M_C) {
        const float cmv = rowok ? alo + mx : POT_NEG_BIGF;
        float Mw = cmv;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Mw = fmaxf(Mw, __shfl_xor_sync(0xffffffffu, Mw, o));
        float v0 = 0.f, v1 = 0.f;
        if (Mw > -1.0e29f) {
          const float f = rowok ? ex2(cmv - Mw) : 0.f;
#pragma unroll
          for (int k = 0; k < 64; ++k) t[k] *= f;
          v0 = transpose_reduce32(t, lane);
          v1 = transpose_reduce32(t + 32, lane);
        }
        const int buf = li & 1;
        float* csb = cs + ((buf * 2 + h) * 4 + q) * 64;
        csb[lane] = v0;
        csb[32 + lane] = v1;
        if (lane == 0) cm[(buf * 2 + h) * 4 + q] = Mw;
        named_bar(1 + h, 128);
        if (q == 0) {
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int c = lane + 32 * cc;
            const int64_t j = j0 + c;
            float M = POT_NEG_BIGF;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) M = fmaxf(M, cm[(buf * 2 + h) * 4 + qq]);
            float S = 0.f;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const float Mq = cm[(buf * 2 + h) * 4 + qq];
              if (Mq > -1.0e29f) S = fmaf(cs[((buf * 2 + h) * 4 + qq) * 64 + c], ex2(Mq - M), S);
            }
            if (j < P.m) P.col_part[rb * P.m + j] = make_float2(M, S);
          }
        }
      }
    }
    // row partials: merge the two column halves
    if (MODE == M_RC || MODE == M_R) {
      rs[h * 128 + r] = make_float2(Mr, Sr);
      named_bar(3, 256);
      if (h == 0 && i < P.n) {
        const float2 o = rs[128 + r];
        float M = Mr, S = Sr;
        if (o.x > M) { S = S * (M > -1.0e29f ? ex2(M - o.x) : 0.f) + o.y; M = o.x; }
        else if (o.x > -1.0e29f) S = fmaf(o.y, ex2(o.x - M), S);
        P.row_part[ch * P.n + i] = make_float2(M > -1.0e29f ? alo + M : POT_NEG_BIGF, S);
      }
    }
    if (MODE == M_MAX || MODE == M_OBJ) {
      double* red = (double*)(smem + SL.red_off);
      double v = (MODE == M_MAX) ? (double)maxc : objacc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, v, o);
        v = (MODE == M_MAX) ? nanmax(v, y) : v + y;
      }
      if (lane == 0) red[warp - 2] = v;
      named_bar(3, 256);
      if (threadIdx.x == 64) {
        double mm = red[0];
        for (int w = 1; w < 8; ++w) mm = (MODE == M_MAX) ? nanmax(mm, red[w]) : mm + red[w];
        P.red_part[unit] = mm;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (*s_abort && threadIdx.x == 0 && P.err) atomicExch(P.err, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool make_map(CUtensorMap* map, const void* base, int64_t rows, int d, int64_t ld, int box_rows = 128) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int MODE>
cudaError_t launch_mode(const PassDesc& P, const TcLayout& L, const CUtensorMap& mx, const CUtensorMap& my,
                        cudaStream_t st) {
  const TcSmemLayout SL = tc_smem_layout(P.d);
  uint32_t smem = SL.total + 1024;
  if (smem < 100 * 1024) smem = 100 * 1024;     // at most two CTAs (2 x 256 TMEM columns) per SM
  static int configured = 0;
  if (configured < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(tc_pass_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = (int)smem;
  }
  tc_pass_kernel<MODE><<<(unsigned)L.v1_units, NTHREADS, smem, st>>>(P, L, mx, my);
  return cudaGetLastError();
}

}  // namespace

TcLayout tc_layout(int64_t n, int64_t m, int d) {
  TcLayout L{};
  L.v1_nrowblk = (n + BM - 1) / BM;
  const int64_t ntiles = (m + BN - 1) / BN;
  // general kernel: choose the number of column chunks so that the work units
  // fill whole waves of 2 x 152 resident CTAs as evenly as possible (>= 8 tiles a unit)
  const int64_t slots = 2 * 152;
  double best = -1.0;
  int64_t best_c = 1;
  for (int64_t c = 1; c <= 64 && c <= ntiles; ++c) {
    const int64_t tpc = (ntiles + c - 1) / c;
    if (tpc < 8 && c > 1) break;
    const int64_t units = L.v1_nrowblk * ((ntiles + tpc - 1) / tpc);
    const double waves = (double)units / slots;
    const double eff = waves / ceil(waves);
    if (eff > best + 1e-9) { best = eff; best_c = c; }
  }
  L.tiles_per_chunk = (ntiles + best_c - 1) / best_c;
  L.nchunks = (ntiles + L.tiles_per_chunk - 1) / L.tiles_per_chunk;
  L.v1_units = L.v1_nrowblk * L.nchunks;
  L.n_pad = L.v1_nrowblk * BM;
  L.m_pad = ntiles * BN;
  L.v3 = tc3_applicable(d) ? 1 : 0;
  if (L.v3) {
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 152;
    }
    tc3_fill_layout(L, n, m, sms);
    tc3_fill_layout_swap(L, n, m, sms);
    if (L.n_pad2 > L.n_pad) L.n_pad = L.n_pad2;
    if (L.swap) {                   // the transposed pass's terms share the row / column term buffers
      if (L.sw_rows_pad > L.n_pad) L.n_pad = L.sw_rows_pad;
      if (L.sw_cols_pad > L.m_pad) L.m_pad = L.sw_cols_pad;
    }
    L.ncolblk = L.nslots;
    L.nrowblk = L.nrb2;
  } else {
    L.ncolblk = L.nchunks;
    L.nrowblk = L.v1_nrowblk;
  }
  L.ok = 1;
  return L;
}

bool tc_supported(const PassDesc& P) {
  if (P.kind != COST_SQEUCLID_BF16) return false;
  if (P.d < 64 || P.d > 256 || (P.d % 64) != 0) return false;
  if ((P.ldx * 2) % 16 != 0 || (P.ldy * 2) % 16 != 0) return false;
  if (((uintptr_t)P.X % 16) != 0 || ((uintptr_t)P.Y % 16) != 0) return false;
  if (P.n >= (int64_t(1) << 30) || P.m >= (int64_t(1) << 30)) return false;
  return true;
}

cudaError_t launch_pass_tc(const PassDesc& P, const TcLayout& L, cudaStream_t st, cudaEvent_t before_main) {
  CUtensorMap mx, my;
  const int md = P.mode;
  cudaError_t e;
  if (tc_swaps_cols(L, P)) {
    // rows of the transposed problem: A tiles from Y, B tiles from X
    if (before_main && (e = cudaEventRecordWithFlags(before_main, st, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (!make_map(&my, P.Y, P.m, P.d, P.ldy, 128) || !make_map(&mx, P.X, P.n, P.d, P.ldx, tc3_tile_cols()))
      return cudaErrorInvalidValue;
    return launch_pass_tc3_cols_swapped(P, L, my, mx, st);
  }
  launch_prep(P, L.n_pad, L.m_pad, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (before_main && (e = cudaEventRecordWithFlags(before_main, st, cudaEventRecordExternal)) != cudaSuccess) return e;
  if (L.v3 && !(md & (PASS_MAXCOST | PASS_OBJ))) {
    if (!make_map(&mx, P.X, P.n, P.d, P.ldx, 128) || !make_map(&my, P.Y, P.m, P.d, P.ldy, tc3_tile_cols()))
      return cudaErrorInvalidValue;
    return launch_pass_tc3(P, L, mx, my, st);
  }
  if (!make_map(&mx, P.X, P.n, P.d, P.ldx) || !make_map(&my, P.Y, P.m, P.d, P.ldy)) return cudaErrorInvalidValue;
  if (md & PASS_MAXCOST) return launch_mode<M_MAX>(P, L, mx, my, st);
  if (md & PASS_OBJ) return launch_mode<M_OBJ>(P, L, mx, my, st);
  if ((md & PASS_ROWS) && (md & PASS_COLS)) return launch_mode<M_RC>(P, L, mx, my, st);
  if (md & PASS_ROWS) return launch_mode<M_R>(P, L, mx, my, st);
  return launch_mode<M_C>(P, L, mx, my, st);
}

}  // namespace pot
