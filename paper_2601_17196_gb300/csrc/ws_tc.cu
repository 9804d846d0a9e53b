// tcgen05 path of the warm-start network (POT_WS_BF16).
//
// One persistent CTA of 128 threads per SM; thread p owns point p of a
// 128-point tile and TMEM lane p.  The three 128 x 128 x 128 contractions of
// a tile run on the tensor cores with BF16 operands and FP32 accumulators in
// TMEM; everything else (features, GELU, the output unit, the losses) is FP32
// on the CUDA cores.  Operands are written by the threads straight into the
// K-major, 128-byte-swizzled shared-memory layout the MMA descriptors name:
// row r of an operand is 256 bytes split into two 64-element slabs, and the
// 16-byte chunk c of a 128-byte slab row sits at chunk position c ^ (r & 7).
// A row of a "transposed" operand (points along K) is written one element
// per thread, 32 consecutive threads filling 64 contiguous bytes.
//
// Forward (pass 0):  A2 = H1 W2^T  -> y.
// Training pass A:   A2 = H1 W2^T  -> y, dy, D2 = dL/dA2
//                    dW2 += D2^T H1            (TMEM accumulator per CTA)
//                    per-tile sums: dq = 1^T D2, db3, loss; per-CTA dw3
// (the per-instance kernel turns dq into dctx_k / n_k)
// Training pass B:   A2 = H1 W2^T -> D2 again, dH1 = D2 W2,
//                    dA1 = (dH1 + dctx_k / n_k) GELU'(A1)
//                    [dW1 | db1]^T += dA1^T [X | 1]   (an N = 16 MMA)
// Every mbarrier wait is bounded (2 s); a wait that gives up raises the CTA's
// abort flag, the CTA leaves its tile loop, waits (bounded) for its own MMAs,
// frees its TMEM and sets the batch error flag, which the final reduction
// turns into a NaN loss and no parameter update.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "tc_common.cuh"
#include "ws_common.cuh"

namespace pot {
pot_status set_last_error(pot_status s, const char* msg);
namespace ws {

using namespace pot::tcx;

namespace {

constexpr int kThreads = 128;
constexpr uint32_t kSlab = 128 * 128;        // bytes of one 64-element slab of 128 rows
constexpr uint32_t kOp = 2 * kSlab;          // a 128 x 128 BF16 operand
constexpr uint32_t kSlabX = 16 * 128;        // one slab of a 16-row operand
constexpr uint32_t kOpX = 2 * kSlabX;
constexpr uint32_t kTmemCols = 256;

__device__ __forceinline__ uint32_t swz(int row, int k, uint32_t slab_bytes) {
  const int slab = k >> 6, ch = (k >> 3) & 7, e = k & 7;
  return slab * slab_bytes + row * 128 + ((uint32_t)(ch ^ (row & 7)) << 4) + (e << 1);
}
__device__ __forceinline__ uint32_t swz_chunk(int row, int c, uint32_t slab_bytes) {
  return (c >> 3) * slab_bytes + row * 128 + ((uint32_t)((c & 7) ^ (row & 7)) << 4);
}
__device__ __forceinline__ uint16_t bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack(float a, float b) { return (uint32_t)bf(a) | ((uint32_t)bf(b) << 16); }
__device__ __forceinline__ void st_chunk(unsigned char* base, uint32_t off, const float* h) {
  *reinterpret_cast<uint4*>(base + off) = make_uint4(pack(h[0], h[1]), pack(h[2], h[3]), pack(h[4], h[5]), pack(h[6], h[7]));
}
__device__ __forceinline__ void st_elem(unsigned char* base, uint32_t off, float x) {
  *reinterpret_cast<uint16_t*>(base + off) = bf(x);
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (+)= A B^T over K = 128: two slabs of four K = 16 steps.
__device__ __forceinline__ void mma_k128(uint32_t d, uint32_t a, uint32_t a_slab, uint32_t b, uint32_t b_slab,
                                         uint32_t idesc, bool accumulate) {
#pragma unroll
  for (int kb = 0; kb < 2; ++kb)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      umma_bf16(d, sdesc(a + kb * a_slab + kk * 32), sdesc(b + kb * b_slab + kk * 32), idesc,
                (accumulate || kb || kk) ? 1u : 0u);
}

// Bounded wait that ignores the abort flag (draining before TMEM is freed).
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = gtime();
  while (!mbar_try(bar, parity) && gtime() - t0 < kTimeoutNs) {}
}

struct Smem {
  static constexpr uint32_t misc = 4 * kOp + kOpX;
  static constexpr uint32_t floats = kTile * FMAX + H * FMAX + 4 * H + 2 * 4 * H + 8;
  static constexpr uint32_t bars = misc + floats * 4;
  static constexpr uint32_t total = bars + 8 * 4 + 16;
};

template <int PASS>   // 0 forward, 1 training pass A, 2 training pass B
__global__ void __launch_bounds__(kThreads, 1) ws_tc_kernel(WsArgs A) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sW2 = sm;
  unsigned char* sW2T = sm + kOp;                                 // pass B
  unsigned char* sT0 = sm + (PASS == 2 ? 2 : 1) * kOp;            // H1, then D2 in pass B
  unsigned char* sT1 = sm + (PASS == 2 ? 3 : 2) * kOp;            // H1^T (A) / dA1^T (B)
  unsigned char* sT2 = sm + 3 * kOp;                              // D2^T (A)
  unsigned char* sXT = sm + 4 * kOp;                              // [X | 1]^T (B), 16 rows
  float* xs = reinterpret_cast<float*>(sm + Smem::misc);
  float* W1s = xs + kTile * FMAX;
  float* b1s = W1s + H * FMAX;
  float* b2q = b1s + H;
  float* w3s = b2q + H;
  float* dcs = w3s + H;
  float* red = dcs + H;                                           // [2][4][H]
  float* wsm = red + 2 * 4 * H;                                   // [2][4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + Smem::bars);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 4);
  int* s_abort = reinterpret_cast<int*>(s_tmem + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int F = A.F;
  const Offs o = A.o;
  if (tid == 0) {
    for (int k = 0; k < 3; ++k) mbar_init(bars + k, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // BF16 operands of W2 (rows = output unit) and, for pass B, W2^T (rows = input unit)
  for (int e = tid; e < H * 16; e += kThreads) {
    const int row = e >> 4, c = e & 15;
    float h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = A.P[o.W2 + row * H + 8 * c + j];
    st_chunk(sW2, swz_chunk(row, c, kSlab), h);
    if (PASS == 2) {
#pragma unroll
      for (int j = 0; j < 8; ++j) h[j] = A.P[o.W2 + (8 * c + j) * H + row];
      st_chunk(sW2T, swz_chunk(row, c, kSlab), h);
    }
  }
  for (int e = tid; e < H * FMAX; e += kThreads) {
    const int k = e / FMAX, f = e % FMAX;
    W1s[e] = f < F ? A.P[o.W1 + k * F + f] : 0.f;
  }
  b1s[tid] = A.P[o.b1 + tid];
  w3s[tid] = A.P[o.w3 + tid];
  const float b3 = A.P[o.b3];
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t idesc = idesc_bf16(128, 128);
  const int p = tid;
  float gw3acc = 0.f;
  int n_g1 = 0, n_g2 = 0;      // products issued on barriers 0 and (pass B) 1

  int it = 0;
  for (int t = blockIdx.x; t < A.T; t += gridDim.x, ++it) {
    const WsTile tl = A.tiles[t];
    const int cnt = tl.count;
    const bool live = p < cnt;
    // the previous tile's last MMA reads operands this tile overwrites
    if (PASS == 1 && it > 0) mbar_wait(bars + 1, (it - 1) & 1, s_abort);
    if (PASS == 2 && it > 0) mbar_wait(bars + 2, (it - 1) & 1, s_abort);
    tc_fence_after();
    if (__syncthreads_or(*(volatile int*)s_abort)) break;
    for (int e = tid; e < kTile * FMAX; e += kThreads) {
      const int pp = e / FMAX, f = e % FMAX;
      xs[e] = (pp < cnt && f < F) ? A.feats[(tl.start + pp) * F + f] : 0.f;
    }
    b2q[tid] = A.P[o.b2 + tid] + A.q[(int64_t)tl.b * H + tid];
    if (PASS == 2) dcs[tid] = A.dctx[(int64_t)tl.b * H + tid];
    __syncthreads();
    float xp[FMAX];
#pragma unroll
    for (int f = 0; f < FMAX; ++f) xp[f] = xs[p * FMAX + f];
    // H1 row p (A of the first product); H1^T column p (pass A); [X | 1]^T column p (pass B)
#pragma unroll 1
    for (int c = 0; c < 16; ++c) {
      float h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = 8 * c + j;
        float a = b1s[k];
#pragma unroll
        for (int f = 0; f < FMAX; ++f) a = fmaf(W1s[k * FMAX + f], xp[f], a);
        h[j] = live ? gelu(a) : 0.f;
      }
      st_chunk(sT0, swz_chunk(p, c, kSlab), h);
      if (PASS == 1) {
#pragma unroll
        for (int j = 0; j < 8; ++j) st_elem(sT1, swz(8 * c + j, p, kSlab), h[j]);
      }
    }
    if (PASS == 2) {
#pragma unroll
      for (int f = 0; f < 16; ++f) {
        const float val = !live ? 0.f : (f < F ? xp[f] : (f == F ? 1.f : 0.f));
        st_elem(sXT, swz(f, p, kSlabX), val);
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      mma_k128(tmem, smem_u32(sT0), kSlab, smem_u32(sW2), kSlab, idesc, false);
      umma_commit(bars + 0);
    }
    ++n_g1;
    mbar_wait(bars + 0, it & 1, s_abort);
    tc_fence_after();
    if (__syncthreads_or(*(volatile int*)s_abort)) break;
    // sweep 1: y
    float y = 0.f;
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32];
      tmem_ld32(trow + ch * 32, v);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int oc = ch * 32 + j;
        y = fmaf(w3s[oc], gelu(v[j] + b2q[oc]), y);
      }
    }
    y += b3;
    if (PASS == 0) {
      if (live) A.y[tl.ybase + p] = y;
      tc_fence_before();
      continue;
    }
    const float dd = live ? y - A.target[tl.start + p] : 0.f;
    const float wt = live ? (A.weight ? A.weight[tl.start + p] : 1.f) : 0.f;
    const float dy = 2.f * wt * dd * A.invN;
    // sweep 2: D2 = dy w3 GELU'(A2)
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32], d2[32];
      tmem_ld32(trow + ch * 32, v);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int oc = ch * 32 + j;
        const float a2 = v[j] + b2q[oc];
        d2[j] = dy * w3s[oc] * gelu_grad(a2);
        v[j] = dy * gelu(a2);
      }
      if (PASS == 1) {
#pragma unroll
        for (int j = 0; j < 32; ++j) st_elem(sT2, swz(ch * 32 + j, p, kSlab), d2[j]);
        const float sw3 = transpose_reduce32(v, lane);
        const float sdq = transpose_reduce32(d2, lane);
        red[(0 * 4 + warp) * H + ch * 32 + lane] = sw3;
        red[(1 * 4 + warp) * H + ch * 32 + lane] = sdq;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) st_chunk(sT0, swz_chunk(p, ch * 4 + q, kSlab), d2 + 8 * q);
      }
    }
    if (PASS == 1) {
      const float sdy = warp_sum(dy), sl = warp_sum(wt * dd * dd * A.invN);
      if (lane == 0) { wsm[warp] = sdy; wsm[4 + warp] = sl; }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (PASS == 1) {
      if (tid == 0) {
        tc_fence_after();
        mma_k128(tmem + 128, smem_u32(sT2), kSlab, smem_u32(sT1), kSlab, idesc, it > 0);   // dW2 += D2^T H1
        umma_commit(bars + 1);
      }
      gw3acc += (red[0 * H + tid] + red[1 * H + tid]) + (red[2 * H + tid] + red[3 * H + tid]);
      A.dqp[(int64_t)t * H + tid] = (red[4 * H + tid] + red[5 * H + tid]) + (red[6 * H + tid] + red[7 * H + tid]);
      if (tid == 0) {
        A.gb3p[t] = (wsm[0] + wsm[1]) + (wsm[2] + wsm[3]);
        A.lossp[t] = (wsm[4] + wsm[5]) + (wsm[6] + wsm[7]);
      }
    } else {
      if (tid == 0) {
        tc_fence_after();
        mma_k128(tmem, smem_u32(sT0), kSlab, smem_u32(sW2T), kSlab, idesc, false);   // dH1 = D2 W2
        umma_commit(bars + 1);
      }
      ++n_g2;
      mbar_wait(bars + 1, it & 1, s_abort);
      tc_fence_after();
      if (__syncthreads_or(*(volatile int*)s_abort)) break;
#pragma unroll 1
      for (int ch = 0; ch < 4; ++ch) {
        float v[32];
        tmem_ld32(trow + ch * 32, v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int k = ch * 32 + j;
          float a = b1s[k];
#pragma unroll
          for (int f = 0; f < FMAX; ++f) a = fmaf(W1s[k * FMAX + f], xp[f], a);
          st_elem(sT1, swz(k, p, kSlab), live ? (v[j] + dcs[k]) * gelu_grad(a) : 0.f);
        }
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        mma_k128(tmem + 128, smem_u32(sT1), kSlab, smem_u32(sXT), kSlabX, idesc_bf16(128, 16), it > 0);
        umma_commit(bars + 2);
      }
    }
  }
  // drain this CTA's MMAs, write the per-CTA accumulators, free TMEM
  const int aborted = *(volatile int*)s_abort;
  if (n_g1 > 0) drain_wait(bars + 0, (n_g1 - 1) & 1);
  if (PASS == 1 && it > 0) drain_wait(bars + 1, (it - 1) & 1);
  if (PASS == 2 && n_g2 > 0) drain_wait(bars + 1, (n_g2 - 1) & 1);
  if (PASS == 2 && it > 0) drain_wait(bars + 2, (it - 1) & 1);
  tc_fence_after();
  if (PASS == 1) {
    float* out = A.gW2p + (int64_t)blockIdx.x * H * H + (int64_t)tid * H;
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32];
      tmem_ld32(trow + 128 + ch * 32, v);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) out[ch * 32 + j] = it > 0 ? v[j] : 0.f;
    }
    A.gw3p[(int64_t)blockIdx.x * H + tid] = gw3acc;
  }
  if (PASS == 2) {
    float v[32];
    tmem_ld32(trow + 128, v);
    tmem_wait_ld();
    const int64_t base = (int64_t)blockIdx.x * H + tid;
    for (int f = 0; f < F; ++f) A.gW1p[base * F + f] = it > 0 ? v[f] : 0.f;
    A.gb1p[base] = it > 0 ? v[F] : 0.f;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  if (tid == 0 && aborted) atomicExch(A.err, 1);
}

// Per instance: dq = sum of D2 over its tiles, dctx / n_k = (U^T dq)[:H] / n_k.
__global__ void __launch_bounds__(H) ws_dctx_kernel(WsArgs A) {
  __shared__ float dqs[H];
  const int b = blockIdx.x, k = threadIdx.x;
  const WsInst I = A.binfo[b];
  float s = 0.f;
  for (int t = I.tile0; t < I.tile0 + I.ntiles; ++t) s += A.dqp[(int64_t)t * H + k];
  dqs[k] = s;
  A.dq[(int64_t)b * H + k] = s;
  __syncthreads();
  float dc = 0.f;
  for (int oc = 0; oc < H; ++oc) dc = fmaf(A.P[A.o.U + (int64_t)oc * (H + 2) + k], dqs[oc], dc);
  A.dctx[(int64_t)b * H + k] = dc / I.npts;
}

template <int PASS>
pot_status launch(const WsArgs& A, cudaStream_t st) {
  const size_t smem = Smem::total + 1024;
  cudaError_t e = cudaFuncSetAttribute(ws_tc_kernel<PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return set_last_error(POT_ECUDA, "cudaFuncSetAttribute failed for the tcgen05 network kernel");
  ws_tc_kernel<PASS><<<(unsigned)A.G, kThreads, smem, st>>>(A);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_last_error(POT_ECUDA, cudaGetErrorString(e));
  return POT_OK;
}

}  // namespace

pot_status launch_ws_main_tc(const WsArgs& A, bool train, cudaStream_t st) {
  if (cudaMemsetAsync(A.err, 0, sizeof(int), st) != cudaSuccess)
    return set_last_error(POT_ECUDA, "cudaMemsetAsync of the error flag failed");
  pot_status s;
  if (!train) return launch<0>(A, st);
  if ((s = launch<1>(A, st)) != POT_OK) return s;
  ws_dctx_kernel<<<(unsigned)A.B, H, 0, st>>>(A);
  return launch<2>(A, st);
}

}  // namespace ws
}  // namespace pot
