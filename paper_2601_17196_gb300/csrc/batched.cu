// Batched ASPOT: many independent POT instances of uneven size solved in
// lockstep (the same iteration t for every instance still running).
//
// Rows and columns of all instances are concatenated; each O(nm) pass is ONE
// launch over a work list of (instance, row block, column block) tiles of the
// CUDA-core pass (squared-Euclidean costs of low-dimensional points, d <= 4),
// followed by the wide partial combine.  The O(n+m) updates of Algorithm 2 run
// with one CTA per instance, so every scalar reduction is a deterministic
// block reduction.  A converged instance sets its own done flag; its tiles and
// its update kernels return at once, and the solve ends when all are done.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>
#include <math.h>
#include <stddef.h>
#include <string>
#include <vector>
#include <algorithm>
#include <map>
#include <mutex>
#include <nvtx3/nvToolsExt.h>

#include "../../include/aspot.h"
#include "common.cuh"
#include "kernels.h"
#include "simt_tile.cuh"
#include "inst_body.cuh"

namespace pot {
pot_status set_last_error(pot_status s, const char* msg);
}

using namespace pot;
using namespace pot::simt;
using namespace pot::inst;

namespace {

constexpr int kBT = 512;       // threads of a per-instance CTA
constexpr int kH = 256;        // default rows of a batched tile (8 warps x 8 chunks of 4 rows)
constexpr int kW = 256;        // default columns of a batched tile

// masses, minima and finiteness of r and c per instance
__global__ void b_stats_kernel(BVecs V) {
  BInst& I = V.inst[blockIdx.x];
  double v[3] = {0, 0, 0};
  double mr = INFINITY, mc = INFINITY;
  for (int64_t i = threadIdx.x; i < I.n; i += kBT) {
    const double x = I.r[i];
    v[0] += x; mr = fmin(mr, x);
    if (!(x >= 0.0) || !isfinite(x)) v[2] = 1.0;
  }
  for (int64_t j = threadIdx.x; j < I.m; j += kBT) {
    const double x = I.c[j];
    v[1] += x; mc = fmin(mc, x);
    if (!(x >= 0.0) || !isfinite(x)) v[2] = 1.0;
  }
  double w[2] = {-mr, -mc};
  block_sums<3>(v);
  __shared__ double smn[2][kBT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    double x = w[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) smn[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = -INFINITY, b = -INFINITY;
    for (int q = 0; q < kBT / 32; ++q) { a = fmax(a, smn[0][q]); b = fmax(b, smn[1][q]); }
    I.mass_r = v[0]; I.mass_c = v[1]; I.bad = v[2]; I.min_r = -a; I.min_c = -b;
  }
}

// largest raw cost per instance from the per-tile maxima
__global__ void b_max_kernel(BInst* inst, const double* red) {
  BInst& I = inst[blockIdx.x];
  double mx = 0.0;
  for (int64_t k = threadIdx.x; k < I.ntile; k += kBT) mx = fmax(mx, red[I.tile0 + k]);
  __shared__ double sm[kBT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < kBT / 32; ++q) a = fmax(a, sm[q]);
    I.maxc = a;
  }
}

// Algorithm 2 setup per instance: smoothed marginals, zero start
__global__ void b_init_kernel(BVecs V) {
  BInst& I = V.inst[blockIdx.x];
  const double e = I.eps_s;
  for (int64_t i = threadIdx.x; i < I.n; i += kBT) {
    const int64_t g = I.row0 + i;
    const double x = (1.0 - e / 8.0) * I.r[i] + e / (8.0 * (double)I.n);
    V.rt[g] = x; V.lrt[g] = x > 0.0 ? log(x) : POT_NEG_BIG;
    V.ut[g] = 0.0; V.uc[g] = 0.0; I.pu[i] = 0.0;
  }
  for (int64_t j = threadIdx.x; j < I.m; j += kBT) {
    const int64_t g = I.col0 + j;
    const double x = (1.0 - e / 8.0) * I.c[j] + e / (8.0 * (double)I.m);
    V.ct[g] = x; V.lct[g] = x > 0.0 ? log(x) : POT_NEG_BIG;
    V.vt[g] = 0.0; V.vc[g] = 0.0; I.pv[j] = 0.0;
  }
  if (threadIdx.x == 0) {
    I.w_tilde = 0.0; I.w_check = 0.0; I.w_out = 0.0; I.w_z = 0.0;
    I.theta = 1.0; I.t = 0; I.done = 0; I.take_hat = 0; I.nonfinite = 0; I.E = INFINITY;
  }
}

__global__ void b_extrap_kernel(BVecs V) {
  BlockTeam tm;
  b_extrap_body(V, blockIdx.x, tm);
}


// ------------------------------------------------- fused batched sweep ---
// One launch per pass of the iteration: a persistent grid walks the tile work
// list (CTA b takes tiles b, b + G, ...); after a tile, the CTA takes a
// ticket on the tile's instance, and the CTA that completes the instance's
// last tile runs, for that instance alone, what used to be separate launches:
// the combine of its partials into FP64 log-sums, its update (gradient step,
// Greenkhorn step and argmin, or the final step with E_t and the stop test;
// the greedy rule's counterparts), the extrapolation for the next iteration
// and the per-pass terms of the next pass.  An iteration is three launches.


template <int KIND, int VV, int MT>
__global__ void __launch_bounds__(kThreads, 2) b_sweep_kernel(BatchPass B, BVecs V, int epi, int k) {
  // Tiles are handed out by an atomic counter (a CTA busy with an instance's
  // update does not hold up any tiles); a finished instance's remaining
  // tiles are skipped in one step.  The last CTA to leave resets the counter.
  __shared__ int s_last, s_tau;
  int* const ctr = V.ndone + 1;
  int* const exits = V.ndone + 2;
  const int ntiles = (int)B.ntiles;
  while (true) {
    if (threadIdx.x == 0) {
      int t;
      while (true) {
        t = atomicAdd(ctr, 1);
        if (t >= ntiles) break;
        const BInst* Ii = B.inst + B.tiles[t].inst;
        if (!*(volatile const int*)&Ii->done) break;
        atomicMax(ctr, (int)(Ii->tile0 + Ii->ntile));   // the rest of a finished instance
      }
      s_tau = t;
    }
    __syncthreads();
    const int tau = s_tau;
    if (tau >= ntiles) break;
    const BTile tl = B.tiles[tau];
    BInst* I = B.inst + tl.inst;
    PassDesc P{};
    P.n = I->n; P.m = I->m; P.kind = KIND;
    P.X = I->X; P.Y = I->Y; P.d = I->d; P.ldx = I->ldx; P.ldy = I->ldy;
    P.xn = B.xn + I->row0; P.yn = B.yn + I->col0;
    P.gC = I->gC;
    P.mode = B.mode;
    P.row_part = B.row_part + I->row0;
    P.col_part = B.col_part + I->col0;
    P.red_part = B.red_part;
    P.kappa = &I->kappa;
    P.rowA = B.rowA + I->row0;
    P.colA = B.colA + I->col0;
    P.colB = B.colB + I->col0;
    simt_tile<KIND, VV, 4, false, MT>(P, B.H, tl.cb, tl.rb, B.Ntot, B.Mtot, tau);
    __threadfence();                             // this tile's partials, before the ticket
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&I->ticket, 1) == I->ntile - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      if (threadIdx.x == 0) I->ticket = 0;
      BlockTeam tm;
      b_epilogue(B, V, tl.inst, epi, k, tm);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(exits, 1) == (int)gridDim.x - 1) { *ctr = 0; *exits = 0; }
  }
}

template <int VV, int MT>
cudaError_t launch_sweep_vm(const BatchPass& B, const BVecs& V, int epi, int k, cudaStream_t st) {
  static int grid[4] = {0, 0, 0, 0};
  auto kern = (B.kind == COST_SQEUCLID_BF16) ? b_sweep_kernel<COST_SQEUCLID_BF16, VV, MT>
            : (B.kind == COST_SQEUCLID_F16) ? b_sweep_kernel<COST_SQEUCLID_F16, VV, MT>
                                             : b_sweep_kernel<COST_SQEUCLID_F32, VV, MT>;
  const int slot = B.kind & 3;
  if (grid[slot] == 0) {
    int per = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, 0) != cudaSuccess || per < 1) per = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) sms = 152;
    grid[slot] = per * sms;
  }
  const int64_t g = B.ntiles < grid[slot] ? B.ntiles : grid[slot];
  kern<<<(unsigned)g, kThreads, 0, st>>>(B, V, epi, k);
  return cudaGetLastError();
}

// one fused pass of the batched iteration (rows + columns, rows, or columns)
cudaError_t launch_sweep(const BatchPass& B, const BVecs& V, int epi, int k, cudaStream_t st) {
  const int mt = (B.mode == (PASS_ROWS | PASS_COLS)) ? 1 : (B.mode == PASS_ROWS ? 2 : 3);
  if (B.W == 128) {
    if (mt == 1) return launch_sweep_vm<1, 1>(B, V, epi, k, st);
    if (mt == 2) return launch_sweep_vm<1, 2>(B, V, epi, k, st);
    return launch_sweep_vm<1, 3>(B, V, epi, k, st);
  }
  if (mt == 1) return launch_sweep_vm<2, 1>(B, V, epi, k, st);
  if (mt == 2) return launch_sweep_vm<2, 2>(B, V, epi, k, st);
  return launch_sweep_vm<2, 3>(B, V, epi, k, st);
}

// rounding reading R1-R4, per instance (original r, c, s)
__global__ void b_round1_kernel(BVecs V) {
  BInst& I = V.inst[blockIdx.x];
  for (int64_t i = threadIdx.x; i < I.n; i += kBT) {
    const double lr = I.r[i] > 0.0 ? log(I.r[i]) : POT_NEG_BIG;
    const double f = clampl(I.pu[i] + I.w_out + fmin(0.0, lr - V.lrow[I.row0 + i]));
    I.pf[i] = f;
    V.fc[I.row0 + i] = f;
  }
}
__global__ void b_round2_kernel(BVecs V) {
  BInst& I = V.inst[blockIdx.x];
  double v[2] = {0, 0};
  for (int64_t j = threadIdx.x; j < I.m; j += kBT) {
    const double Cc = V.lcol[I.col0 + j];
    const double lc = I.c[j] > 0.0 ? log(I.c[j]) : POT_NEG_BIG;
    const double lb = fmin(0.0, lc - Cc);
    const double gj = clampl(I.pv[j] + lb);
    I.pg[j] = gj;
    V.gc[I.col0 + j] = gj;
    const double cm = sexp(Cc + lb);
    const double qj = fmax(I.c[j] - cm, 0.0);
    I.pq[j] = qj;
    V.vh[I.col0 + j] = qj;
    v[0] += cm;
    v[1] += qj;
  }
  block_sums<2>(v);
  if (threadIdx.x == 0) { I.m2 = v[0]; I.sum_q = v[1]; }
}
// after the row pass at (f, g): R3 (uniform scale) or R4 (rank-one fill)
__global__ void b_round34_kernel(BVecs V) {
  BInst& I = V.inst[blockIdx.x];
  const bool r3 = I.m2 >= I.s;
  double v[1] = {0};
  if (r3) {
    const double lk = log(I.s / I.m2);
    for (int64_t i = threadIdx.x; i < I.n; i += kBT) {
      const double f = clampl(I.pf[i] + lk);
      I.pf[i] = f; V.fc[I.row0 + i] = f;
      I.pp[i] = 0.0; V.uh[I.row0 + i] = 0.0;
    }
    for (int64_t j = threadIdx.x; j < I.m; j += kBT) { I.pq[j] = 0.0; V.vh[I.col0 + j] = 0.0; }
  } else {
    for (int64_t i = threadIdx.x; i < I.n; i += kBT) {
      const double pi = fmax(I.r[i] - sexp(V.lrow[I.row0 + i]), 0.0);
      I.pp[i] = pi;
      V.uh[I.row0 + i] = pi;
      v[0] += pi;
    }
  }
  block_sums<1>(v);
  if (threadIdx.x == 0) {
    const double den = v[0] * I.sum_q;
    I.kappa = r3 ? 0.0 : (den > 0.0 ? (I.s - I.m2) / den : 0.0);
    I.branch = r3 ? 3 : 4;
    *I.pkappa = I.kappa;
    *I.pw = I.w_out;
  }
}
__global__ void b_obj_kernel(BInst* inst, const double* red) {
  BInst& I = inst[blockIdx.x];
  double v[1] = {0};
  for (int64_t k = threadIdx.x; k < I.ntile; k += kBT) v[0] += red[I.tile0 + k];
  block_sums<1>(v);
  if (threadIdx.x == 0) I.obj = v[0] * I.cost_scale;
}
__global__ void b_sqnorm_kernel(BInst* inst, float* xn, float* yn) {
  BInst& I = inst[blockIdx.x];
  for (int64_t i = threadIdx.x; i < I.n + I.m; i += kBT) {
    const bool row = i < I.n;
    const int64_t k = row ? i : i - I.n;
    const void* P = row ? I.X : I.Y;
    const int64_t ld = row ? I.ldx : I.ldy;
    float acc = 0.f;
    for (int t = 0; t < I.d; ++t) {
      float x;
      if (I.kind == COST_SQEUCLID_BF16) x = __uint_as_float(((unsigned)reinterpret_cast<const unsigned short*>(P)[k * ld + t]) << 16);
      else if (I.kind == COST_SQEUCLID_F16) x = __half2float(reinterpret_cast<const __half*>(P)[k * ld + t]);
      else x = reinterpret_cast<const float*>(P)[k * ld + t];
      acc = fmaf(x, x, acc);
    }
    if (row) xn[I.row0 + k] = acc; else yn[I.col0 + k] = acc;
  }
}
__global__ void b_clear_kernel(float2* a, int64_t na, float2* b, int64_t nb) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < na) a[t] = make_float2(POT_NEG_BIGF, 0.f);
  else if (t < na + nb) b[t - na] = make_float2(POT_NEG_BIGF, 0.f);
}

// ----------------------------------------------------------------- host ---

// Tile geometry of the batched pass: H rows x W columns per CTA, the work
// list in instance order, and the partial strides the combines read.
struct Geom {
  int H = kH, W = kW;
  int64_t T = 0, maxcb = 0, maxrb = 0;
  std::vector<BTile> tiles;
  std::vector<int64_t> tile0, ntile;
};

Geom b_geom(const pot_problem* P, int count, int H, int W) {
  Geom G;
  G.H = H; G.W = W;
  G.tile0.resize(count); G.ntile.resize(count);
  // instances in order of decreasing size, so the largest per-instance
  // updates of a fused sweep start early; each instance's tiles stay contiguous
  std::vector<int> order(count);
  for (int k = 0; k < count; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P[a].n * P[a].m > P[b].n * P[b].m; });
  for (int k : order) {
    const int64_t nrb = (P[k].n + H - 1) / H, ncb = (P[k].m + W - 1) / W;
    G.tile0[k] = G.T; G.ntile[k] = nrb * ncb;
    G.T += nrb * ncb;
    G.maxcb = std::max(G.maxcb, ncb); G.maxrb = std::max(G.maxrb, nrb);
    for (int64_t rb = 0; rb < nrb; ++rb)
      for (int64_t cb = 0; cb < ncb; ++cb) G.tiles.push_back(BTile{k, (int32_t)rb, (int32_t)cb, 0});
  }
  return G;
}

// Candidate tile shapes of the autotuner (rows a multiple of 32: eight warps
// of four-row chunks; columns 128 or 256: one or two float4 groups per lane).
// The smallest of each dimension bounds every workspace region.
constexpr int kCandH[] = {32, 64, 128, 256};
constexpr int kCandW[] = {128, 256};
constexpr int kMinH = 32, kMinW = 128;

struct BLayout {
  int64_t N = 0, M = 0, T = 0, maxcb = 0, maxrb = 0;   // worst case over the candidate shapes
  size_t off_inst, off_tiles, off_cnt, off_xn, off_yn, off_rowp, off_colp, off_red, off_u[16], off_v[16], total;
  size_t off_trace;
  size_t off_rowA, off_colA, off_colB;
};

size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr int kBSlots = 10;   // rt lrt ut uc ub ug uh lrow + spare

BLayout b_layout(const pot_problem* P, int count) {
  BLayout L;
  for (int k = 0; k < count; ++k) {
    const int64_t nrb = (P[k].n + kMinH - 1) / kMinH, ncb = (P[k].m + kMinW - 1) / kMinW;
    L.N += P[k].n; L.M += P[k].m; L.T += nrb * ncb;
    L.maxcb = std::max(L.maxcb, ncb); L.maxrb = std::max(L.maxrb, nrb);
  }
  size_t o = 0;
  L.off_inst = o; o = al(o + sizeof(BInst) * count);
  L.off_tiles = o; o = al(o + sizeof(BTile) * L.T);
  L.off_cnt = o; o = al(o + 64);
  L.off_xn = o; o = al(o + sizeof(float) * L.N);
  L.off_yn = o; o = al(o + sizeof(float) * L.M);
  L.off_rowp = o; o = al(o + sizeof(float2) * L.maxcb * L.N);
  L.off_colp = o; o = al(o + sizeof(float2) * L.maxrb * L.M);
  L.off_red = o; o = al(o + sizeof(double) * (L.T + 1));
  L.off_rowA = o; o = al(o + sizeof(float4) * L.N);
  L.off_colA = o; o = al(o + sizeof(float2) * L.M);
  L.off_colB = o; o = al(o + sizeof(float2) * L.M);
  for (int s = 0; s < kBSlots; ++s) { L.off_u[s] = o; o = al(o + sizeof(double) * L.N); }
  for (int s = 0; s < kBSlots; ++s) { L.off_v[s] = o; o = al(o + sizeof(double) * L.M); }
  L.off_trace = o; o = al(o + (size_t)kBTrace * count);
  L.total = o;
  return L;
}

pot_status bfail(pot_status s, const char* msg) { return set_last_error(s, msg); }

// ---------------------------------------------------------- autotuner ---
// Tile shapes chosen per batch signature (cost kind, largest d, number of
// instances, total and largest n and m), kept for the process; save / load
// write them as text lines "signature H W".
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;

std::string batch_signature(const pot_problem* P, int count) {
  int64_t N = 0, M = 0, nmax = 0, mmax = 0;
  int dmax = 0;
  for (int k = 0; k < count; ++k) {
    N += P[k].n; M += P[k].m;
    nmax = std::max<int64_t>(nmax, P[k].n); mmax = std::max<int64_t>(mmax, P[k].m);
    dmax = std::max<int>(dmax, P[k].d);
  }
  char b[160];
  snprintf(b, sizeof(b), "k%d_d%d_c%d_N%lld_M%lld_n%lld_m%lld", (int)P[0].kind, dmax, count, (long long)N,
           (long long)M, (long long)nmax, (long long)mmax);
  return b;
}

bool valid_shape(int H, int W) {
  bool h = false, w = false;
  for (int x : kCandH) h |= (x == H);
  for (int x : kCandW) w |= (x == W);
  return h && w;
}

pot_status check_batch(const pot_problem* probs, int32_t count) {
  if (!probs || count < 1) return bfail(POT_EINVAL, "batched: probs must be a host array of count >= 1 problems");
  for (int k = 0; k < count; ++k) {
    const pot_problem& p = probs[k];
    if (p.n < 1 || p.m < 1 || p.n > (1 << 24) || p.m > (1 << 24)) return bfail(POT_EINVAL, "batched: bad n or m");
    if (p.kind != POT_COST_SQEUCLID_F32 && p.kind != POT_COST_SQEUCLID_BF16 && p.kind != POT_COST_SQEUCLID_F16)
      return bfail(POT_EINVAL, "batched: only squared-Euclidean point clouds are batched");
    if (p.kind != probs[0].kind) return bfail(POT_EINVAL, "batched: all instances must share one cost kind");
    if (p.d < 1 || p.d > 4) return bfail(POT_EINVAL, "batched: point dimension must be 1..4");
    if (!p.X || !p.Y || !p.r || !p.c) return bfail(POT_EINVAL, "batched: NULL pointer in a problem");
    if (p.ldx < p.d || p.ldy < p.d) return bfail(POT_EINVAL, "batched: ldx, ldy must be >= d");
    if (!(p.s > 0.0) || !isfinite(p.s)) return bfail(POT_EINVAL, "batched: s must be finite and > 0");
    if (!(p.cost_scale >= 0.0) || !isfinite(p.cost_scale)) return bfail(POT_EINVAL, "batched: bad cost_scale");
  }
  return POT_OK;
}

#define BCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      char b_[256];                                                                       \
      snprintf(b_, sizeof(b_), "batched: %s: %s", #call, cudaGetErrorString(e_));         \
      return bfail(POT_ECUDA, b_);                                                        \
    }                                                                                     \
  } while (0)

}  // namespace

extern "C" {

POT_API pot_status pot_workspace_size_batched(const pot_problem* probs, int32_t count, size_t* bytes) {
  pot_status s = check_batch(probs, count);
  if (s != POT_OK) return s;
  if (!bytes) return bfail(POT_EINVAL, "bytes is NULL");
  *bytes = b_layout(probs, count).total;
  return POT_OK;
}

POT_API pot_status pot_trace_batched(void* workspace, const pot_problem* probs, int32_t count, int32_t iters,
                                     uint8_t* out, void* stream) {
  pot_status s = check_batch(probs, count);
  if (s != POT_OK) return s;
  if (!workspace || !out) return bfail(POT_EINVAL, "trace: workspace and out must not be NULL");
  if (iters < 0 || iters > kBTrace) return bfail(POT_EINVAL, "trace: iters must be in 0 .. 1024");
  if (iters == 0) return POT_OK;
  const BLayout L = b_layout(probs, count);
  const unsigned char* src = (const unsigned char*)workspace + L.off_trace;
  BCK(cudaMemcpy2DAsync(out, (size_t)iters, src, (size_t)kBTrace, (size_t)iters, (size_t)count,
                        cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  BCK(cudaStreamSynchronize((cudaStream_t)stream));
  return POT_OK;
}

POT_API pot_status pot_autotune_set(const pot_problem* probs, int32_t count, int32_t tile_rows, int32_t tile_cols) {
  pot_status s = check_batch(probs, count);
  if (s != POT_OK) return s;
  if (!valid_shape(tile_rows, tile_cols))
    return bfail(POT_EINVAL, "autotune: tile_rows must be 32, 64, 128 or 256 and tile_cols 128 or 256");
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[batch_signature(probs, count)] = {tile_rows, tile_cols};
  return POT_OK;
}

POT_API pot_status pot_autotune_lookup(const pot_problem* probs, int32_t count, int32_t* tile_rows,
                                       int32_t* tile_cols) {
  pot_status s = check_batch(probs, count);
  if (s != POT_OK) return s;
  if (!tile_rows || !tile_cols) return bfail(POT_EINVAL, "autotune: NULL output");
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find(batch_signature(probs, count));
  if (it == g_tune.end()) { *tile_rows = 0; *tile_cols = 0; return POT_OK; }
  *tile_rows = it->second.first; *tile_cols = it->second.second;
  return POT_OK;
}

POT_API pot_status pot_autotune_clear(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune.clear();
  return POT_OK;
}

POT_API pot_status pot_autotune_save(const char* path) {
  if (!path) return bfail(POT_EINVAL, "autotune: path is NULL");
  std::lock_guard<std::mutex> g(g_tune_mu);
  FILE* f = fopen(path, "w");
  if (!f) return bfail(POT_EINVAL, "autotune: cannot open the file for writing");
  for (const auto& e : g_tune) fprintf(f, "%s %d %d\n", e.first.c_str(), e.second.first, e.second.second);
  const bool ok = fclose(f) == 0;
  return ok ? POT_OK : bfail(POT_EINVAL, "autotune: write failed");
}

POT_API pot_status pot_autotune_load(const char* path) {
  if (!path) return bfail(POT_EINVAL, "autotune: path is NULL");
  FILE* f = fopen(path, "r");
  if (!f) return bfail(POT_EINVAL, "autotune: cannot open the file");
  std::map<std::string, std::pair<int, int>> got;
  char key[160];
  int H = 0, W = 0, r;
  while ((r = fscanf(f, "%159s %d %d", key, &H, &W)) == 3) {
    if (!valid_shape(H, W)) { fclose(f); return bfail(POT_EINVAL, "autotune: bad tile shape in the file"); }
    got[key] = {H, W};
  }
  fclose(f);
  if (r != EOF) return bfail(POT_EINVAL, "autotune: malformed line in the file");
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (const auto& e : got) g_tune[e.first] = e.second;
  return POT_OK;
}

POT_API pot_status aspot_solve_batched(const pot_problem* probs, int32_t count, const pot_params* params,
                                       void* workspace, size_t ws_bytes, pot_plan* plans, pot_result* res,
                                       void* stream) {
  pot_status s = check_batch(probs, count);
  if (s != POT_OK) return s;
  if (!params || !(params->eps > 0.0) || params->max_iter < 1 || !isfinite(params->gamma))
    return bfail(POT_EINVAL, "batched: bad params");
  // NVTX range over the whole call (no effect without an attached profiler)
  struct Range {
    Range() { nvtxRangePushA("aspot_solve_batched"); }
    ~Range() { nvtxRangePop(); }
  } range_all;
  if (params->block_rule != 0 && params->block_rule != 1)
    return bfail(POT_EINVAL, "batched: block_rule must be 0 (cyclic) or 1 (greedy)");
  if (params->resume) return bfail(POT_EINVAL, "batched: resume applies to single ASPOT solves only");
  const bool greedy = params->block_rule == 1;
  if (!plans || !res) return bfail(POT_EINVAL, "batched: plans and results must be host arrays of count entries");
  for (int k = 0; k < count; ++k) {
    const pot_plan& pl = plans[k];
    if (!pl.u || !pl.v || !pl.w || !pl.f || !pl.g || !pl.p || !pl.q || !pl.kappa)
      return bfail(POT_EINVAL, "batched: every plan pointer must be a device buffer");
  }
  if (!workspace || (uintptr_t)workspace % 256) return bfail(POT_EINVAL, "batched: workspace NULL or not 256-byte aligned");
  {
    // the solve synchronises its stream (setup, tuning, stop polling): no caller capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      return bfail(POT_EINVAL, "batched: the stream is being captured");
  }
  const BLayout L = b_layout(probs, count);
  if (ws_bytes < L.total) return bfail(POT_ENOMEM, "batched: workspace too small");
  Geom G = b_geom(probs, count, kH, kW);
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  BInst* dinst = (BInst*)(ws + L.off_inst);
  BTile* dtiles = (BTile*)(ws + L.off_tiles);
  int* ndone = (int*)(ws + L.off_cnt);
  float* xn = (float*)(ws + L.off_xn);
  float* yn = (float*)(ws + L.off_yn);
  float2* rowp = (float2*)(ws + L.off_rowp);
  float2* colp = (float2*)(ws + L.off_colp);
  double* red = (double*)(ws + L.off_red);
  double* U[kBSlots];
  double* Vv[kBSlots];
  for (int q = 0; q < kBSlots; ++q) { U[q] = (double*)(ws + L.off_u[q]); Vv[q] = (double*)(ws + L.off_v[q]); }

  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  BCK(cudaEventRecord(e0, st));

  // instance table
  std::vector<BInst> hi(count);
  int64_t r0 = 0, c0 = 0;
  for (int k = 0; k < count; ++k) {
    const pot_problem& p = probs[k];
    BInst& I = hi[k];
    memset(&I, 0, sizeof(I));
    I.n = p.n; I.m = p.m; I.row0 = r0; I.col0 = c0;
    I.tile0 = G.tile0[k]; I.ntile = G.ntile[k];
    I.X = p.X; I.Y = p.Y; I.d = p.d; I.kind = p.kind; I.ldx = p.ldx; I.ldy = p.ldy;
    I.r = p.r; I.c = p.c; I.s = p.s; I.cost_scale = p.cost_scale;
    I.max_iter = params->max_iter;
    I.pu = plans[k].u; I.pv = plans[k].v; I.pw = plans[k].w; I.pf = plans[k].f; I.pg = plans[k].g;
    I.pp = plans[k].p; I.pq = plans[k].q; I.pkappa = plans[k].kappa;
    r0 += p.n; c0 += p.m;
  }
  BCK(cudaMemcpyAsync(dinst, hi.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(dtiles, G.tiles.data(), sizeof(BTile) * G.T, cudaMemcpyHostToDevice, st));
  BCK(cudaMemsetAsync(ndone, 0, 64, st));

  BVecs V{};
  V.inst = dinst;
  V.rt = U[0]; V.lrt = U[1]; V.ut = U[2]; V.uc = U[3]; V.ub = U[4]; V.ug = U[5]; V.uh = U[6];
  V.ct = Vv[0]; V.lct = Vv[1]; V.vt = Vv[2]; V.vc = Vv[3]; V.vb = Vv[4]; V.vg = Vv[5]; V.vh = Vv[6];
  double* lrow = U[7];
  double* lcol = Vv[7];
  V.lrow = lrow; V.lcol = lcol; V.ndone = ndone;
  V.uo = U[8]; V.vo = Vv[8]; V.fc = U[9]; V.gc = Vv[9];
  V.trace = (unsigned char*)(ws + L.off_trace);
  V.trace4 = nullptr;

  BatchPass B{};
  B.kind = probs[0].kind; B.H = G.H; B.W = G.W; B.Ntot = L.N; B.Mtot = L.M; B.tiles = dtiles; B.ntiles = G.T;
  B.inst = dinst;
  B.xn = xn; B.yn = yn; B.row_part = rowp; B.col_part = colp; B.red_part = red; B.aoff0 = -1; B.aoff1 = -1;
  B.count = count;
  B.rowA = (float4*)(ws + L.off_rowA); B.colA = (float2*)(ws + L.off_colA); B.colB = (float2*)(ws + L.off_colB);
  int64_t launches = 0;
  bool in_loop = false;
  auto pass = [&](int mode, const double* a0, const double* b0, int w0, const double* a1, const double* b1, int w1,
                  int use_sel) -> pot_status {
    BatchPass q = B;
    q.check_done = in_loop ? 1 : 0;
    q.mode = mode; q.arow0 = a0; q.bcol0 = b0; q.aoff0 = w0; q.arow1 = a1; q.bcol1 = b1; q.aoff1 = w1;
    q.use_sel = use_sel;
    if (mode & (PASS_ROWS | PASS_COLS)) {
      const int64_t na = (mode & PASS_ROWS) ? G.maxcb * L.N : 0, nb = (mode & PASS_COLS) ? G.maxrb * L.M : 0;
      b_clear_kernel<<<(unsigned)((na + nb + 255) / 256), 256, 0, st>>>(rowp, na, colp, nb);
      ++launches;
    }
    if (mode & (PASS_ROWS | PASS_COLS | PASS_OBJ)) {
      launch_prep_batched(q, st);
      ++launches;
    }
    launch_pass_simt_batched(q, st);
    ++launches;
    if (mode & (PASS_ROWS | PASS_COLS)) {
      launch_combine(rowp, G.maxcb, L.N, (mode & PASS_ROWS) ? lrow : nullptr, colp, G.maxrb, L.M,
                     (mode & PASS_COLS) ? lcol : nullptr, nullptr, st);
      ++launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(POT_ECUDA, cudaGetErrorString(e));
    return POT_OK;
  };

  // prologue: masses, squared norms, largest cost of every instance
  b_stats_kernel<<<count, kBT, 0, st>>>(V);
  b_sqnorm_kernel<<<count, kBT, 0, st>>>(dinst, xn, yn);
  launches += 2;
  if ((s = pass(PASS_MAXCOST, nullptr, nullptr, -1, nullptr, nullptr, -1, 0)) != POT_OK) return s;
  b_max_kernel<<<count, kBT, 0, st>>>(dinst, red);
  ++launches;
  BCK(cudaMemcpyAsync(hi.data(), dinst, sizeof(BInst) * count, cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  // Algorithm 2 setup per instance (host, FP64)
  for (int k = 0; k < count; ++k) {
    BInst& I = hi[k];
    if (I.bad != 0.0) return bfail(POT_EINVAL, "batched: r and c must be finite and non-negative");
    if (!(I.mass_r > 0.0) || !(I.mass_c > 0.0)) return bfail(POT_EINVAL, "batched: r and c must have positive mass");
    if (I.s > std::min(I.mass_r, I.mass_c) * (1.0 + 1e-12)) return bfail(POT_EINVAL, "batched: s exceeds a mass");
    I.cost_scale = I.cost_scale > 0.0 ? I.cost_scale : (I.maxc > 0.0 ? 1.0 / I.maxc : 1.0);
    const double nn = (double)std::max(I.n, I.m);
    const double gamma = params->gamma > 0.0 ? params->gamma : params->eps / (4.0 * log(std::max(nn, 2.0)));
    I.gC = I.cost_scale / gamma;
    const double cmax = I.cost_scale * I.maxc;
    double thr = params->eps / (8.0 * (cmax > 0.0 ? cmax : 1.0));
    double e = thr;
    if (I.mass_r > 1.0) e = std::min(e, 8.0 * (I.mass_r - I.s) / (I.mass_r - 1.0));
    if (I.mass_c > 1.0) e = std::min(e, 8.0 * (I.mass_c - I.s) / (I.mass_c - 1.0));
    if ((params->flags & POT_FLAG_NO_SMOOTH) || !(e > 0.0)) e = 0.0;
    I.eps_s = e;
    I.sum_rt = (1.0 - e / 8.0) * I.mass_r + e / 8.0;
    I.sum_ct = (1.0 - e / 8.0) * I.mass_c + e / 8.0;
    I.L = 3.0 * (I.sum_rt + I.sum_ct - I.s) / gamma;
    if (params->flags & POT_FLAG_STOP_RAW_EPS) thr = params->eps;
    I.thr = (params->flags & POT_FLAG_NO_STOP) ? -1.0 : thr;
    I.log_s = log(I.s);
  }
  BCK(cudaMemcpyAsync(dinst, hi.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, st));

  // tile shape: a pinned or earlier choice for this batch signature, else
  // (POT_FLAG_AUTOTUNE) the fastest candidate, timed with CUDA events on a
  // two-sided pass at the zero dual point (a pass's cost does not depend on
  // the potentials)
  float tune_ms = 0.f;
  if (params->flags & POT_FLAG_AUTOTUNE) {
    const std::string sig = batch_signature(probs, count);
    int th = 0, tw = 0;
    {
      std::lock_guard<std::mutex> g(g_tune_mu);
      auto it = g_tune.find(sig);
      if (it != g_tune.end()) { th = it->second.first; tw = it->second.second; }
    }
    if (th == 0) {
      cudaEvent_t a, b;
      BCK(cudaEventCreate(&a));
      BCK(cudaEventCreate(&b));
      BCK(cudaMemsetAsync(V.ut, 0, sizeof(double) * L.N, st));
      BCK(cudaMemsetAsync(V.vt, 0, sizeof(double) * L.M, st));
      float best = 3.4e38f;
      for (int cw : kCandW)
        for (int ch : kCandH) {
          G = b_geom(probs, count, ch, cw);
          BCK(cudaMemcpyAsync(dtiles, G.tiles.data(), sizeof(BTile) * G.T, cudaMemcpyHostToDevice, st));
          B.H = G.H; B.W = G.W; B.ntiles = G.T;
          if ((s = pass(PASS_ROWS | PASS_COLS, V.ut, V.vt, -1, nullptr, nullptr, -1, 0)) != POT_OK) return s;
          BCK(cudaEventRecord(a, st));
          for (int rep = 0; rep < 3; ++rep)
            if ((s = pass(PASS_ROWS | PASS_COLS, V.ut, V.vt, -1, nullptr, nullptr, -1, 0)) != POT_OK) return s;
          BCK(cudaEventRecord(b, st));
          BCK(cudaEventSynchronize(b));
          float t = 0.f;
          BCK(cudaEventElapsedTime(&t, a, b));
          tune_ms += t;
          if (t < best) { best = t; th = ch; tw = cw; }
        }
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tune[sig] = {th, tw};
    }
    G = b_geom(probs, count, th, tw);
    for (int k = 0; k < count; ++k) { hi[k].tile0 = G.tile0[k]; hi[k].ntile = G.ntile[k]; }
    BCK(cudaMemcpyAsync(dinst, hi.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(dtiles, G.tiles.data(), sizeof(BTile) * G.T, cudaMemcpyHostToDevice, st));
    B.H = G.H; B.W = G.W; B.ntiles = G.T;
  }
  b_init_kernel<<<count, kBT, 0, st>>>(V);
  ++launches;

  const int offw_bar = (int)offsetof(BInst, w_bar), offw_out = (int)offsetof(BInst, w_out);
  // The iteration as three fused sweeps (see b_sweep_kernel): each pass's
  // tiles, and per instance the combine, the update and the next pass's
  // terms.  The first iteration's extrapolation and terms are formed here.
  b_extrap_kernel<<<count, kBT, 0, st>>>(V);
  {
    BatchPass q = B;
    q.mode = PASS_ROWS | PASS_COLS; q.arow0 = V.ub; q.bcol0 = V.vb; q.aoff0 = offw_bar; q.check_done = 1;
    launch_prep_batched(q, st);
  }
  launches += 2;
  BCK(cudaGetLastError());
  auto sweep = [&](int mode, int epi, int k) -> pot_status {
    BatchPass q = B;
    q.mode = mode;
    cudaError_t e = launch_sweep(q, V, epi, k, st);
    ++launches;
    if (e != cudaSuccess) return bfail(POT_ECUDA, cudaGetErrorString(e));
    return POT_OK;
  };
  auto body = [&](int k) -> pot_status {
    pot_status q;
    if ((q = sweep(PASS_ROWS | PASS_COLS, E_GRAD, k)) != POT_OK) return q;
    if (greedy) {
      if ((q = sweep(PASS_ROWS | PASS_COLS, E_GGK, k)) != POT_OK) return q;
      return sweep(PASS_ROWS | PASS_COLS, E_GFINAL, k);
    }
    if ((q = sweep(k == 1 ? PASS_COLS : PASS_ROWS, E_GK, k)) != POT_OK) return q;
    return sweep(PASS_ROWS | PASS_COLS, E_FINAL, k);
  };

  // the loop: graphs of `per` iterations, host polls the number of finished instances
  in_loop = true;
  const bool graphs = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
  const int per = std::max(3, ((params->check_every > 0 ? params->check_every : 24) + 2) / 3 * 3);
  cudaGraphExec_t exec = nullptr;
  int64_t per_graph = 0;
  if (graphs) {
    cudaGraph_t g = nullptr;
    const int64_t l0 = launches;
    BCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    pot_status q = POT_OK;
    for (int it = 0; it < per && q == POT_OK; ++it) q = body(it % 3);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (q != POT_OK) { if (g) cudaGraphDestroy(g); return q; }
    BCK(e);
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    BCK(e);
    per_graph = launches - l0;
    launches = l0;
  }
  int hdone = 0, rounds = 0;
  while (rounds * per < params->max_iter + per) {
    if (graphs) {
      BCK(cudaGraphLaunch(exec, st));
      launches += per_graph;
    } else {
      for (int it = 0; it < per; ++it)
        if ((s = body(it % 3)) != POT_OK) return s;
    }
    ++rounds;
    BCK(cudaMemcpyAsync(&hdone, ndone, sizeof(int), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    if (hdone >= count) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (hdone < count) return bfail(POT_ETIMEOUT, "batched: not every instance set its stop flag");

  in_loop = false;
  // rounding (R1-R4) and the objective, all instances at once
  if ((s = pass(PASS_ROWS, V.uo, V.vo, offw_out, nullptr, nullptr, -1, 0)) != POT_OK) return s;
  b_round1_kernel<<<count, kBT, 0, st>>>(V);
  if ((s = pass(PASS_COLS, V.fc, V.vo, -1, nullptr, nullptr, -1, 0)) != POT_OK) return s;
  b_round2_kernel<<<count, kBT, 0, st>>>(V);
  if ((s = pass(PASS_ROWS, V.fc, V.gc, -1, nullptr, nullptr, -1, 0)) != POT_OK) return s;
  b_round34_kernel<<<count, kBT, 0, st>>>(V);
  launches += 3;
  {
    BatchPass q = B;
    q.mode = PASS_OBJ; q.arow0 = V.fc; q.bcol0 = V.gc; q.aoff0 = -1; q.p = V.uh; q.q = V.vh; q.check_done = 0;
    launch_prep_batched(q, st);
    launch_pass_simt_batched(q, st);
    b_obj_kernel<<<count, kBT, 0, st>>>(dinst, red);
    launches += 2;
  }
  BCK(cudaGetLastError());
  BCK(cudaEventRecord(e1, st));
  BCK(cudaMemcpyAsync(hi.data(), dinst, sizeof(BInst) * count, cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pot_status worst = POT_OK;
  for (int k = 0; k < count; ++k) {
    const BInst& I = hi[k];
    pot_result& R = res[k];
    memset(&R, 0, sizeof(R));
    R.iters = I.t;
    R.objective = I.obj;
    R.err_final = I.E;
    R.eps_stop = I.thr;
    R.gamma = I.cost_scale / I.gC;
    R.cost_scale = I.cost_scale;
    R.mass = I.s;
    R.ms = ms;
    R.rounding_branch = I.branch;
    R.nonfinite = I.nonfinite;
    R.kernel_launches = launches;
    R.tile_rows = G.H;
    R.tile_cols = G.W;
    R.tune_ms = tune_ms;
    R.status = I.nonfinite ? POT_ENONFINITE
                           : ((I.E <= I.thr || (params->flags & POT_FLAG_NO_STOP)) ? POT_OK : POT_ENOCONV);
    if (R.status == POT_ENONFINITE) worst = POT_ENONFINITE;
    else if (R.status == POT_ENOCONV && worst == POT_OK) worst = POT_ENOCONV;
  }
  if (worst == POT_ENOCONV) bfail(POT_ENOCONV, "batched: some instances reached max_iter");
  if (worst == POT_ENONFINITE) bfail(POT_ENONFINITE, "batched: non-finite potentials in some instances");
  return worst;
}

}  // extern "C"
