// Shared declarations of the warm-start network kernels (warmstart.cu, the
// CUDA-core path, and ws_tc.cu, the tcgen05 path).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/warmstart.h"

namespace pot {
namespace ws {

constexpr int H = POT_WS_HIDDEN;      // hidden width
constexpr int kTile = 128;            // points per tile (one instance per tile)
constexpr int kLds = H + 1;           // padded shared-memory row (floats)
constexpr int FMAX = POT_WS_MAX_D + POT_WS_EXTRA;

// Offsets (in floats) of the parameter blocks (F = d + 3): W1[H][F], b1[H], W2[H][H],
// U[H][H+2], b2[H], w3[H], b3[1].
struct Offs {
  int F;
  int64_t W1, b1, W2, U, b2, w3, b3, total;
};

inline __host__ __device__ Offs offsets(int d) {
  Offs o;
  o.F = d + POT_WS_EXTRA;
  o.W1 = 0;
  o.b1 = o.W1 + (int64_t)H * o.F;
  o.W2 = o.b1 + H;
  o.U = o.W2 + (int64_t)H * H;
  o.b2 = o.U + (int64_t)H * (H + 2);
  o.w3 = o.b2 + H;
  o.b3 = o.w3 + H;
  o.total = o.b3 + 1;
  return o;
}

struct WsTile {
  int64_t start;   // first point (index into the set's point arrays)
  int64_t ybase;   // first output position in the batch
  int32_t b;       // batch slot of the instance
  int32_t count;   // points in the tile (1..128)
};

struct WsInst {
  int64_t inst;    // instance index in the set
  int32_t tile0, ntiles;
  float npts;
  float pad;
};

struct WsArgs {
  int F, T, B, G;
  Offs o;
  const WsTile* tiles;
  const WsInst* binfo;
  const float* feats;
  const float* extra;
  const float* target;
  const float* weight;   // loss weights or nullptr (all 1)
  const float* P;
  float* ctxp;     // [T][H] per-tile sums of H1
  float* cin;      // [B][H+2] context inputs
  float* q;        // [B][H] U cin
  float* y;        // forward output
  float invN;      // 1 / points in the batch
  // per-tile gradient partials
  float *gW1p, *Mp, *gb1p, *Sp, *gw3p, *dqp, *lossp, *gb3p;
  // per-instance gradient pieces
  float *dq, *cW1, *cb1;
  float* gW2p;     // [G][H][H] per-CTA dW2
  float* dctx;     // [B][H] context gradient / n_k (tensor-core path)
  int* err;        // device error flag (tensor-core path: a wait that timed out)
  // rows of the partial arrays the final reduction sums
  int n_w1p;       // gW1p / gb1p rows (T per tile, or G per CTA)
  int n_cw;        // cW1 / cb1 rows (B, or 0 when the context share is already in gW1p)
  int n_w3p;       // gw3p rows (T or G)
};

__device__ __forceinline__ float gelu(float a) {
  return 0.5f * a * (1.f + erff(a * 0.70710678118654752f));
}
// d/da [a Phi(a)] = Phi(a) + a phi(a)
__device__ __forceinline__ float gelu_grad(float a) {
  return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}

// SplitMix64 finaliser (Steele, Lea and Flood, 2014).
__host__ __device__ inline uint64_t splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// tcgen05 path (ws_tc.cu).  Forward only: writes A.y.  Training: the
// per-tile dq, loss and db3 partials (as the CUDA-core path), per-CTA gW2p,
// gw3p, gW1p and gb1p (context share included), and A.dq / A.dctx.
pot_status launch_ws_main_tc(const WsArgs& A, bool train, cudaStream_t st);

}  // namespace ws
}  // namespace pot
