// Descriptor of one O(nm) pass over the (implicit) Gibbs matrix B(z).
//
// The pass evaluates, for i < n, j < m,
//     logit_ij = a_i + b_j - gC * cost_ij,
//     a_i = arow[i] + (aoff ? *aoff : 0),   b_j = bcol[j]
// with cost_ij either a dense FP32 entry C[i*ldc + j] or the squared
// Euclidean distance |x_i - y_j|^2 between point rows.  It writes log-sum-exp
// partials: for every row i and column block, (max, sum) with
//     log2 sum_j 2^(logit_ij * log2 e) = max + log2(sum),
// and for every column j and row block the same over i (the column shift is
// shared by a stripe of columns, see the kernels).  The objective mode sums
// cost_ij * (exp(logit_ij) + kappa p_i q_j) instead.
#pragma once
#include <stdint.h>

namespace pot {

enum PassMode { PASS_ROWS = 1, PASS_COLS = 2, PASS_OBJ = 4, PASS_MAXCOST = 8 };

constexpr uint64_t kDefaultWaitNs = 2000000000ull;   // default bound of a pass's pipeline waits (2 s)

enum CostKind { COST_DENSE_F32 = 0, COST_SQEUCLID_BF16 = 1, COST_SQEUCLID_F16 = 2, COST_SQEUCLID_F32 = 3 };

struct PassDesc {
  int64_t n, m;
  int kind;
  const float* C; int64_t ldc;
  const void* X; const void* Y; int d; int64_t ldx, ldy;
  const float* xn; const float* yn;     // squared norms of the point rows (FP32)
  double gC;                            // logit multiplier of the raw cost (cost_scale / gamma)
  // potentials: set 0, or set 1 when sel != nullptr && *sel != 0
  const double* arow0; const double* bcol0; const double* aoff0;
  const double* arow1; const double* bcol1; const double* aoff1;
  const int* sel;
  int mode;
  float2* row_part;      // [ncolblk][n]
  float2* col_part;      // [nrowblk][m]
  double* red_part;      // objective / max-cost partials, one per CTA
  const double* p; const double* q; const double* kappa;   // objective rank-one term
  const int* done;       // when non-null and *done != 0 the pass returns at once
  const int* skip;       // when non-null and *skip == skip_if the pass returns at once
  int skip_if;
  // tensor-core path only: per-pass row / column terms (padded) and an error flag
  float4* rowA; float2* colA; float2* colB;
  int* err;              // set to 1 when a bounded pipeline wait of the pass ran out
  uint64_t wait_ns;      // bound of each pipeline wait (ns)
  int stall;             // test hook: the hot-loop tcgen05 pass withholds its first accumulator hand-off
  int transpose;         // a columns-only tcgen05 pass may run as the rows-only kernel of the transposed
                         // problem (where the layout allows it, TcLayout::swap)
};

// True when the pass must not run (the solve has stopped, or its skip
// condition holds); every kernel of a pass returns at once then.
__host__ __device__ inline bool pass_off(const PassDesc& P) {
  return (P.done && *P.done) || (P.skip && *P.skip == P.skip_if);
}

}  // namespace pot
