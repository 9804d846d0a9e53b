// C-ABI entry points (include/aspot.h): argument checks, workspace layout,
// the host drivers of ASPOT (Algorithm 2) and of the feasible Sinkhorn
// baseline (Algorithm 3), rounding and objective.
//
// The iteration loops run as CUDA graphs of `check_every` iterations; every
// kernel of an iteration returns at once when the device stop flag is set,
// and the host reads the flag between graph launches.  No device memory is
// allocated: all scratch is carved from the caller's workspace.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdarg.h>
#include <stddef.h>
#include <string.h>
#include <math.h>
#include <string>
#include <vector>
#include <algorithm>
#include <nvtx3/nvToolsExt.h>

#include "../../include/aspot.h"
#include "kernels.h"

using namespace pot;

namespace {

thread_local std::string g_err;

pot_status fail(pot_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(POT_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define CKL()                                                                             \
  do {                                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess) return fail(POT_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

constexpr int kSlots = 12;

struct Layout {
  bool use_tc = false;
  SimtLayout sl{};
  TcLayout tl{};
  int64_t ncolblk = 0, nrowblk = 0;
  int64_t red_doubles = 0;
  size_t off_state = 0, off_red = 0, off_cnt = 0, off_stats = 0, off_xn = 0, off_yn = 0;
  size_t off_rowp = 0, off_colp = 0, off_u[kSlots] = {}, off_v[kSlots] = {};
  size_t off_rowA = 0, off_colA = 0, off_colB = 0;
  size_t off_binst = 0;       // the single-cluster loop's instance record and stop counter
  size_t total = 0;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

bool wants_tc(const pot_problem* P, int flags) {
  if (flags & POT_FLAG_FORCE_SIMT) return false;
  if (P->kind != POT_COST_SQEUCLID_BF16) return false;
  PassDesc d{};
  d.n = P->n; d.m = P->m; d.kind = P->kind; d.X = P->X; d.Y = P->Y; d.d = P->d; d.ldx = P->ldx; d.ldy = P->ldy;
  return tc_supported(d);
}

// nslots: FP64 potential slots per side (the solvers use kSlots; a lone pass
// needs one, for its combined log-sums)
Layout make_layout(const pot_problem* P, int flags, int nslots = kSlots) {
  Layout L;
  const int64_t n = P->n, m = P->m;
  L.sl = simt_layout(n, m);
  if (P->kind == POT_COST_DENSE_F32 && (m % 4) == 0 && (P->ldc % 4) == 0 && ((uintptr_t)P->C % 16) == 0) {
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 152;
    }
    simt_dense_layout(L.sl, n, m, sms);
  }
  L.use_tc = wants_tc(P, flags);
  if (L.use_tc) {
    L.tl = tc_layout(n, m, P->d);
    L.ncolblk = L.tl.ncolblk;
    L.nrowblk = L.tl.nrowblk;
  } else {
    L.ncolblk = L.sl.ncolblk;
    L.nrowblk = L.sl.dense_fast ? L.sl.nslots : L.sl.nrowblk;
  }
  const int64_t vblk = std::max<int64_t>(vec_blocks(n + m + 2), loop_blocks_max(n + m + 2));
  const int64_t pass_ctas = std::max<int64_t>(L.sl.ncolblk * L.sl.nrowblk, L.use_tc ? L.tl.v1_units : 0);
  L.red_doubles = std::max<int64_t>(vblk * 12, pass_ctas) + 64;   // up to 9 sums + (max, sum) per block
  size_t o = 0;
  L.off_state = o; o = align_up(o + sizeof(DevState));
  L.off_red = o; o = align_up(o + sizeof(double) * L.red_doubles);
  L.off_cnt = o; o = align_up(o + sizeof(unsigned int) * 8);
  L.off_stats = o; o = align_up(o + sizeof(double) * 8);
  L.off_xn = o; o = align_up(o + sizeof(float) * (n + 1));
  L.off_yn = o; o = align_up(o + sizeof(float) * (m + 1));
  // column partials: also room for the CUDA-core tiles of the single-cluster
  // loop, which are never fewer rows than the layout's H
  const int64_t colblk = L.use_tc ? L.nrowblk : std::max<int64_t>(L.nrowblk, L.sl.nrowblk);
  L.off_rowp = o; o = align_up(o + sizeof(float2) * L.ncolblk * n);
  L.off_colp = o; o = align_up(o + sizeof(float2) * colblk * m);
  for (int k = kSlots - nslots; k < kSlots; ++k) { L.off_u[k] = o; o = align_up(o + sizeof(double) * (n + 2)); }
  for (int k = kSlots - nslots; k < kSlots; ++k) { L.off_v[k] = o; o = align_up(o + sizeof(double) * (m + 2)); }
  {
    const int64_t np = L.use_tc ? std::max<int64_t>(L.tl.n_pad, n) : n;
    const int64_t mp = L.use_tc ? std::max<int64_t>(L.tl.m_pad, m) : m;
    L.off_rowA = o; o = align_up(o + sizeof(float4) * np);
    L.off_colA = o; o = align_up(o + sizeof(float2) * mp);
    L.off_colB = o; o = align_up(o + sizeof(float2) * mp);
  }
  L.off_binst = o; o = align_up(o + sizeof(BInst) + 64);
  L.total = o;
  return L;
}

struct Ctx {
  const pot_problem* P;
  cudaStream_t st;
  Layout L;
  char* ws;
  DevState* S;
  double* red;
  unsigned int* cnt;
  double* stats;
  float *xn, *yn;
  float2 *rowp, *colp;
  float4* rowA = nullptr;
  float2 *colA = nullptr, *colB = nullptr;
  double *lrow = nullptr, *lcol = nullptr;     // combined log-sums of the last row / column pass
  BInst* binst = nullptr;                      // single-cluster loop: instance record
  int* bndone = nullptr;                       // and its stop counter
  double* U[kSlots];
  double* V[kSlots];
  double cost_scale = 1.0;
  double max_raw = 0.0;
  uint64_t wait_ns = 0;         // bound of the tcgen05 passes' pipeline waits (0: their 2 s default)
  int stall = 0;                // test hook: hot-loop tcgen05 passes withhold their first hand-off
  double sum_r = 0, sum_c = 0, min_r = 0, min_c = 0;
  // kernel launch count and optional CUDA-event timing of the main-loop passes
  int64_t launches = 0;
  bool prof = false;
  bool in_loop = false;
  int pass_ord = 0;
  std::vector<cudaEvent_t> ev;      // pairs (start, end) per pass ordinal of one graph
  double pass_ms = 0.0;
  int64_t pass_count = 0;
  ~Ctx() { for (cudaEvent_t e : ev) cudaEventDestroy(e); }
};

pot_status check_problem(const pot_problem* P) {
  if (!P) return fail(POT_EINVAL, "problem is NULL");
  if (P->n < 1 || P->m < 1) return fail(POT_EINVAL, "n and m must be >= 1 (got %lld, %lld)", (long long)P->n, (long long)P->m);
  if (P->n > (int64_t(1) << 31) || P->m > (int64_t(1) << 31)) return fail(POT_EINVAL, "n, m too large");
  if (!P->r || !P->c) return fail(POT_EINVAL, "r and c must be device pointers");
  if (!(P->s > 0.0) || !isfinite(P->s)) return fail(POT_EINVAL, "s must be finite and > 0");
  if (!(P->cost_scale >= 0.0) || !isfinite(P->cost_scale)) return fail(POT_EINVAL, "cost_scale must be finite and >= 0");
  switch (P->kind) {
    case POT_COST_DENSE_F32:
      if (!P->C) return fail(POT_EINVAL, "dense cost pointer is NULL");
      if (P->ldc < P->m) return fail(POT_EINVAL, "ldc < m");
      break;
    case POT_COST_SQEUCLID_BF16:
    case POT_COST_SQEUCLID_F16:
    case POT_COST_SQEUCLID_F32:
      if (!P->X || !P->Y) return fail(POT_EINVAL, "point pointers are NULL");
      if (P->d < 1 || P->d > 4096) return fail(POT_EINVAL, "d must be in [1, 4096]");
      if (P->ldx < P->d || P->ldy < P->d) return fail(POT_EINVAL, "ldx, ldy must be >= d");
      break;
    default:
      return fail(POT_EINVAL, "unknown cost kind %d", (int)P->kind);
  }
  return POT_OK;
}

pot_status check_params(const pot_params* Q) {
  if (!Q) return fail(POT_EINVAL, "params is NULL");
  if (!(Q->eps > 0.0) || !isfinite(Q->eps)) return fail(POT_EINVAL, "eps must be finite and > 0");
  if (!isfinite(Q->gamma)) return fail(POT_EINVAL, "gamma must be finite");
  if (Q->max_iter < 1) return fail(POT_EINVAL, "max_iter must be >= 1");
  if (Q->block_rule != 0 && Q->block_rule != 1) return fail(POT_EINVAL, "block_rule must be 0 (cyclic) or 1 (greedy)");
  if (Q->check_every < 0) return fail(POT_EINVAL, "check_every must be >= 0");
  if (!isfinite(Q->w0)) return fail(POT_EINVAL, "w0 must be finite");
  if (Q->resume) {
    const pot_aspot_state* R = Q->resume;
    if (Q->u0 || Q->v0 || Q->w0 != 0.0) return fail(POT_EINVAL, "resume excludes a warm start (u0, v0, w0)");
    if (!R->u_tilde || !R->v_tilde || !R->u_check || !R->v_check)
      return fail(POT_EINVAL, "resume: every state vector must be a device buffer");
    if (!(R->theta > 0.0) || R->theta > 1.0 || R->t < 0) return fail(POT_EINVAL, "resume: bad theta or t");
    if (!isfinite(R->w_tilde) || !isfinite(R->w_check) || !isfinite(R->phi_check))
      return fail(POT_EINVAL, "resume: non-finite scalars");
    if (R->t >= Q->max_iter) return fail(POT_EINVAL, "resume: max_iter must exceed the state's t");
  }
  return POT_OK;
}

pot_status bind(Ctx& X, const pot_problem* P, int flags, void* ws, size_t ws_bytes, void* stream,
                int nslots = kSlots) {
  X.P = P;
  X.st = (cudaStream_t)stream;
  X.L = make_layout(P, flags, nslots);
  if (!ws) return fail(POT_EINVAL, "workspace is NULL");
  if ((uintptr_t)ws % 256 != 0) return fail(POT_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < X.L.total) return fail(POT_ENOMEM, "workspace too small: %zu < %zu bytes", ws_bytes, X.L.total);
  X.ws = (char*)ws;
  X.S = (DevState*)(X.ws + X.L.off_state);
  X.red = (double*)(X.ws + X.L.off_red);
  X.cnt = (unsigned int*)(X.ws + X.L.off_cnt);
  X.stats = (double*)(X.ws + X.L.off_stats);
  X.xn = (float*)(X.ws + X.L.off_xn);
  X.yn = (float*)(X.ws + X.L.off_yn);
  X.rowp = (float2*)(X.ws + X.L.off_rowp);
  X.colp = (float2*)(X.ws + X.L.off_colp);
  for (int k = 0; k < kSlots; ++k) { X.U[k] = (double*)(X.ws + X.L.off_u[k]); X.V[k] = (double*)(X.ws + X.L.off_v[k]); }
  X.lrow = X.U[kSlots - 1];
  X.lcol = X.V[kSlots - 1];
  X.rowA = (float4*)(X.ws + X.L.off_rowA);
  X.colA = (float2*)(X.ws + X.L.off_colA);
  X.colB = (float2*)(X.ws + X.L.off_colB);
  X.binst = (BInst*)(X.ws + X.L.off_binst);
  X.bndone = (int*)(X.ws + X.L.off_binst + ((sizeof(BInst) + 15) & ~size_t(15)));
  return POT_OK;
}

PassDesc base_desc(const Ctx& X, double gamma) {
  PassDesc d{};
  const pot_problem* P = X.P;
  d.n = P->n; d.m = P->m; d.kind = P->kind;
  d.C = P->C; d.ldc = P->ldc;
  d.X = P->X; d.Y = P->Y; d.d = P->d; d.ldx = P->ldx; d.ldy = P->ldy;
  d.xn = X.xn; d.yn = X.yn;
  d.gC = gamma > 0.0 ? X.cost_scale / gamma : 0.0;
  d.row_part = X.rowp; d.col_part = X.colp; d.red_part = X.red;
  d.rowA = X.rowA; d.colA = X.colA; d.colB = X.colB; d.err = &X.S->tc_err;
  d.wait_ns = X.wait_ns > 0 ? X.wait_ns : kDefaultWaitNs;
  d.stall = X.stall;
  return d;
}

// A tcgen05 pass whose bounded pipeline wait ran out raises S->tc_err (its
// sums are then invalid).  clear_tc resets the flag at the start of a call;
// check_tc synchronises the stream and turns a raised flag into POT_ETIMEOUT.
pot_status clear_tc(Ctx& X) {
  CK(cudaMemsetAsync(&X.S->tc_err, 0, sizeof(int), X.st));
  return POT_OK;
}

pot_status tc_timeout() {
  return fail(POT_ETIMEOUT, "a tcgen05 pass gave up waiting on its pipeline (bounded mbarrier wait ran out); "
                            "its sums are invalid");
}

pot_status check_tc(Ctx& X) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, &X.S->tc_err, sizeof(int), cudaMemcpyDeviceToHost, X.st));
  CK(cudaStreamSynchronize(X.st));
  return e ? tc_timeout() : POT_OK;
}

// combine: launch the combine of the partials into lrow / lcol (the solvers'
// loop kernels combine them themselves and pass false)
pot_status run_pass(Ctx& X, const PassDesc& d, bool profile = true, bool combine = true) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (X.prof && X.in_loop && profile) {
    const size_t need = 2 * (size_t)(X.pass_ord + 1);
    while (X.ev.size() < need) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      X.ev.push_back(e);
    }
    e0 = X.ev[2 * X.pass_ord];
    e1 = X.ev[2 * X.pass_ord + 1];
    X.pass_ord++;
  }
  // events inside a captured graph must be external event-record nodes
  if (X.L.use_tc) {
    CK(launch_pass_tc(d, X.L.tl, X.st, e0));
    // terms, (row-partial clear,) pass
    X.launches += ((d.mode & PASS_ROWS) && X.L.tl.v3) || tc_swaps_cols(X.L.tl, d) ? 3 : 2;
  } else {
    if (d.mode & (PASS_ROWS | PASS_COLS | PASS_OBJ)) {
      launch_prep(d, d.n, d.m, X.st);
      X.launches += 1;
    }
    if (e0) CK(cudaEventRecordWithFlags(e0, X.st, cudaEventRecordExternal));
    launch_pass_simt(d, X.L.sl, X.st);
    X.launches += 1;
  }
  if (e1) CK(cudaEventRecordWithFlags(e1, X.st, cudaEventRecordExternal));
  // a transposed columns-only pass (large tcgen05 problems) leaves sw_nslots
  // partials per column; the loop kernels' inline combine never sees one
  const bool swapped = X.L.use_tc && tc_swaps_cols(X.L.tl, d);
  if (swapped && !combine) return fail(POT_ECUDA, "internal: a transposed column pass needs the combine launch");
  if (combine && (d.mode & (PASS_ROWS | PASS_COLS))) {
    launch_combine(X.rowp, X.L.ncolblk, d.n, (d.mode & PASS_ROWS) ? X.lrow : nullptr, X.colp,
                   swapped ? X.L.tl.sw_nslots : X.L.nrowblk, d.m, (d.mode & PASS_COLS) ? X.lcol : nullptr, d.done,
                   X.st, d.skip, d.skip_if);
    X.launches += 1;
  }
  CKL();
  return POT_OK;
}

// Whether the solver loops' update kernels combine the pass partials inline
// (one thread per row / column) instead of a combine launch: when every entry
// has at most 32 partials.
int fuse_combine(const Ctx& X) { return (X.L.ncolblk <= 32 && X.L.nrowblk <= 32) ? 1 : 0; }

int64_t pass_ctas(const Ctx& X) {  // one partial per CTA of a max / objective pass
  return X.L.use_tc ? X.L.tl.v1_units : X.L.sl.ncolblk * X.L.sl.nrowblk;
}

// masses, minima, finiteness of r, c; squared norms; max of the raw cost
pot_status prologue(Ctx& X, bool need_max) {
  const pot_problem* P = X.P;
  CK(cudaMemsetAsync(X.cnt, 0, sizeof(unsigned int) * 8, X.st));
  pot_status s0 = clear_tc(X);
  if (s0 != POT_OK) return s0;
  launch_marg_stats(P->r, P->c, P->n, P->m, X.red, X.cnt, X.stats, X.st); X.launches += 1;
  CKL();
  if (P->kind != POT_COST_DENSE_F32) {
    launch_sqnorm(P->kind, P->X, P->n, P->d, P->ldx, X.xn, X.st);
    launch_sqnorm(P->kind, P->Y, P->m, P->d, P->ldy, X.yn, X.st);
    X.launches += 2;
    CKL();
  }
  if (need_max) {
    PassDesc d = base_desc(X, 0.0);
    d.mode = PASS_MAXCOST;
    pot_status s = run_pass(X, d);
    if (s != POT_OK) return s;
    launch_reduce_parts(X.red, pass_ctas(X), 1, X.stats + 6, X.st); X.launches += 1;
    CKL();
  }
  double h[8];
  int tce = 0;
  CK(cudaMemcpyAsync(h, X.stats, sizeof(h), cudaMemcpyDeviceToHost, X.st));
  CK(cudaMemcpyAsync(&tce, &X.S->tc_err, sizeof(int), cudaMemcpyDeviceToHost, X.st));
  CK(cudaStreamSynchronize(X.st));
  if (tce) return tc_timeout();
  X.sum_r = h[0]; X.sum_c = h[1]; X.min_r = h[2]; X.min_c = h[3];
  if (h[4] != 0.0) return fail(POT_EINVAL, "r and c must be finite and non-negative");
  if (!(X.sum_r > 0.0) || !(X.sum_c > 0.0)) return fail(POT_EINVAL, "r and c must have positive mass");
  const double mn = std::min(X.sum_r, X.sum_c);
  if (P->s > mn * (1.0 + 1e-12)) return fail(POT_EINVAL, "s = %.17g exceeds min(|r|_1, |c|_1) = %.17g", P->s, mn);
  if (need_max) {
    X.max_raw = h[6];
    if (!(X.max_raw >= 0.0) || !isfinite(X.max_raw)) return fail(POT_EINVAL, "cost contains NaN/Inf");
  }
  X.cost_scale = P->cost_scale > 0.0 ? P->cost_scale : (X.max_raw > 0.0 ? 1.0 / X.max_raw : 1.0);
  return POT_OK;
}

struct SetupOut { double gamma, eps_stop, eps_s, sum_rt, sum_ct, T, L, cmax; };

// Algorithm 2 setup: gamma = eps/(4 log n), eps~ = eps/(8 max C), mass guards,
// smoothing coefficient (guards shrink it; the stop threshold is unguarded).
SetupOut approx_setup(const Ctx& X, const pot_params* Q) {
  SetupOut o;
  const double nn = (double)std::max(X.P->n, X.P->m);
  o.gamma = Q->gamma > 0.0 ? Q->gamma : Q->eps / (4.0 * log(std::max(nn, 2.0)));
  o.cmax = X.cost_scale * X.max_raw;
  o.eps_stop = Q->eps / (8.0 * (o.cmax > 0.0 ? o.cmax : 1.0));
  double e = o.eps_stop;
  const double s = X.P->s;
  if (X.sum_r > 1.0) e = std::min(e, 8.0 * (X.sum_r - s) / (X.sum_r - 1.0));
  if (X.sum_c > 1.0) e = std::min(e, 8.0 * (X.sum_c - s) / (X.sum_c - 1.0));
  if ((Q->flags & POT_FLAG_NO_SMOOTH) || !(e > 0.0)) e = 0.0;
  o.eps_s = e;
  o.sum_rt = (1.0 - e / 8.0) * X.sum_r + e / 8.0;
  o.sum_ct = (1.0 - e / 8.0) * X.sum_c + e / 8.0;
  o.T = o.sum_rt + o.sum_ct - s;
  o.L = 3.0 * o.T / o.gamma;
  if (Q->flags & POT_FLAG_STOP_RAW_EPS) o.eps_stop = Q->eps;
  return o;
}

pot_status upload_state(Ctx& X, const DevState& h) {
  CK(cudaMemcpyAsync(X.S, &h, offsetof(DevState, trace), cudaMemcpyHostToDevice, X.st));
  return POT_OK;
}

pot_status read_state(Ctx& X, DevState& h) {
  CK(cudaMemcpyAsync(&h, X.S, offsetof(DevState, trace), cudaMemcpyDeviceToHost, X.st));
  CK(cudaStreamSynchronize(X.st));
  return POT_OK;
}

// Run `body` (one iteration per call, k = iteration index mod 3, the index
// starting at k0) until the device stop flag is set.  With a capturable stream the iterations are
// captured into a CUDA graph of `per` iterations.
// passes_per_iter(k): timed passes of an iteration with block k
template <class Body, class PassesPerIter>
pot_status drive(Ctx& X, int per, int max_iter, PassesPerIter passes_per_iter, Body body, int k0 = 0) {
  cudaStreamCaptureStatus cs;
  CK(cudaStreamIsCapturing(X.st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(POT_EINVAL, "the stream is being captured");
  const bool graphs = X.st != nullptr && X.st != cudaStreamLegacy && X.st != cudaStreamPerThread;
  per = std::max(3, (per + 2) / 3 * 3);
  int done = 0, launched = 0;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t per_graph_launches = 0;
  X.in_loop = true;
  if (graphs) {
    const int64_t l0 = X.launches;
    X.pass_ord = 0;
    CK(cudaStreamBeginCapture(X.st, cudaStreamCaptureModeThreadLocal));
    pot_status s = POT_OK;
    {
      // kernel-to-kernel edges of the graph become programmatic ones (each
      // kernel's blocks are scheduled while its predecessor runs and wait for
      // it on the device), except in profiled solves, whose timing events sit
      // between the kernels
      pdl_scope pdl(!X.prof);
      for (int it = 0; it < per && s == POT_OK; ++it) s = body((it + k0) % 3);
    }
    per_graph_launches = X.launches - l0;
    X.launches = l0;
    cudaGraph_t g2 = nullptr;
    cudaError_t e = cudaStreamEndCapture(X.st, &g2);
    if (s != POT_OK) { if (g2) cudaGraphDestroy(g2); return s; }
    if (e != cudaSuccess) return fail(POT_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    graph = g2;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return fail(POT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
  }
  pot_status st = POT_OK;
  int flags3[6] = {0, 0, 0, 0, 0, 0};   // DevState t, take_hat, done, max_iter, nonfinite, tc_err (adjacent ints)
  int t_prev = 0;
  while (launched < max_iter + per) {
    if (graphs) {
      cudaError_t e = cudaGraphLaunch(exec, X.st);
      if (e != cudaSuccess) { st = fail(POT_ECUDA, "graph launch: %s", cudaGetErrorString(e)); break; }
      X.launches += per_graph_launches;
    } else {
      X.pass_ord = 0;
      for (int it = 0; it < per && st == POT_OK; ++it) st = body((it + k0) % 3);
      if (st != POT_OK) break;
    }
    launched += per;
    cudaError_t e = cudaMemcpyAsync(flags3, &X.S->t, sizeof(flags3), cudaMemcpyDeviceToHost, X.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(X.st);
    if (e != cudaSuccess) { st = fail(POT_ECUDA, "stop flag: %s", cudaGetErrorString(e)); break; }
    if (X.prof) {
      // passes of the iterations that ran in this launch (later ones returned at once)
      const int ran = std::min(flags3[0] - t_prev, per);
      int npass = 0;
      for (int it = 0; it < ran; ++it) npass += passes_per_iter((it + k0) % 3);
      npass = std::min<int>(npass, (int)X.ev.size() / 2);
      for (int k = 0; k < npass; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, X.ev[2 * k], X.ev[2 * k + 1]) == cudaSuccess) { X.pass_ms += ms; X.pass_count++; }
      }
    }
    t_prev = flags3[0];
    done = flags3[2];
    if (flags3[5]) { st = tc_timeout(); break; }
    if (done) break;
  }
  X.in_loop = false;
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (st == POT_OK && !done) st = fail(POT_ETIMEOUT, "device stop flag never set");
  return st;
}

// ------------------------------------------------ single-cluster loop ---
// Problems up to kClusterEntries cost entries with CUDA-core passes iterate in
// one thread-block cluster (cluster.cu): one launch per `per` iterations
// instead of about ten dependent kernels per iteration.  Beyond about 512 x 512
// the 16 SMs of one cluster do the passes more slowly than the whole GPU
// (measured: 256^2 49 against 62 us per iteration, 512^2 68 against 72,
// 1000^2 113 against 86).
constexpr double kClusterEntries = 262144.0;

// tile rows of the cluster loop: the CUDA-core layout's, raised so that a
// column has at most 16 row-block partials for the epilogue CTA to combine
int cluster_rows(int64_t n, int H) {
  const int64_t h = ((n + 16 * 32 - 1) / (16 * 32)) * 32;
  return (int)std::max<int64_t>(H, h);
}

bool use_cluster(const Ctx& X, const pot_params* p, const PassDesc& d) {
  if (X.L.use_tc) return false;
  if (p->flags & (POT_FLAG_STAGED | POT_FLAG_PROFILE)) return false;
  if ((double)X.P->n * (double)X.P->m > kClusterEntries) return false;
  return cluster_loop_kind(d) != 0 && cluster_loop_size(d, X.L.sl.V) > 0;
}

pot_status cluster_drive(Ctx& X, const AspotVecs& V, const PassDesc& d, int per, int max_iter, bool greedy) {
  cudaStreamCaptureStatus cs;
  CK(cudaStreamIsCapturing(X.st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(POT_EINVAL, "the stream is being captured");
  const pot_problem* P = X.P;
  ClusterLoop A{};
  A.P = d;
  A.vecs = V;
  A.inst = X.binst;
  A.ndone = X.bndone;
  A.V = X.L.sl.V;
  A.H = cluster_rows(P->n, X.L.sl.H);
  A.ncta = cluster_loop_size(d, A.V);
  A.trace4 = V.trace ? &X.S->trace[0][0] : nullptr;
  BInst hI;
  memset(&hI, 0, sizeof(hI));
  hI.n = P->n; hI.m = P->m;
  hI.ntile = ((P->n + A.H - 1) / A.H) * ((P->m + 128 * A.V - 1) / (128 * A.V));
  hI.X = P->X; hI.Y = P->Y; hI.d = P->d; hI.kind = P->kind; hI.ldx = P->ldx; hI.ldy = P->ldy;
  hI.r = P->r; hI.c = P->c; hI.s = P->s; hI.cost_scale = X.cost_scale; hI.gC = d.gC;
  hI.pu = V.uo; hI.pv = V.vo;
  CK(cudaMemcpyAsync(X.binst, &hI, sizeof(BInst), cudaMemcpyHostToDevice, X.st));
  CK(cudaMemsetAsync(X.bndone, 0, sizeof(int), X.st));
  if (P->kind == POT_COST_DENSE_F32) {      // the per-pass terms read zero norms
    CK(cudaMemsetAsync(X.xn, 0, sizeof(float) * (P->n + 1), X.st));
    CK(cudaMemsetAsync(X.yn, 0, sizeof(float) * (P->m + 1), X.st));
  }
  CK(launch_cluster_enter(X.binst, X.S, X.st));
  X.launches += 1;
  int done = 0, launched = 0;
  pot_status st = POT_OK;
  while (launched < max_iter + per) {
    cudaError_t e = launch_cluster_loop(A, per, greedy ? 1 : 0, launched == 0 ? 1 : 0, X.st);
    if (e != cudaSuccess) { st = fail(POT_ECUDA, "cluster loop launch: %s", cudaGetErrorString(e)); break; }
    X.launches += 1;
    launched += per;
    e = cudaMemcpyAsync(&done, &X.binst->done, sizeof(int), cudaMemcpyDeviceToHost, X.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(X.st);
    if (e != cudaSuccess) { st = fail(POT_ECUDA, "stop flag: %s", cudaGetErrorString(e)); break; }
    if (done) break;
  }
  if (st != POT_OK) return st;
  CK(launch_cluster_exit(X.binst, X.S, X.st));
  X.launches += 1;
  if (!done) return fail(POT_ETIMEOUT, "device stop flag never set");
  return POT_OK;
}

pot_status do_round(Ctx& X, double gamma, const double* u, const double* v, pot_plan* plan, int* branch) {
  // w is expected in S->w_out
  const pot_problem* P = X.P;
  RoundVecs R{};
  R.n = P->n; R.m = P->m; R.r = P->r; R.c = P->c; R.u = u; R.v = v;
  R.f = plan->f; R.g = plan->g; R.p = plan->p; R.q = plan->q; R.kappa = plan->kappa;
  R.row_part = X.rowp; R.col_part = X.colp; R.ncolblk = X.L.ncolblk; R.nrowblk = X.L.nrowblk;
  R.lrow = X.lrow; R.lcol = X.lcol;
  R.red = X.red; R.counter = X.cnt; R.S = X.S;
  PassDesc d = base_desc(X, gamma);
  // R1: rows of B(u, v, w)
  d.mode = PASS_ROWS; d.arow0 = u; d.bcol0 = v; d.aoff0 = &X.S->w_out;
  pot_status s = run_pass(X, d);
  if (s != POT_OK) return s;
  launch_round_r1(R, X.st); X.launches += 1;
  CKL();
  // R2: columns of diag(a) B
  d.mode = PASS_COLS; d.arow0 = plan->f; d.bcol0 = v; d.aoff0 = nullptr;
  if ((s = run_pass(X, d)) != POT_OK) return s;
  launch_round_r2(R, X.st); X.launches += 1;
  CKL();
  DevState h;
  if ((s = read_state(X, h)) != POT_OK) return s;
  if (h.tc_err) return tc_timeout();
  if (h.m2 >= P->s) {
    launch_round_r3(R, X.st); X.launches += 1;
    CKL();
    if (branch) *branch = 3;
  } else {
    d.mode = PASS_ROWS; d.arow0 = plan->f; d.bcol0 = plan->g; d.aoff0 = nullptr;
    if ((s = run_pass(X, d)) != POT_OK) return s;
    launch_round_r4(R, X.st); X.launches += 1;
    CKL();
    if (branch) *branch = 4;
  }
  return POT_OK;
}

pot_status do_objective(Ctx& X, double gamma, const pot_plan* plan, double* out) {
  PassDesc d = base_desc(X, gamma);
  d.mode = PASS_OBJ; d.arow0 = plan->f; d.bcol0 = plan->g; d.aoff0 = nullptr;
  d.p = plan->p; d.q = plan->q; d.kappa = plan->kappa;
  pot_status s = run_pass(X, d);
  if (s != POT_OK) return s;
  launch_reduce_parts(X.red, pass_ctas(X), 0, X.stats + 7, X.st); X.launches += 1;
  CKL();
  double h;
  int tce = 0;
  CK(cudaMemcpyAsync(&h, X.stats + 7, sizeof(double), cudaMemcpyDeviceToHost, X.st));
  CK(cudaMemcpyAsync(&tce, &X.S->tc_err, sizeof(int), cudaMemcpyDeviceToHost, X.st));
  CK(cudaStreamSynchronize(X.st));
  if (tce) return tc_timeout();
  *out = h * X.cost_scale;
  return POT_OK;
}

// pot_params.wait_limit_ns: > 0 bounds the tcgen05 passes' pipeline waits;
// < 0 also injects a stall into the hot-loop passes (a test hook); 0 keeps 2 s.
void set_wait(Ctx& X, const pot_params* Q) {
  const int64_t w = Q->wait_limit_ns;
  X.wait_ns = w == 0 ? 0 : (uint64_t)(w < 0 ? -w : w);
  X.stall = w < 0 ? 1 : 0;
}

pot_status check_plan(const pot_plan* plan) {
  if (!plan) return fail(POT_EINVAL, "plan is NULL");
  if (!plan->u || !plan->v || !plan->w || !plan->f || !plan->g || !plan->p || !plan->q || !plan->kappa)
    return fail(POT_EINVAL, "every pot_plan pointer must be a device buffer");
  return POT_OK;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a); cudaEventCreate(&b); cudaEventRecord(a, st);
  }
  double stop() {
    float ms = 0.f;
    cudaEventRecord(b, st); cudaEventSynchronize(b); cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
};

// NVTX range for the whole scope (solver phases show up by name in profilers;
// without an attached tool the calls do nothing).
struct Nvtx {
  explicit Nvtx(const char* name) { nvtxRangePushA(name); }
  ~Nvtx() { nvtxRangePop(); }
  Nvtx(const Nvtx&) = delete;
  Nvtx& operator=(const Nvtx&) = delete;
};

}  // namespace

namespace pot {
// Records a failure message for pot_last_error() from another translation unit.
pot_status set_last_error(pot_status s, const char* msg) {
  g_err = msg;
  return s;
}
// Scratch bytes pot_marginals needs for this problem (its one-pass layout).
size_t marginals_scratch_bytes(const pot_problem* prob) { return make_layout(prob, 0, 1).total; }
}  // namespace pot

extern "C" {

const char* pot_last_error(void) { return g_err.c_str(); }

pot_status pot_workspace_size(const pot_problem* prob, const pot_params* params, size_t* bytes) {
  g_err.clear();
  pot_status s = check_problem(prob);
  if (s != POT_OK) return s;
  if (!bytes) return fail(POT_EINVAL, "bytes is NULL");
  *bytes = make_layout(prob, params ? params->flags : 0).total;
  return POT_OK;
}

pot_status pot_marginals_workspace_size(const pot_problem* prob, size_t* bytes) {
  g_err.clear();
  pot_status s = check_problem(prob);
  if (s != POT_OK) return s;
  if (!bytes) return fail(POT_EINVAL, "bytes is NULL");
  *bytes = make_layout(prob, 0, 1).total;
  return POT_OK;
}

pot_status aspot_solve(const pot_problem* prob, const pot_params* params, void* workspace, size_t ws_bytes,
                       pot_plan* plan, pot_result* res, void* stream) {
  g_err.clear();
  pot_status s;
  if ((s = check_problem(prob)) != POT_OK) return s;
  if ((s = check_params(params)) != POT_OK) return s;
  if ((s = check_plan(plan)) != POT_OK) return s;
  if (!res) return fail(POT_EINVAL, "result is NULL");
  memset(res, 0, sizeof(*res));
  Ctx X;
  if ((s = bind(X, prob, params->flags, workspace, ws_bytes, stream)) != POT_OK) return s;
  X.prof = (params->flags & POT_FLAG_PROFILE) != 0;
  set_wait(X, params);
  Nvtx range_all("aspot_solve");
  Timer tm(X.st);
  {
    Nvtx range("aspot: setup");
    if ((s = prologue(X, true)) != POT_OK) return s;
  }
  const SetupOut so = approx_setup(X, params);
  const int64_t n = prob->n, m = prob->m;
  DevState h{};
  h.L = so.L; h.s = prob->s; h.thr = (params->flags & POT_FLAG_NO_STOP) ? -1.0 : so.eps_stop;
  h.log_s = log(prob->s); h.sum_rt = so.sum_rt; h.sum_ct = so.sum_ct; h.max_iter = params->max_iter;
  h.theta = 1.0;
  if ((s = upload_state(X, h)) != POT_OK) return s;

  AspotVecs V{};
  V.n = n; V.m = m;
  V.rt = X.U[0]; V.lrt = X.U[1]; V.ct = X.V[0]; V.lct = X.V[1];
  V.ut = X.U[2]; V.vt = X.V[2]; V.uc = X.U[3]; V.vc = X.V[3]; V.ub = X.U[4]; V.vb = X.V[4];
  V.ug = X.U[5]; V.vg = X.V[5]; V.uh = X.U[6]; V.vh = X.V[6]; V.uo = plan->u; V.vo = plan->v;
  V.row_part = X.rowp; V.col_part = X.colp; V.ncolblk = X.L.ncolblk; V.nrowblk = X.L.nrowblk;
  V.lrow = X.lrow; V.lcol = X.lcol;
  V.red = X.red; V.counter = X.cnt; V.S = X.S; V.trace = (params->flags & POT_FLAG_TRACE) ? 1 : 0;
  V.fused = 0;                             // the warm-start check below uses combined passes
  launch_aspot_init(V, prob->r, prob->c, so.eps_s, params->u0, params->v0, params->w0, X.st); X.launches += 1;
  CKL();
  const pot_aspot_state* RS = params->resume;
  if (RS) {
    // continue a solve: z~, z_check (and z^t = z_check until the first iteration), theta, t, phi(z_check)
    CK(cudaMemcpyAsync(V.ut, RS->u_tilde, sizeof(double) * n, cudaMemcpyDeviceToDevice, X.st));
    CK(cudaMemcpyAsync(V.vt, RS->v_tilde, sizeof(double) * m, cudaMemcpyDeviceToDevice, X.st));
    CK(cudaMemcpyAsync(V.uc, RS->u_check, sizeof(double) * n, cudaMemcpyDeviceToDevice, X.st));
    CK(cudaMemcpyAsync(V.vc, RS->v_check, sizeof(double) * m, cudaMemcpyDeviceToDevice, X.st));
    CK(cudaMemcpyAsync(V.uo, RS->u_check, sizeof(double) * n, cudaMemcpyDeviceToDevice, X.st));
    CK(cudaMemcpyAsync(V.vo, RS->v_check, sizeof(double) * m, cudaMemcpyDeviceToDevice, X.st));
    DevState h2;
    if ((s = read_state(X, h2)) != POT_OK) return s;
    h2.theta = RS->theta; h2.t = RS->t;
    h2.w_tilde = RS->w_tilde; h2.w_check = RS->w_check; h2.w_out = RS->w_check; h2.w_z = RS->w_check;
    h2.phi_check = RS->phi_check;
    if ((s = upload_state(X, h2)) != POT_OK) return s;
  }

  const double gamma = so.gamma;
  PassDesc d = base_desc(X, gamma);
  const bool warm_check = (params->flags & POT_FLAG_WARM_CHECK) && (params->u0 || params->v0);
  if (warm_check) {
    // E at the given start and at zero; keep the given start only if it is not worse
    PassDesc pw = d;
    pw.mode = PASS_ROWS | PASS_COLS; pw.arow0 = V.uc; pw.bcol0 = V.vc; pw.aoff0 = &X.S->w_check;
    if ((s = run_pass(X, pw)) != POT_OK) return s;
    launch_aspot_start_eval(V, V.uc, V.vc, 0, X.st);
    launch_aspot_zero_bar(V, X.st);
    PassDesc pz = d;
    pz.mode = PASS_ROWS | PASS_COLS; pz.arow0 = V.ub; pz.bcol0 = V.vb; pz.aoff0 = &X.S->w_bar;
    if ((s = run_pass(X, pz)) != POT_OK) return s;
    launch_aspot_start_eval(V, V.ub, V.vb, 1, X.st);
    launch_aspot_start_select(V, X.st);
    X.launches += 4;
    CKL();
  }
  auto body = [&](int k) -> pot_status {
    pot_status q;
    PassDesc p1 = d;                       // gradient pass at z_bar (both sides)
    p1.mode = PASS_ROWS | PASS_COLS; p1.arow0 = V.ub; p1.bcol0 = V.vb; p1.aoff0 = &X.S->w_bar; p1.done = &X.S->done;
    if ((q = run_pass(X, p1, true, !V.fused)) != POT_OK) return q;
    launch_aspot_after_grad(V, X.st); X.launches += 1;
    // Greenkhorn pass at z_grave: the side of block k (both sides for the w-step,
    // whose column sums give those of z^ in closed form)
    PassDesc p2 = d;
    p2.mode = (k == 1) ? PASS_COLS : (k == 2 ? (PASS_ROWS | PASS_COLS) : PASS_ROWS);
    p2.arow0 = V.ug; p2.bcol0 = V.vg; p2.aoff0 = &X.S->w_grave;
    p2.done = &X.S->done;
    if ((q = run_pass(X, p2, true, !V.fused)) != POT_OK) return q;
    launch_aspot_after_greenkhorn(V, k, X.st); X.launches += 1;
    // pass at z^t = argmin.  When the argmin keeps z^ (take_hat), the sums of
    // the side block k just updated follow from the Greenkhorn pass in closed
    // form (u-step: log r(B(z^))_i = log r(B(z_grave))_i + u^_i - u_grave_i;
    // w-step: both sides shift by w^ - w_grave), so P3a computes only the other
    // side (nothing for k = 2) and P3b the remaining ones only when z^t = z_check.
    PassDesc p3 = d;
    p3.arow0 = V.uc; p3.bcol0 = V.vc; p3.aoff0 = &X.S->w_check;
    p3.arow1 = (k == 0) ? V.uh : V.ug; p3.bcol1 = (k == 1) ? V.vh : V.vg; p3.aoff1 = &X.S->w_hat;
    p3.sel = &X.S->take_hat; p3.done = &X.S->done;
    if (k != 2) {
      PassDesc p3a = p3;
      p3a.mode = (k == 0) ? PASS_COLS : PASS_ROWS;
      // after a u-step the column sums at z^t enter E_t alone, so this pass may
      // run transposed.  The v-step's Greenkhorn pass keeps the kernel's own
      // column side: its sums decide the argmin phi(z^) < phi(z_check), a
      // near-tie that the other summation order tipped to z_check in two thirds
      // of the v-steps at n = 32768, each then paying the pass at z_check.
      p3a.transpose = 1;
      if ((q = run_pass(X, p3a, true, !V.fused)) != POT_OK) return q;
    }
    PassDesc p3b = p3;
    p3b.mode = (k == 0) ? PASS_ROWS : (k == 1 ? PASS_COLS : (PASS_ROWS | PASS_COLS));
    p3b.skip = &X.S->take_hat; p3b.skip_if = 1;
    if ((q = run_pass(X, p3b, false, !V.fused)) != POT_OK) return q;
    launch_aspot_after_final(V, k, X.st); X.launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(POT_ECUDA, "iteration launch: %s", cudaGetErrorString(e));
    return POT_OK;
  };
  // Greedy block rule: k is chosen on the device from a two-sided pass at
  // z_grave (P2); at z^t one of three passes runs, selected by device flags:
  // both sides at z_check, rows after a v-step, columns after a u-step
  // (nothing after a w-step, whose sums follow in closed form).
  auto body_greedy = [&](int) -> pot_status {
    pot_status q;
    PassDesc p1 = d;
    p1.mode = PASS_ROWS | PASS_COLS; p1.arow0 = V.ub; p1.bcol0 = V.vb; p1.aoff0 = &X.S->w_bar; p1.done = &X.S->done;
    if ((q = run_pass(X, p1, true, !V.fused)) != POT_OK) return q;
    launch_aspot_after_grad(V, X.st); X.launches += 1;
    PassDesc p2 = d;
    p2.mode = PASS_ROWS | PASS_COLS; p2.arow0 = V.ug; p2.bcol0 = V.vg; p2.aoff0 = &X.S->w_grave;
    p2.done = &X.S->done;
    if ((q = run_pass(X, p2, true, !V.fused)) != POT_OK) return q;
    launch_aspot_greedy_pick(V, X.st);
    launch_aspot_after_greenkhorn(V, -1, X.st); X.launches += 2;
    PassDesc p3 = d;
    p3.arow0 = V.uc; p3.bcol0 = V.vc; p3.aoff0 = &X.S->w_check;
    p3.arow1 = V.uh; p3.bcol1 = V.vh; p3.aoff1 = &X.S->w_hat;
    p3.sel = &X.S->take_hat; p3.done = &X.S->done;
    PassDesc p3z = p3;                     // z^t = z_check: both sides
    p3z.mode = PASS_ROWS | PASS_COLS; p3z.skip = &X.S->take_hat; p3z.skip_if = 1;
    if ((q = run_pass(X, p3z, false, !V.fused)) != POT_OK) return q;
    PassDesc p3r = p3;                     // z^t = z^ after a v-step: rows
    p3r.mode = PASS_ROWS; p3r.skip = &X.S->run_r3; p3r.skip_if = 0;
    if ((q = run_pass(X, p3r, false, !V.fused)) != POT_OK) return q;
    PassDesc p3c = p3;                     // z^t = z^ after a u-step: columns
    p3c.mode = PASS_COLS; p3c.skip = &X.S->run_c3; p3c.skip_if = 0;
    if ((q = run_pass(X, p3c, false, !V.fused)) != POT_OK) return q;
    launch_aspot_greedy_final(V, X.st);
    launch_aspot_greedy_apply(V, X.st); X.launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(POT_ECUDA, "iteration launch: %s", cudaGetErrorString(e));
    return POT_OK;
  };
  const int per = params->check_every > 0 ? params->check_every : 24;
  auto aspot_passes = [](int k) { return k == 2 ? 2 : 3; };      // P1, P2 (, P3a); P3b is not timed
  auto greedy_passes = [](int) { return 2; };                     // P1, P2; the passes at z^t are not timed
  const bool cluster = use_cluster(X, params, d);
  if (cluster) {
    Nvtx range("aspot: iterations (cluster loop)");
    s = cluster_drive(X, V, d, per, params->max_iter, params->block_rule == 1);
  } else {
    // z_bar of the first iteration; later ones are formed by the iteration's last kernel
    launch_aspot_extrap(V, X.st); X.launches += 1;
    // from here the loop kernels combine the partials themselves when there are
    // few per entry (small problems, where a launch costs more than the work);
    // with many (the tcgen05 pass at large n: one per 256-row block) the wide
    // combine kernel, eight threads per entry, is faster
    V.fused = fuse_combine(X);
    CKL();
    Nvtx range("aspot: iterations");
    const int k0 = RS ? RS->t % 3 : 0;      // the cyclic rule goes on with block t mod 3
    if (params->block_rule == 1) s = drive(X, per, params->max_iter, greedy_passes, body_greedy);
    else s = drive(X, per, params->max_iter, aspot_passes, body, k0);
  }
  if (s != POT_OK) return s;
  res->cluster_loop = cluster ? 1 : 0;
  if ((s = read_state(X, h)) != POT_OK) return s;
  CK(cudaMemcpyAsync(plan->w, &X.S->w_out, sizeof(double), cudaMemcpyDeviceToDevice, X.st));
  res->iters = h.t;
  res->err_final = h.E;
  res->eps_stop = h.thr;
  res->gamma = gamma;
  res->cost_scale = X.cost_scale;
  res->nonfinite = h.nonfinite;
  int branch = 0;
  {
    Nvtx range("aspot: round + objective");
    if ((s = do_round(X, gamma, plan->u, plan->v, plan, &branch)) != POT_OK) return s;
    res->rounding_branch = branch;
    if ((s = do_objective(X, gamma, plan, &res->objective)) != POT_OK) return s;
  }
  res->mass = prob->s;
  res->ms = tm.stop();
  res->pass_ms = X.pass_ms;
  res->pass_launches = X.pass_count;
  res->kernel_launches = X.launches;
  if (warm_check) {
    res->err_warm = h.e_start[0];
    res->err_zero = h.e_start[1];
    res->warm_used = h.warm_used;
  } else {
    res->warm_used = (params->u0 || params->v0 || params->w0 != 0.0) ? 1 : 0;
  }
  if (h.nonfinite) { res->status = POT_ENONFINITE; return fail(POT_ENONFINITE, "non-finite potentials or sums"); }
  const bool conv = h.E <= h.thr;
  res->status = (conv || (params->flags & POT_FLAG_NO_STOP)) ? POT_OK : POT_ENOCONV;
  if (res->status == POT_ENOCONV) fail(POT_ENOCONV, "max_iter reached with E = %.3e > %.3e", h.E, h.thr);
  return (pot_status)res->status;
}

pot_status aspot_state_export(const pot_problem* prob, const pot_params* params, void* workspace, size_t ws_bytes,
                              pot_aspot_state* state, void* stream) {
  g_err.clear();
  pot_status s;
  if ((s = check_problem(prob)) != POT_OK) return s;
  if (!params) return fail(POT_EINVAL, "params is NULL");
  if (!state || !state->u_tilde || !state->v_tilde || !state->u_check || !state->v_check)
    return fail(POT_EINVAL, "state: every vector must be a device buffer");
  Ctx X;
  if ((s = bind(X, prob, params->flags, workspace, ws_bytes, stream)) != POT_OK) return s;
  const int64_t n = prob->n, m = prob->m;
  // the solve's slots: z~ in U[2] / V[2], z_check in U[3] / V[3]
  CK(cudaMemcpyAsync(state->u_tilde, X.U[2], sizeof(double) * n, cudaMemcpyDeviceToDevice, X.st));
  CK(cudaMemcpyAsync(state->v_tilde, X.V[2], sizeof(double) * m, cudaMemcpyDeviceToDevice, X.st));
  CK(cudaMemcpyAsync(state->u_check, X.U[3], sizeof(double) * n, cudaMemcpyDeviceToDevice, X.st));
  CK(cudaMemcpyAsync(state->v_check, X.V[3], sizeof(double) * m, cudaMemcpyDeviceToDevice, X.st));
  DevState h;
  if ((s = read_state(X, h)) != POT_OK) return s;
  state->w_tilde = h.w_tilde;
  state->w_check = h.w_check;
  state->phi_check = h.phi_check;
  state->theta = h.theta;
  state->t = h.t;
  state->pad = 0;
  return POT_OK;
}

pot_status sinkhorn_pot_solve(const pot_problem* prob, const pot_params* params, void* workspace,
                              size_t ws_bytes, pot_plan* plan, pot_result* res, void* stream) {
  g_err.clear();
  pot_status s;
  if ((s = check_problem(prob)) != POT_OK) return s;
  if ((s = check_params(params)) != POT_OK) return s;
  if (params->resume) return fail(POT_EINVAL, "resume applies to ASPOT only");
  if ((s = check_plan(plan)) != POT_OK) return s;
  if (!res) return fail(POT_EINVAL, "result is NULL");
  memset(res, 0, sizeof(*res));
  Ctx X;
  if ((s = bind(X, prob, params->flags, workspace, ws_bytes, stream)) != POT_OK) return s;
  X.prof = (params->flags & POT_FLAG_PROFILE) != 0;
  set_wait(X, params);
  Nvtx range_all("sinkhorn_pot_solve");
  Timer tm(X.st);
  if ((s = prologue(X, true)) != POT_OK) return s;
  SetupOut so = approx_setup(X, params);
  double gamma = so.gamma, thr = so.eps_stop;
  if (params->p_tune >= 1.0) {
    // Theorem 2: H_min from the original marginals (host copy, O(n + m))
    std::vector<double> hr(prob->n), hc(prob->m);
    CK(cudaMemcpyAsync(hr.data(), prob->r, sizeof(double) * prob->n, cudaMemcpyDeviceToHost, X.st));
    CK(cudaMemcpyAsync(hc.data(), prob->c, sizeof(double) * prob->m, cudaMemcpyDeviceToHost, X.st));
    CK(cudaStreamSynchronize(X.st));
    double Hr = 0, Hc = 0;
    for (double x : hr) if (x > 0) Hr -= x * log(x);
    for (double x : hc) if (x > 0) Hc -= x * log(x);
    const double hmin = std::min(Hr, Hc);
    if (!(hmin > 0.0)) return fail(POT_EINVAL, "tuned gamma needs H_min > 0");
    gamma = pow(2.0 * params->eps / (49.0 * hmin), 1.0 / params->p_tune);
    thr = hmin * pow(gamma, params->p_tune);
  }
  if (params->flags & POT_FLAG_NO_STOP) thr = -1.0;
  const double A = 8.0 * so.cmax / params->eps;
  const int64_t n = prob->n, m = prob->m;
  DevState h{};
  h.s = prob->s; h.thr = thr; h.sum_rt = so.sum_rt; h.sum_ct = so.sum_ct; h.max_iter = params->max_iter;
  h.A_over_g = A / gamma;
  if ((s = upload_state(X, h)) != POT_OK) return s;
  SinkVecs V{};
  V.n = n; V.m = m;
  V.drow = (so.sum_ct - prob->s) > 1e-14 * prob->s;
  V.dcol = (so.sum_rt - prob->s) > 1e-14 * prob->s;
  V.re = X.U[0]; V.lre = X.U[1]; V.ce = X.V[0]; V.lce = X.V[1];
  V.u = X.U[2]; V.v = X.V[2]; V.uprev = X.U[3];
  V.row_part = X.rowp; V.col_part = X.colp; V.ncolblk = X.L.ncolblk; V.nrowblk = X.L.nrowblk;
  V.lrow = X.lrow; V.lcol = X.lcol;
  V.red = X.red; V.counter = X.cnt; V.S = X.S; V.trace = (params->flags & POT_FLAG_TRACE) ? 1 : 0;
  V.fused = fuse_combine(X);               // the update kernels combine the pass partials themselves
  launch_sink_init(V, prob->r, prob->c, so.eps_s, prob->s, X.st); X.launches += 1;
  CKL();
  PassDesc d = base_desc(X, gamma);
  auto body = [&](int) -> pot_status {
    pot_status q;
    PassDesc pr = d;
    pr.mode = PASS_ROWS; pr.arow0 = V.u; pr.bcol0 = V.v; pr.aoff0 = nullptr; pr.done = &X.S->done;
    if ((q = run_pass(X, pr, true, !V.fused)) != POT_OK) return q;
    launch_sink_after_rows(V, X.st); X.launches += 2;
    PassDesc pc = d;
    pc.mode = PASS_COLS; pc.arow0 = V.u; pc.bcol0 = V.v; pc.aoff0 = nullptr; pc.done = &X.S->done;
    if ((q = run_pass(X, pc, true, !V.fused)) != POT_OK) return q;
    launch_sink_after_cols(V, X.st); X.launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(POT_ECUDA, "iteration launch: %s", cudaGetErrorString(e));
    return POT_OK;
  };
  const int per = params->check_every > 0 ? params->check_every : 24;
  {
    Nvtx range("sinkhorn: iterations");
    if ((s = drive(X, per, params->max_iter, [](int) { return 2; }, body)) != POT_OK) return s;
  }
  if ((s = read_state(X, h)) != POT_OK) return s;
  // final duals: the first n / m extended potentials, w = 0
  CK(cudaMemcpyAsync(plan->u, V.u, sizeof(double) * n, cudaMemcpyDeviceToDevice, X.st));
  CK(cudaMemcpyAsync(plan->v, V.v, sizeof(double) * m, cudaMemcpyDeviceToDevice, X.st));
  CK(cudaMemsetAsync(plan->w, 0, sizeof(double), X.st));
  CK(cudaMemsetAsync(&X.S->w_out, 0, sizeof(double), X.st));
  res->iters = h.t;
  res->err_final = h.E;
  res->eps_stop = thr;
  res->gamma = gamma;
  res->cost_scale = X.cost_scale;
  res->nonfinite = h.nonfinite;
  int branch = 0;
  if ((s = do_round(X, gamma, plan->u, plan->v, plan, &branch)) != POT_OK) return s;
  res->rounding_branch = branch;
  if ((s = do_objective(X, gamma, plan, &res->objective)) != POT_OK) return s;
  res->mass = prob->s;
  res->ms = tm.stop();
  res->pass_ms = X.pass_ms;
  res->pass_launches = X.pass_count;
  res->kernel_launches = X.launches;
  if (h.nonfinite || h.done == 3) { res->status = POT_ENONFINITE; return fail(POT_ENONFINITE, "non-finite potentials or sums"); }
  const bool conv = h.done == 2;
  res->status = (conv || (params->flags & POT_FLAG_NO_STOP)) ? POT_OK : POT_ENOCONV;
  if (res->status == POT_ENOCONV) fail(POT_ENOCONV, "max_iter reached with residual %.3e > %.3e", h.E, thr);
  return (pot_status)res->status;
}

pot_status pot_round(const pot_problem* prob, double gamma, const double* u, const double* v, double w,
                     void* workspace, size_t ws_bytes, pot_plan* plan, int32_t* branch, void* stream) {
  g_err.clear();
  pot_status s;
  if ((s = check_problem(prob)) != POT_OK) return s;
  if (!(gamma > 0.0) || !isfinite(gamma)) return fail(POT_EINVAL, "gamma must be finite and > 0");
  if (!u || !v || !isfinite(w)) return fail(POT_EINVAL, "u, v must be device pointers and w finite");
  if (!plan || !plan->f || !plan->g || !plan->p || !plan->q || !plan->kappa) return fail(POT_EINVAL, "plan buffers missing");
  Ctx X;
  if ((s = bind(X, prob, 0, workspace, ws_bytes, stream)) != POT_OK) return s;
  if ((s = prologue(X, prob->cost_scale == 0.0)) != POT_OK) return s;
  CK(cudaMemcpyAsync(&X.S->w_out, &w, sizeof(double), cudaMemcpyHostToDevice, X.st));
  double s2 = prob->s;
  CK(cudaMemcpyAsync(&X.S->s, &s2, sizeof(double), cudaMemcpyHostToDevice, X.st));
  int b = 0;
  if ((s = do_round(X, gamma, u, v, plan, &b)) != POT_OK) return s;
  if (branch) *branch = b;
  return check_tc(X);
}

pot_status pot_objective(const pot_problem* prob, const pot_plan* plan, double gamma, void* workspace,
                         size_t ws_bytes, double* out, void* stream) {
  g_err.clear();
  pot_status s;
  if ((s = check_problem(prob)) != POT_OK) return s;
  if (!(gamma > 0.0) || !isfinite(gamma)) return fail(POT_EINVAL, "gamma must be finite and > 0");
  if (!plan || !plan->f || !plan->g || !plan->p || !plan->q || !plan->kappa) return fail(POT_EINVAL, "plan buffers missing");
  if (!out) return fail(POT_EINVAL, "out is NULL");
  Ctx X;
  if ((s = bind(X, prob, 0, workspace, ws_bytes, stream)) != POT_OK) return s;
  if ((s = prologue(X, prob->cost_scale == 0.0)) != POT_OK) return s;
  return do_objective(X, gamma, plan, out);
}

pot_status pot_marginals(const pot_problem* prob, double gamma, const double* u, const double* v, double w,
                         void* workspace, size_t ws_bytes, double* lrow, double* lcol, double* tot, void* stream) {
  g_err.clear();
  pot_status s;
  if ((s = check_problem(prob)) != POT_OK) return s;
  if (!(gamma > 0.0) || !isfinite(gamma)) return fail(POT_EINVAL, "gamma must be finite and > 0");
  if (!u || !v || !isfinite(w)) return fail(POT_EINVAL, "u, v must be device pointers and w finite");
  if (prob->cost_scale == 0.0) return fail(POT_EINVAL, "pot_marginals needs an explicit cost_scale > 0");
  Ctx X;
  if ((s = bind(X, prob, 0, workspace, ws_bytes, stream, 1)) != POT_OK) return s;   // one pass: one slot per side
  X.cost_scale = prob->cost_scale;
  if (prob->kind != POT_COST_DENSE_F32) {
    launch_sqnorm(prob->kind, prob->X, prob->n, prob->d, prob->ldx, X.xn, X.st);
    launch_sqnorm(prob->kind, prob->Y, prob->m, prob->d, prob->ldy, X.yn, X.st);
    CKL();
  }
  // w (by value in a kernel argument), the reduction counters and the stall flag
  launch_marginals_setup(X.S, w, X.cnt, X.st);
  PassDesc d = base_desc(X, gamma);
  // rows unless only the columns are asked for (then |B|_1 comes from the columns)
  d.mode = ((lrow || !lcol) ? PASS_ROWS : 0) | (lcol ? PASS_COLS : 0);
  d.transpose = 1;
  d.arow0 = u; d.bcol0 = v; d.aoff0 = &X.S->w_out;
  if ((s = run_pass(X, d)) != POT_OK) return s;
  launch_marginals_out(prob->n, prob->m, (d.mode & PASS_ROWS) ? X.lrow : nullptr, lcol ? X.lcol : nullptr, lrow,
                       lcol, X.red, X.cnt, tot, &X.S->tc_err, X.st);
  CKL();
  return POT_OK;
}

pot_status pot_cost_max(const pot_problem* prob, void* workspace, size_t ws_bytes, double* out, void* stream) {
  g_err.clear();
  pot_status s;
  if ((s = check_problem(prob)) != POT_OK) return s;
  if (!out) return fail(POT_EINVAL, "out is NULL");
  Ctx X;
  if ((s = bind(X, prob, 0, workspace, ws_bytes, stream)) != POT_OK) return s;
  if ((s = prologue(X, true)) != POT_OK) return s;
  *out = X.max_raw;
  return POT_OK;
}

pot_status pot_plan_dense(const pot_problem* prob, const pot_plan* plan, double gamma, float* Xout, int64_t ldx,
                          void* stream) {
  g_err.clear();
  pot_status s;
  if ((s = check_problem(prob)) != POT_OK) return s;
  if (!(prob->cost_scale > 0.0)) return fail(POT_EINVAL, "pot_plan_dense needs an explicit cost_scale > 0");
  if (!(gamma > 0.0)) return fail(POT_EINVAL, "gamma must be > 0");
  if (!plan || !plan->f || !plan->g || !plan->p || !plan->q || !plan->kappa || !Xout) return fail(POT_EINVAL, "missing buffers");
  if (ldx < prob->m) return fail(POT_EINVAL, "ldx < m");
  PassDesc d{};
  d.n = prob->n; d.m = prob->m; d.kind = prob->kind; d.C = prob->C; d.ldc = prob->ldc;
  d.X = prob->X; d.Y = prob->Y; d.d = prob->d; d.ldx = prob->ldx; d.ldy = prob->ldy;
  d.gC = prob->cost_scale / gamma;
  launch_dense_plan(d, plan->f, plan->g, plan->p, plan->q, plan->kappa, Xout, ldx, (cudaStream_t)stream);
  CKL();
  return POT_OK;
}

const char* pot_pass_kernel(const pot_problem* prob, int32_t flags) {
  if (check_problem(prob) != POT_OK) return "";
  const Layout L = make_layout(prob, flags);
  if (L.use_tc) return L.tl.v3 ? "tc3_pass_kernel" : "tc_pass_kernel";
  if (prob->kind == POT_COST_DENSE_F32 && L.sl.dense_fast) return "dense_pass_kernel";
  return "pass_simt_kernel";
}

pot_status pot_pass_status(void* workspace, void* stream) {
  g_err.clear();
  if (!workspace) return fail(POT_EINVAL, "workspace is NULL");
  const DevState* S = (const DevState*)((char*)workspace);   // the state sits at offset 0
  int e = 0;
  CK(cudaMemcpyAsync(&e, &S->tc_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return e ? tc_timeout() : POT_OK;
}

pot_status pot_trace(void* workspace, int32_t iters, double* out, void* stream) {
  g_err.clear();
  if (!workspace || !out || iters < 0) return fail(POT_EINVAL, "bad arguments");
  const DevState* S = (const DevState*)((char*)workspace);   // the state sits at offset 0
  const int k = std::min(iters, 4096);
  CK(cudaMemcpyAsync(out, S->trace, sizeof(double) * 4 * k, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return POT_OK;
}

}  // extern "C"
