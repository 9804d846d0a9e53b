// pot_marginals_static: the log row / column sums of B(u, v, w) for callers
// that cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc (or a framework allocator)
// at the point where they need this pass: code that runs while another
// component's caching allocator owns the device memory, real-time loops that
// forbid allocation after start-up, or host libraries that have no handle on
// the application's allocator and so cannot provide the workspace that
// pot_marginals takes.  For them this entry point runs exactly the same pass
// with its scratch in a file-scope device array of fixed size instead of a
// caller workspace.
//
// Limits and sharing rules:
//  * the array holds kStaticScratchBytes (16 MiB) on every GPU that loads the
//    library, until the process exits; problems whose one-pass scratch (the
//    layout pot_marginals binds: state, pass partials, one slot of log-sums
//    per side, per-pass terms) would exceed it are rejected with POT_ENOMEM
//    before anything is launched;
//  * every call uses the same array, which keeps the previous call's contents;
//    the counters that must start at zero are cleared by the pass itself, and
//    two calls whose work overlaps on the GPU (different streams, or
//    different host threads on the same device) race on the array;
//  * the first call on a device looks up the array's device address with that
//    device current (cudaGetSymbolAddress); make that first call before any
//    stream capture.
#include <cuda_runtime.h>
#include <mutex>

#include "../../include/aspot.h"

namespace pot {
pot_status set_last_error(pot_status s, const char* msg);
size_t marginals_scratch_bytes(const pot_problem* prob);
}

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per device).
pot_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return pot::set_last_error(POT_ECUDA, "pot_marginals_static: no current CUDA device");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return pot::set_last_error(POT_ECUDA, "pot_marginals_static: cudaGetSymbolAddress of the scratch array failed");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return POT_OK;
}

}  // namespace

extern "C" POT_API pot_status pot_marginals_static(const pot_problem* prob, double gamma, const double* u,
                                                   const double* v, double w, double* lrow, double* lcol,
                                                   double* tot, void* stream) {
  size_t need = 0;
  pot_status s = pot_workspace_size(prob, nullptr, &need);     // argument checks
  if (s != POT_OK) return s;
  need = pot::marginals_scratch_bytes(prob);                   // what the pass itself binds
  if (need > kStaticScratchBytes)
    return pot::set_last_error(POT_ENOMEM, "pot_marginals_static: the problem needs more scratch than the "
                                           "16 MiB static array; use pot_marginals with a workspace");
  void* base = nullptr;
  if ((s = scratch_address(&base)) != POT_OK) return s;
  return pot_marginals(prob, gamma, u, v, w, base, kStaticScratchBytes, lrow, lcol, tot, stream);
}
