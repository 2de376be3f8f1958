// fst_rnea_vjp_noalloc: the RNEA adjoint for callers that must not allocate
// device memory.
//
// fst_rnea_vjp needs a caller-provided scratch buffer for the per-block
// partial sums of theta_bar. Some callers cannot provide one: code running
// inside a memory pool or arena that owns all device memory, real-time loops
// where a cudaMalloc (and its implicit device synchronisation) is not allowed,
// or plugins that only receive tensors from a host framework. This entry
// point takes its scratch from a fixed array in device memory that the
// library defines, so the call itself allocates nothing.
//
// Costs and limits:
//  * the array is 4 MiB (2^20 floats) and is held by every GPU that loads the
//    library, until the process exits;
//  * it holds ceil(B / 32) * (10 * n_bodies + 1) floats, so B is limited (about
//    300,000 environments for an 11-body tree); larger B is rejected with
//    FST_ERR_INVALID_ARG before anything is launched;
//  * all calls share the one array and it keeps the last call's contents.
//    Nothing needs clearing: every call overwrites each partial sum it later
//    reads. Two calls whose kernels overlap on the GPU (different streams, no
//    ordering between them) race on the array and give wrong theta_bar;
//  * the first call on a device looks up the array's device address (one
//    cudaGetSymbolAddress with that device current) and caches it; make that
//    first call before any stream capture. The cached address is valid for
//    the life of the device's primary context: a process that calls
//    cudaDeviceReset must not call this entry point afterwards.
//
// After these checks the call is fst_rnea_vjp with the built-in array as its
// scratch, so it runs the same kernel (generic or specialised) that
// fst_rnea_vjp would run for the model and gives the same results.
#include <cuda_runtime.h>

#include <mutex>
#include <sstream>
#include <string>

#include "fst_internal.h"
#include "launch.h"

namespace {

constexpr size_t kStaticScratchFloats = size_t(1) << 20;
static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on `dev` (which must be current). The
// name is only a host-side handle for the symbol; the kernel needs the
// address that cudaGetSymbolAddress returns.
cudaError_t static_scratch(int dev, float** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_static_scratch);
    if (err != cudaSuccess) return err;
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

fst_status arg_error(const std::string& msg) { return fst::set_error(FST_ERR_INVALID_ARG, msg); }

}  // namespace

extern "C" fst_status fst_rnea_vjp_noalloc(const fst_model* m, int64_t B, const float* q, const float* qd,
                                           const float* qdd, const float* theta, const float* tau_bar, float* q_bar,
                                           float* qd_bar, float* qdd_bar, float* theta_bar, void* stream) {
  static const char* fn = "fst_rnea_vjp_noalloc";
  bool skip = false;
  // the checks of every entry point (model, B <= 2^31 - 1, current device),
  // before anything touches the device
  const fst_status st = fst::check_call(fn, m, B, &skip);
  if (st != FST_OK) return st;
  const size_t need = fst::vjp_scratch_floats(m->n, B);
  if (theta_bar && need > kStaticScratchFloats) {
    std::ostringstream os;
    os << fn << ": B=" << B << " needs " << need << " floats of scratch for theta_bar, more than the built-in "
       << kStaticScratchFloats << " (use fst_rnea_vjp with a caller-provided scratch buffer)";
    return arg_error(os.str());
  }
  if (!skip && m->nv > 0 && (!q || !qd || !qdd || !tau_bar))
    return arg_error(std::string(fn) + ": null q, qd, qdd or tau_bar");
  float* scratch = nullptr;
  if (theta_bar) {
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return fst::set_error(FST_ERR_CUDA, std::string(fn) + ": " + cudaGetErrorString(err));
    if (dev < 0 || dev >= kMaxDevices) {
      std::ostringstream os;
      os << fn << ": device ordinal " << dev << " is beyond the " << kMaxDevices
         << " devices this entry point keeps a scratch address for";
      return arg_error(os.str());
    }
    err = static_scratch(dev, &scratch);
    if (err != cudaSuccess)
      return fst::set_error(FST_ERR_CUDA, std::string(fn) + ": cudaGetSymbolAddress: " + cudaGetErrorString(err));
  }
  return fst_rnea_vjp(m, B, q, qd, qdd, theta, tau_bar, q_bar, qd_bar, qdd_bar, theta_bar, scratch,
                      kStaticScratchFloats * sizeof(float), stream);
}
