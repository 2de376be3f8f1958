// fst_fp32_probe: a throughput probe of the FP32 fused multiply-add pipes,
// the denominator of the roofline fractions that the operators report
// against arithmetic (their flops are FP32 adds, multiplies and FMAs).
//
// Every thread runs kChains independent FMA chains (a = a * m + c, with m
// and c kernel arguments the compiler cannot fold), so each SM sub-partition
// always has independent FMAs to issue while earlier ones are in flight.
// The grid is a whole number of blocks per SM. The caller times the launch
// with CUDA events and divides the flop count this call returns by it.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fst_internal.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, float m, float c, float* __restrict__ out) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(int64_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" fst_status fst_fp32_probe(int32_t blocks_per_sm, int32_t iters, float* out, size_t out_bytes,
                                     double* flops, void* stream) {
  static const char* fn = "fst_fp32_probe";
  if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !out || !flops)
    return fst::set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": bad argument");
  int dev = -1, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return fst::set_error(FST_ERR_CUDA, std::string(fn) + ": " + cudaGetErrorString(err));
  const int64_t blocks = (int64_t)sms * blocks_per_sm;
  if (out_bytes < (size_t)blocks * kThreads * sizeof(float))
    return fst::set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": out smaller than SMs x blocks_per_sm x 256 floats");
  // m and c keep every chain bounded (|a| converges to c / (1 - m))
  fma_probe_kernel<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(iters, 0.999f, 0.001f, out);
  err = cudaGetLastError();
  if (err != cudaSuccess) return fst::set_error(FST_ERR_CUDA, std::string(fn) + ": " + cudaGetErrorString(err));
  *flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  return FST_OK;
}

// ---- SM ids -------------------------------------------------------------------
// The ids (%smid) of the SMs a launch can land on need not be 0 .. SMs - 1
// (a GPU may number its SMs with gaps). The SM-pinned launches give roles by
// SM id, so they need the ids that exist.

namespace {

__global__ void sm_id_kernel(int* out) {
  if (threadIdx.x == 0) {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    out[blockIdx.x] = (int)r;
  }
}

}  // namespace

namespace fst {

// Ids of the SMs of the current device, sorted: one block per SM (a shared
// memory request larger than half an SM's keeps blocks apart), recorded and
// deduplicated, three rounds united in case a busy SM missed one.
// Synchronous.
cudaError_t sm_ids(std::vector<int>& ids) {
  int dev = -1, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  int* d = nullptr;
  err = cudaMalloc((void**)&d, sizeof(int) * sms);
  if (err != cudaSuccess) return err;
  const int sh = 120 * 1024;
  err = cudaFuncSetAttribute(sm_id_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sh);
  std::vector<int> h(sms);
  std::vector<bool> seen(1024, false);
  for (int round = 0; round < 3 && err == cudaSuccess; ++round) {
    sm_id_kernel<<<sms, 32, sh>>>(d);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpy(h.data(), d, sizeof(int) * sms, cudaMemcpyDeviceToHost);
    if (err == cudaSuccess)
      for (int v : h)
        if (v >= 0 && v < 1024) seen[v] = true;
  }
  cudaFree(d);
  ids.clear();
  for (int v = 0; v < 1024; ++v)
    if (seen[v]) ids.push_back(v);
  return err;
}

}  // namespace fst

extern "C" fst_status fst_sm_ids(int32_t* ids, int32_t capacity, int32_t* n) {
  static const char* fn = "fst_sm_ids";
  if (!n || capacity < 0 || (capacity > 0 && !ids))
    return fst::set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": bad argument");
  std::vector<int> v;
  const cudaError_t err = fst::sm_ids(v);
  if (err != cudaSuccess) return fst::set_error(FST_ERR_CUDA, std::string(fn) + ": " + cudaGetErrorString(err));
  *n = (int32_t)v.size();
  for (int k = 0; k < (int)v.size() && k < capacity; ++k) ids[k] = v[k];
  return FST_OK;
}

// ---- addressability ---------------------------------------------------------

extern "C" fst_status fst_device_can_access(const void* ptr, int32_t* ok) {
  static const char* fn = "fst_device_can_access";
  if (!ok) return fst::set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null ok");
  *ok = 0;
  if (!ptr) return FST_OK;
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return fst::set_error(FST_ERR_CUDA, std::string(fn) + ": " + cudaGetErrorString(err));
  cudaPointerAttributes a{};
  err = cudaPointerGetAttributes(&a, ptr);
  if (err != cudaSuccess) {
    cudaGetLastError();  // an unregistered host pointer: not addressable, not an error of the caller's stream
    return FST_OK;
  }
  if (a.type == cudaMemoryTypeDevice) *ok = a.device == dev;
  else if (a.type == cudaMemoryTypeManaged) *ok = 1;
  else if (a.type == cudaMemoryTypeHost) *ok = a.devicePointer == ptr;  // pinned and mapped at the same address
  return FST_OK;
}
