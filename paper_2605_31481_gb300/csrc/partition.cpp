// SM partitions: disjoint sets of a device's SMs, each with a stream whose
// kernels run only on those SMs (CUDA green contexts). The operators of one
// step can then run side by side, each on SMs that execute only its own
// code, so no SM refetches another operator's instructions between launches.
//
// The driver functions come from cudaGetDriverEntryPointByVersion, like the
// run-time compiler's (jit.cpp), so libfst.so does not link the driver
// library: on a host without green contexts the create call reports
// FST_ERR_UNSUPPORTED.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "fst_internal.h"

namespace fst {
namespace {

struct GreenDriver {
  bool ok = false;
  CUresult (*device_get)(CUdevice*, int) = nullptr;
  CUresult (*get_resource)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
  CUresult (*split)(CUdevResource*, unsigned*, const CUdevResource*, CUdevResource*, unsigned, unsigned) = nullptr;
  CUresult (*gen_desc)(CUdevResourceDesc*, CUdevResource*, unsigned) = nullptr;
  CUresult (*create)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned) = nullptr;
  CUresult (*stream_create)(CUstream*, CUgreenCtx, unsigned, int) = nullptr;
  CUresult (*destroy)(CUgreenCtx) = nullptr;
  CUresult (*stream_destroy)(CUstream) = nullptr;
  std::string missing;
};

std::string g_missing;

template <typename F>
bool entry(const char* name, F& out, int version) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    g_missing = name;
    return false;
  }
  out = reinterpret_cast<F>(p);
  return true;
}

const GreenDriver& green_driver() {
  static GreenDriver D;
  static std::once_flag once;
  std::call_once(once, [] {
    // the ABI of the toolkit's own headers (the prototypes above)
    const int v = CUDART_VERSION;
    D.ok = entry("cuDeviceGet", D.device_get, v) && entry("cuDeviceGetDevResource", D.get_resource, v) &&
           entry("cuDevSmResourceSplitByCount", D.split, v) && entry("cuDevResourceGenerateDesc", D.gen_desc, v) &&
           entry("cuGreenCtxCreate", D.create, v) && entry("cuGreenCtxStreamCreate", D.stream_create, v) &&
           entry("cuGreenCtxDestroy", D.destroy, v) && entry("cuStreamDestroy", D.stream_destroy, v);
    D.missing = g_missing;
  });
  return D;
}

}  // namespace
}  // namespace fst

struct fst_sm_partition {
  int device = -1;
  std::vector<CUgreenCtx> ctx;
  std::vector<CUstream> stream;
  std::vector<int> sms;
};

namespace {

void release(fst_sm_partition* p) {
  const fst::GreenDriver& D = fst::green_driver();
  for (CUstream s : p->stream)
    if (s) D.stream_destroy(s);
  for (CUgreenCtx c : p->ctx)
    if (c) D.destroy(c);
  delete p;
}

}  // namespace

extern "C" {

fst_status fst_sm_partition_create(int32_t device, const int32_t* sm_counts, int32_t n, fst_sm_partition** out) {
  using namespace fst;
  static const char* fn = "fst_sm_partition_create";
  if (!out) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null out");
  *out = nullptr;
  if (!sm_counts || n < 1 || n > FST_MAX_PARTITIONS)
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": need 1 to FST_MAX_PARTITIONS SM counts");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": no such device");
  const GreenDriver& D = green_driver();
  if (!D.ok)
    return set_error(FST_ERR_UNSUPPORTED, std::string(fn) + ": the driver has no green contexts (missing " +
                                              D.missing + ")");
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {
    cudaSetDevice(prev);
    return set_error(FST_ERR_CUDA, std::string(fn) + ": cannot initialise the device");
  }
  cudaSetDevice(prev);
  CUdevice dev;
  CUdevResource all{};
  if (D.device_get(&dev, device) != CUDA_SUCCESS || D.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS)
    return set_error(FST_ERR_UNSUPPORTED, std::string(fn) + ": the device's SMs cannot be partitioned");
  // one split of all SMs into groups of the smallest partition size; each
  // partition is a run of whole groups (the split API combines groups of
  // one split, and discourages splitting a remainder again)
  // groups of 8 SMs, ignoring the GPC co-scheduling structure (no kernel
  // here uses thread-block clusters): 19 groups on a 152-SM GB300
  unsigned ng = 0;
  const unsigned gmin = all.sm.minSmPartitionSize > 8 ? all.sm.minSmPartitionSize : 8;
  const unsigned flags = CU_DEV_SM_RESOURCE_SPLIT_IGNORE_SM_COSCHEDULING;
  if (D.split(nullptr, &ng, &all, nullptr, flags, gmin) != CUDA_SUCCESS || ng == 0)
    return set_error(FST_ERR_UNSUPPORTED, std::string(fn) + ": the device's SMs cannot be partitioned");
  std::vector<CUdevResource> grp(ng);
  CUdevResource rem{};
  if (D.split(grp.data(), &ng, &all, &rem, flags, gmin) != CUDA_SUCCESS || ng == 0)
    return set_error(FST_ERR_UNSUPPORTED, std::string(fn) + ": the device's SMs cannot be partitioned");
  const int gsize = (int)grp[0].sm.smCount;
  std::vector<int> take(n);
  unsigned total = 0;
  for (int k = 0; k < n; ++k) {
    if (sm_counts[k] < 1) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": SM counts must be positive");
    take[k] = (sm_counts[k] + gsize - 1) / gsize;
    total += (unsigned)take[k];
  }
  if (total > ng)
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": the SM counts, rounded up to groups of " +
                                              std::to_string(gsize) + " SMs, need " + std::to_string(total) +
                                              " groups; the device has " + std::to_string(ng));
  fst_sm_partition* p = new fst_sm_partition;
  p->device = device;
  unsigned used = 0;
  for (int k = 0; k < n; ++k) {
    CUdevResourceDesc desc;
    CUgreenCtx ctx = nullptr;
    CUstream s = nullptr;
    if (D.gen_desc(&desc, &grp[used], (unsigned)take[k]) != CUDA_SUCCESS ||
        D.create(&ctx, desc, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) {
      release(p);
      return set_error(FST_ERR_CUDA, std::string(fn) + ": green context creation failed");
    }
    p->ctx.push_back(ctx);
    if (D.stream_create(&s, ctx, CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS) {
      release(p);
      return set_error(FST_ERR_CUDA, std::string(fn) + ": stream creation failed");
    }
    p->stream.push_back(s);
    int sms = 0;
    for (int j = 0; j < take[k]; ++j) sms += (int)grp[used + j].sm.smCount;
    p->sms.push_back(sms);
    used += (unsigned)take[k];
  }
  *out = p;
  return FST_OK;
}

fst_status fst_sm_partition_info(const fst_sm_partition* p, int32_t k, void** stream, int32_t* sm_count) {
  using namespace fst;
  if (!p || k < 0 || k >= (int)p->stream.size())
    return set_error(FST_ERR_INVALID_ARG, "fst_sm_partition_info: no such partition");
  if (stream) *stream = (void*)p->stream[k];
  if (sm_count) *sm_count = p->sms[k];
  return FST_OK;
}

fst_status fst_sm_partition_destroy(fst_sm_partition* p) {
  if (p) release(p);
  return FST_OK;
}

}  // extern "C"
