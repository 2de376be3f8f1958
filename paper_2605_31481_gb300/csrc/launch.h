// Launch helpers shared by the kernel translation units and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "fst_internal.h"

namespace fst {

struct LinkList {
  int n;
  int idx[FST_MAX_LINKS];
};

struct Launch {
  int block;          // threads per block (environments per block for 1 env/thread)
  cudaStream_t stream;
};

// Threads per block for B environments, one environment per thread. Small
// batches use 32-thread blocks so the blocks spread over all 152 SMs.
inline int default_block(int64_t B) {
  if (B <= 152 * 32) return 32;
  if (B <= 152 * 64 * 2) return 64;
  return 128;
}

// Instantiates a kernel template for the smallest per-thread body capacity
// NB in {16, 32, 64} that holds n bodies.
#define FST_NB_DISPATCH(n, ...)        \
  do {                                 \
    if ((n) <= 16) {                   \
      constexpr int NB = 16;           \
      __VA_ARGS__;                     \
    } else if ((n) <= 32) {            \
      constexpr int NB = 32;           \
      __VA_ARGS__;                     \
    } else {                           \
      constexpr int NB = 64;           \
      __VA_ARGS__;                     \
    }                                  \
  } while (0)

inline unsigned grid_for(int64_t B, int block) { return (unsigned)((B + block - 1) / block); }

// Kernel launchers (return the cudaGetLastError() after the launch).
cudaError_t launch_fk(const ModelView& mv, int64_t B, const float* q, float* poses, const Launch& L);
cudaError_t launch_jacobian(const ModelView& mv, int64_t B, const float* q, const LinkList& links, float* J,
                            const Launch& L);
cudaError_t launch_rnea(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                        float* tau, const Launch& L);
cudaError_t launch_crba(const ModelView& mv, int64_t B, const float* q, float* M,
                        const Launch& L);
cudaError_t launch_aba(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                       float* qdd, const Launch& L);

}  // namespace fst
