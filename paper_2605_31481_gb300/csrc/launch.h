// Launch helpers shared by the kernel translation units and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>
#include <unordered_map>

#include "fst_internal.h"

namespace fst {

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

// Per-kernel launch attributes, set once per kernel (and again only when a
// launch needs more dynamic shared memory than configured so far):
//  * the dynamic shared-memory limit, when above the 48 KB default;
//  * the shared-memory carveout: just enough shared memory for ~4 resident
//    blocks, leaving the rest of the 256 KB unified L1 for the per-thread
//    sweep state (local memory). FST_SMEM_CARVEOUT=<percent> overrides it.
// Library-wide carveout override (fst_set_smem_carveout): -1 = per kernel,
// else the percentage for every kernel; `generation` changes on every set so
// kernels pick the new value up at their next launch.
int carveout_override();
int carveout_generation();

template <typename K>
inline void prepare(K* kernel, size_t smem) {
  struct Done {
    size_t smem;
    int gen;
  };
  static std::mutex mu;
  static std::unordered_map<const void*, Done> done;
  const int gen = carveout_generation();
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find((const void*)kernel);
  if (it != done.end() && it->second.smem >= smem && it->second.gen == gen) return;
  // The attribute only ever grows: a launch of another model with less
  // shared memory must not shrink the limit a larger one already relies on.
  const size_t keep = (it != done.end() && it->second.smem > smem) ? it->second.smem : smem;
  if (keep > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)keep);
  int pct = (int)((4 * keep * 100 + 228 * 1024 - 1) / (228 * 1024));
  if (const char* env = std::getenv("FST_SMEM_CARVEOUT")) pct = std::atoi(env);
  if (carveout_override() >= 0) pct = carveout_override();
  pct = pct < 0 ? 0 : (pct > 100 ? 100 : pct);
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  done[(const void*)kernel] = Done{keep, gen};
}

// Kernel launchers (return the cudaGetLastError() after the launch).
cudaError_t launch_fk(const ModelView& mv, int64_t B, const float* q, float* poses, const Launch& L);
cudaError_t launch_jacobian(const ModelView& mv, int64_t B, const float* q, const LinkList& links, float* J,
                            const Launch& L);
cudaError_t launch_rnea(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                        float* tau, const Launch& L);
cudaError_t launch_crba(const ModelView& mv, int64_t B, const float* q, float* M,
                        const Launch& L);
cudaError_t launch_eval(const ModelView& mv, int64_t B, const EvalArgs& a, const Launch& L);
cudaError_t launch_aba(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                       float* qdd, const Launch& L);

// Level-parallel kernels (level.cu): tiles of 32 environments, the warps of
// a tile splitting each tree level's bodies; per-body state in shared memory.
enum LevelKind { LEVEL_FK = 0, LEVEL_JAC, LEVEL_RNEA, LEVEL_CRBA, LEVEL_ABA, LEVEL_EVAL };
constexpr size_t kLevelSmemLimit = 227 * 1024;

// Floats per body and environment on the store-variant RNEA tape (X 12, v 6, a 6, F 6).
constexpr int kTapeFloatsPerBody = 30;
// `tiles` tiles of 32 environments per block (1, or 2 for FST_VARIANT_LEVEL2),
// `block` threads in all.
size_t level_smem_needed(const ModelView& mv, int kind, int tiles = 1);
// Bytes of the model copy a kernel stages in shared memory (stage_model).
size_t model_smem_bytes(int n);
cudaError_t launch_fk_level(const ModelView& mv, int64_t B, const float* q, float* poses, int block, int tiles,
                            cudaStream_t s);
cudaError_t launch_jac_level(const ModelView& mv, int64_t B, const float* q, const LinkList& links, float* J,
                             int block, int tiles, cudaStream_t s);
cudaError_t launch_rnea_level(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                              float* tau, int block, int tiles, cudaStream_t s);
cudaError_t launch_crba_level(const ModelView& mv, int64_t B, const float* q, float* M, int block, int tiles,
                              cudaStream_t s);
cudaError_t launch_aba_level(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                             float* qdd, int block, int tiles, cudaStream_t s);
cudaError_t launch_eval_level(const ModelView& mv, int64_t B, const EvalArgs& a, int block, int tiles,
                              cudaStream_t s);
// The lean level-parallel ABA (FST_VARIANT_LEVEL_LEAN); maxw = bodies of the
// widest tree level.
size_t aba_lean_smem_needed(const ModelView& mv, int maxw, int tiles = 1);
cudaError_t launch_aba_level_lean(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                                  float* qdd, int block, int maxw, cudaStream_t s);
// The lean level-parallel CRBA (FST_VARIANT_LEVEL_LEAN).
size_t crba_lean_smem_needed(const ModelView& mv, int maxw);
cudaError_t launch_crba_level_lean(const ModelView& mv, int64_t B, const float* q, float* M, int block, int maxw,
                                   cudaStream_t s);

// Adjoints (adjoint.cu). scratch: vjp_scratch_floats(n, B) floats of device
// memory for the per-block partial sums of thetabar (and the loss).
size_t vjp_scratch_floats(int n, int64_t B);
// out[p] = sum over b < nblk of partial[b * P + p] (in block order)
cudaError_t launch_partial_reduce(const float* partial, int nblk, int P, float* out, cudaStream_t s);
cudaError_t launch_fk_vjp(const ModelView& mv, int64_t B, const float* q, const float* pbar, float* qbar,
                          cudaStream_t s);
cudaError_t launch_rnea_vjp(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                            const float* tbar, float* qbar, float* qdbar, float* qddbar, float* thbar, float* scratch,
                            cudaStream_t s);
cudaError_t launch_rnea_store(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                              float* tau, float* tape, const Launch& L);
cudaError_t launch_rnea_vjp_stored(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tape,
                                   const float* tbar, float* qbar, float* qdbar, float* qddbar, float* thbar,
                                   float* scratch, cudaStream_t s);
cudaError_t launch_rnea_derivs(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                               float* dq, float* dqd, const Launch& L);
cudaError_t launch_aba_derivs(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                              float* qdd, float* dq, float* dqd, float* Minv, const Launch& L);
cudaError_t launch_jac_vjp(const ModelView& mv, int64_t B, const float* q, const LinkList& links, const float* Jbar,
                           float* qbar, cudaStream_t s);
cudaError_t launch_crba_vjp(const ModelView& mv, int64_t B, const float* q, const float* Mbar, float* qbar,
                            float* thbar, float* scratch, cudaStream_t s);
cudaError_t launch_aba_level_pinned(const ModelView& mv, int64_t B, const float* q, const float* qd,
                                    const float* tau, float* qdd, int block, const PinArgs& p, cudaStream_t s);
cudaError_t launch_aba_vjp(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                           const float* qddbar, float* qbar, float* qdbar, float* taubar, float* thbar, float* scratch,
                           cudaStream_t s);
cudaError_t launch_rnea_loss_grad(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                                  const float* tau_meas, float* loss_theta, float* qbar, float* qdbar, float* scratch,
                                  cudaStream_t s);

}  // namespace fst
