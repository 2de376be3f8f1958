// Run-time specialised kernels (jit.cpp): which kernels exist per model and
// how to launch them.
#pragma once

#include <cuda_runtime.h>

#include "fst_internal.h"

namespace fst {

// Kernel kinds; bit k of a specialisation mask selects kind k.
enum JitKind {
  JK_FK = 0,
  JK_JACOBIAN,
  JK_RNEA,
  JK_CRBA,
  JK_ABA,
  JK_EVAL,
  JK_FK_VJP,
  JK_RNEA_VJP,
  JK_ABA_VJP,
  JK_LOSS_GRAD,
  JK_EVAL_MIXED,
  JK_RNEA_STORE,
  JK_RNEA_VJP_STORED,
  JK_RNEA_DERIVS,
  JK_ABA_DERIVS,
  JK_COUNT
};
static_assert(JK_COUNT <= 16, "fst_model keeps 16 launch slots");

fst_status jit_specialize(fst_model* m, unsigned mask);
void jit_release(fst_model* m);
unsigned jit_mask(const fst_model* m);
bool jit_has(const fst_model* m, int kind);
// Kernel slots of a kind: 0 one environment per thread, 1 path-parallel with
// a lane per path, 2 path-parallel with a warp per path, 3 SM-pinned (eval),
// 4 the extended fused kernel (eval with the RNEA adjoint, the shared
// kinematics sweep or the packed layouts).
constexpr int JK_SLOTS = 5;
constexpr int JK_SLOT_EVAL_EXT = 4;
bool jit_has_slot(const fst_model* m, int kind, int slot);
int jit_path_lanes(const fst_model* m);   // lanes per environment of slot 1
int jit_path_count(const fst_model* m);   // warps per block of slot 2
cudaError_t jit_launch_slot(const fst_model* m, int kind, int slot, dim3 grid, int block, size_t smem,
                            cudaStream_t s, void** args);
cudaError_t jit_launch(const fst_model* m, int kind, dim3 grid, int block, size_t smem, cudaStream_t s, void** args);
// the same with a block of any shape
cudaError_t jit_launch_slot3(const fst_model* m, int kind, int slot, dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, void** args);

}  // namespace fst
