// One persistent launch over several kinematic trees (fst_multi_eval).
//
// A mixed batch (say 4096 environments of a 7-DOF arm, 2048 of an 11-DOF
// quadruped, ... 256 of a 23-DOF humanoid) would otherwise take one launch
// per tree and operator, each too small to fill the GPU. Here the work is
// cut into items of one tile of environments x one operator x one tree; a
// grid of (SMs x resident blocks) blocks pulls items from an atomic counter
// until none is left. Items are ordered heaviest first (ABA, CRBA, RNEA, FK;
// within an operator the trees with most bodies first), so the long items
// start early and the short ones fill the tail. A block re-stages a tree's
// constants into shared memory only when its next item belongs to another
// tree. The counter is reset by a memset on the same stream before the
// launch, so the pair can be captured into a CUDA graph; there is no
// inter-block waiting of any kind.
#include "launch.h"
#include "level.cuh"
#include "multi.h"

namespace fst {
namespace {

template <int NB>
__global__ void __launch_bounds__(256) multi_kernel(MultiArgs a) {
  extern __shared__ float4 smem[];
  __shared__ int s_item;
  float* tile = reinterpret_cast<float*>(reinterpret_cast<char*>(smem) + a.model_bytes);
  const int T = blockDim.x;
  int cur = -1;
  SmemModel sm{nullptr, nullptr, 0};
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();  // every thread has read s_item before thread 0 can overwrite it for the next item
    if (item >= a.n_items) break;
    int sg = 0;
    while (item >= a.seg_start[sg + 1]) ++sg;
    const int m = a.seg_model[sg];
    const int op = a.seg_op[sg];
    const ModelView& mv = a.mv[m];
    const MultiIO& io = a.io[m];
    if (m != cur) {
      sm = stage_model(mv, smem);  // synchronises the block
      cur = m;
    }
    const int64_t e = (int64_t)(item - a.seg_start[sg]) * T + threadIdx.x;
    if (e < io.B) {
      const int64_t B = io.B;
      const Col cq = stage_rows(tile, io.q, mv.nq, B, e);
      Col c1{}, c2{};
      if (op == ROLE_RNEA) {
        c1 = stage_rows(tile + mv.nq * T, io.qd, mv.nv, B, e);
        c2 = stage_rows(tile + (mv.nq + mv.nv) * T, io.qdd, mv.nv, B, e);
      } else if (op == ROLE_ABA) {
        c1 = stage_rows(tile + mv.nq * T, io.qd, mv.nv, B, e);
        c2 = stage_rows(tile + (mv.nq + mv.nv) * T, io.tau, mv.nv, B, e);
      }
      cp_async_wait_all();
      switch (op) {
        case ROLE_ABA:
          aba_env<NB>(sm, world_accel(mv), cq, c1, c2, io.qdd_out, B, e);
          break;
        case ROLE_CRBA:
          crba_env<NB>(sm, cq, mv.nv, io.M, B, e);
          break;
        case ROLE_RNEA:
          rnea_env<NB>(sm, world_accel(mv), cq, c1, c2, io.tau_out, B, e);
          break;
        default:
          fk_env<NB>(sm, cq, io.poses, B, e);
          break;
      }
    }
    __syncthreads();  // everyone is done with this item's shared memory
  }
}

// The same work list run with the level-parallel bodies (level.cuh): an item
// is 32 environments (one per lane) of one operator on one tree, and the
// block's warps split each of the tree's levels. Shared memory: the largest
// tree's model, the staged input rows, then the per-body state of the
// largest (tree, operator) pair. ABA runs in its lean form (aba_level_lean:
// 14 floats per body and a ring of contributions instead of 59 floats per
// body), so that the block's shared memory, sized for the largest pair, is
// not set by ABA.
__global__ void __launch_bounds__(256) multi_level_kernel(MultiArgs a) {
  extern __shared__ float4 smem[];
  __shared__ int s_item;
  float* tile = reinterpret_cast<float*>(reinterpret_cast<char*>(smem) + a.model_bytes);
  const int lane = threadIdx.x & 31;
  int cur = -1;
  SmemModel sm{nullptr, nullptr, 0};
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();  // every thread has read s_item before thread 0 can overwrite it for the next item
    if (item >= a.n_items) break;
    int sg = 0;
    while (item >= a.seg_start[sg + 1]) ++sg;
    const int m = a.seg_model[sg];
    const int op = a.seg_op[sg];
    const ModelView& mv = a.mv[m];
    const MultiIO& io = a.io[m];
    if (m != cur) {
      sm = stage_model(mv, smem);  // synchronises the block
      cur = m;
    }
    const int64_t B = io.B;
    const int64_t e = (int64_t)(item - a.seg_start[sg]) * kLaneEnvs + lane;
    const bool act = e < B;
    stage_block_rows(tile, io.q, mv.nq, B, e);
    if (op == ROLE_RNEA) {
      stage_block_rows(tile + mv.nq * kLaneEnvs, io.qd, mv.nv, B, e);
      stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, io.qdd, mv.nv, B, e);
    } else if (op == ROLE_ABA) {
      stage_block_rows(tile + mv.nq * kLaneEnvs, io.qd, mv.nv, B, e);
      stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, io.tau, mv.nv, B, e);
    }
    cp_async_wait_all();
    __syncthreads();
    const Col cq{tile + lane, kLaneEnvs};
    const Col c1{tile + mv.nq * kLaneEnvs + lane, kLaneEnvs};
    const Col c2{tile + (mv.nq + mv.nv) * kLaneEnvs + lane, kLaneEnvs};
    float* state = tile + a.max_rows * kLaneEnvs;
    switch (op) {
      case ROLE_ABA:
        aba_level_lean(sm, world_accel(mv), cq, c1, c2, LaneState{state, kAbaLeanBodyFloats},
                       LaneState{state + kAbaLeanBodyFloats * mv.n * kLaneEnvs, kAbaLeanRingFloats}, a.maxw[m],
                       io.qdd_out, B, e, act);
        break;
      case ROLE_CRBA:
        crba_level(sm, cq, mv.nv, LaneState{state, kCrbaState}, io.M, B, e, act);
        break;
      case ROLE_RNEA:
        rnea_level(sm, world_accel(mv), cq, c1, c2, LaneState{state, kRneaState}, io.tau_out, B, e, act);
        break;
      default:
        fk_level(sm, cq, LaneState{state, kFkState}, io.poses, B, e, act);
        break;
    }
    __syncthreads();  // everyone is done with this item's shared memory
  }
}

}  // namespace

// Grid = resident blocks per SM x SMs (from the occupancy calculator), but
// never more blocks than items.
template <typename K>
int persistent_grid(K* kernel, int block, size_t smem, int n_items) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  const int g = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  return g < n_items ? g : n_items;
}

cudaError_t launch_multi(const MultiArgs& a, int max_n, int block, cudaStream_t s) {
  const size_t sh = a.model_bytes + (size_t)a.max_rows * block * sizeof(float);
  cudaError_t err = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (err != cudaSuccess) return err;
  FST_NB_DISPATCH(max_n, prepare(multi_kernel<NB>, sh);
                  const int grid = persistent_grid(multi_kernel<NB>, block, sh, a.n_items);
                  multi_kernel<NB><<<grid, block, sh, s>>>(a));
  return cudaGetLastError();
}

cudaError_t launch_multi_level(const MultiArgs& a, size_t state_bytes, int block, cudaStream_t s) {
  const size_t sh = a.model_bytes + (size_t)a.max_rows * kLaneEnvs * sizeof(float) + state_bytes;
  if (sh > kLevelSmemLimit) return cudaErrorInvalidConfiguration;
  cudaError_t err = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (err != cudaSuccess) return err;
  prepare(multi_level_kernel, sh);
  const int grid = persistent_grid(multi_level_kernel, block, sh, a.n_items);
  multi_level_kernel<<<grid, block, sh, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fst
