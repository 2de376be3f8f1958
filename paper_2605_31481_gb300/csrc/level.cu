// Level-parallel kernels (bodies in level.cuh): tiles of 32 environments,
// W warps per tile splitting each tree level's bodies. A block is one tile
// (1-D, 32 W threads) or T tiles (3-D, (32, T, W); see warp_id()).
//
// Shared memory: model | per tile: input rows (rows x 32) | per-body state
// (F x n x 32); `stride` floats per tile.
#include "launch.h"
#include "level.cuh"

namespace fst {
namespace {

__device__ __forceinline__ float* level_tile(float4* smem, int n) { return smem_tile(smem, n); }

#define FST_LEVEL_PROLOGUE_S(rows, F, stride)                                            \
  extern __shared__ float4 smem[];                                                       \
  float* tile = level_tile(smem, mv.n) + (size_t)threadIdx.y * (stride);                 \
  const LaneState S{tile + (rows) * kLaneEnvs, (F)};                                     \
  const int lane = threadIdx.x & 31;                                                     \
  const int64_t e = ((int64_t)blockIdx.x * blockDim.y + threadIdx.y) * kLaneEnvs + lane; \
  const bool act = e < B

#define FST_LEVEL_PROLOGUE(rows, F) FST_LEVEL_PROLOGUE_S(rows, F, ((rows) + (F) * mv.n) * kLaneEnvs)

// stage_model waits for the model and for this thread's staged rows, then
// synchronises the block, so everything staged is visible to every warp.
#define FST_LEVEL_READY const SmemModel sm = stage_model(mv, smem)

__global__ void __launch_bounds__(256) fk_level_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                       float* __restrict__ poses) {
  FST_LEVEL_PROLOGUE(mv.nq, kFkState);
  stage_block_rows(tile, q, mv.nq, B, e);
  FST_LEVEL_READY;
  fk_level(sm, Col{tile + lane, kLaneEnvs}, S, poses, B, e, act);
}

__global__ void __launch_bounds__(256) jac_level_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                        LinkList links, float* __restrict__ poses,
                                                        float* __restrict__ J) {
  FST_LEVEL_PROLOGUE(mv.nq, kFkState);
  stage_block_rows(tile, q, mv.nq, B, e);
  FST_LEVEL_READY;
  kin_level(sm, Col{tile + lane, kLaneEnvs}, mv.nv, links, S, poses, J, B, e, act);
}

__global__ void __launch_bounds__(256) rnea_level_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                         const float* __restrict__ qd, const float* __restrict__ qdd,
                                                         float* __restrict__ tau) {
  FST_LEVEL_PROLOGUE(mv.nq + 2 * mv.nv, kRneaState);
  stage_block_rows(tile, q, mv.nq, B, e);
  stage_block_rows(tile + mv.nq * kLaneEnvs, qd, mv.nv, B, e);
  stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, qdd, mv.nv, B, e);
  FST_LEVEL_READY;
  rnea_level(sm, world_accel(mv), Col{tile + lane, kLaneEnvs}, Col{tile + mv.nq * kLaneEnvs + lane, kLaneEnvs},
             Col{tile + (mv.nq + mv.nv) * kLaneEnvs + lane, kLaneEnvs}, S, tau, B, e, act);
}

__global__ void __launch_bounds__(256) crba_level_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                         float* __restrict__ M) {
  FST_LEVEL_PROLOGUE(mv.nq, kCrbaState);
  stage_block_rows(tile, q, mv.nq, B, e);
  FST_LEVEL_READY;
  crba_level(sm, Col{tile + lane, kLaneEnvs}, mv.nv, S, M, B, e, act);
}

__global__ void __launch_bounds__(256) aba_level_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                        const float* __restrict__ qd, const float* __restrict__ tau,
                                                        float* __restrict__ qdd) {
  FST_LEVEL_PROLOGUE(mv.nq + 2 * mv.nv, kAbaState);
  stage_block_rows(tile, q, mv.nq, B, e);
  stage_block_rows(tile + mv.nq * kLaneEnvs, qd, mv.nv, B, e);
  stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, tau, mv.nv, B, e);
  FST_LEVEL_READY;
  aba_level(sm, world_accel(mv), Col{tile + lane, kLaneEnvs}, Col{tile + mv.nq * kLaneEnvs + lane, kLaneEnvs},
            Col{tile + (mv.nq + mv.nv) * kLaneEnvs + lane, kLaneEnvs}, S, qdd, B, e, act);
}

// ABA with the lean per-tile state (FST_VARIANT_LEVEL_LEAN): per body
// kAbaLeanBodyFloats, plus a ring of 2 x maxw contribution slots.
__global__ void __launch_bounds__(256) aba_lean_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                       const float* __restrict__ qd, const float* __restrict__ tau,
                                                       float* __restrict__ qdd, int maxw) {
  const int rows = mv.nq + 2 * mv.nv;
  FST_LEVEL_PROLOGUE_S(rows, kAbaLeanBodyFloats,
                       (rows + kAbaLeanBodyFloats * mv.n + 2 * kAbaLeanRingFloats * maxw) * kLaneEnvs);
  const LaneState R{tile + (rows + kAbaLeanBodyFloats * mv.n) * kLaneEnvs, kAbaLeanRingFloats};
  stage_block_rows(tile, q, mv.nq, B, e);
  stage_block_rows(tile + mv.nq * kLaneEnvs, qd, mv.nv, B, e);
  stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, tau, mv.nv, B, e);
  FST_LEVEL_READY;
  aba_level_lean(sm, world_accel(mv), Col{tile + lane, kLaneEnvs}, Col{tile + mv.nq * kLaneEnvs + lane, kLaneEnvs},
                 Col{tile + (mv.nq + mv.nv) * kLaneEnvs + lane, kLaneEnvs}, S, R, maxw, qdd, B, e, act);
}

// CRBA with the lean per-tile state (FST_VARIANT_LEVEL_LEAN): no staged
// rows (q is read from global memory), kCrbaLeanBodyFloats per body, a ring
// of 2 x maxw contribution slots. Up to three blocks per SM.
__global__ void __launch_bounds__(256, 3) crba_lean_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                           float* __restrict__ M, int maxw) {
  FST_LEVEL_PROLOGUE_S(0, kCrbaLeanBodyFloats,
                       (kCrbaLeanBodyFloats * mv.n + 2 * kCrbaLeanRingFloats * maxw) * kLaneEnvs);
  const LaneState R{tile + kCrbaLeanBodyFloats * mv.n * kLaneEnvs, kCrbaLeanRingFloats};
  FST_LEVEL_READY;
  crba_level_lean(sm, q, mv.nv, S, R, maxw, M, B, e, act);
}

// SM-pinned ABA (FST_VARIANT_PINNED): blocks on SMs pinned to ABA take
// tiles of 32 environments until none is left (pinned_tiles). The model is
// staged only by blocks that get work.
__global__ void __launch_bounds__(256) aba_level_pin_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                            const float* __restrict__ qd,
                                                            const float* __restrict__ tau, float* __restrict__ qdd,
                                                            PinArgs p) {
  extern __shared__ float4 smem[];
  float* tile = level_tile(smem, mv.n);
  const LaneState S{tile + (mv.nq + 2 * mv.nv) * kLaneEnvs, kAbaState};
  const int lane = threadIdx.x & 31;
  const int my = pinned_role(p) == ROLE_ABA ? 0 : -1;
  bool staged = false;
  SmemModel sm{nullptr, nullptr, 0};
  auto body = [&](int, int t) {
    if (!staged) {
      sm = stage_model(mv, smem);  // synchronises the block
      staged = true;
    }
    const int64_t e = (int64_t)t * kLaneEnvs + lane;
    const bool act = e < B;
    stage_block_rows(tile, q, mv.nq, B, e);
    stage_block_rows(tile + mv.nq * kLaneEnvs, qd, mv.nv, B, e);
    stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, tau, mv.nv, B, e);
    cp_async_wait_all();
    __syncthreads();
    aba_level(sm, world_accel(mv), Col{tile + lane, kLaneEnvs}, Col{tile + mv.nq * kLaneEnvs + lane, kLaneEnvs},
              Col{tile + (mv.nq + mv.nv) * kLaneEnvs + lane, kLaneEnvs}, S, qdd, B, e, act);
    __syncthreads();  // the next tile reuses the staged rows and the state
  };
  pinned_tiles(p, my, 1, (int)((B + kLaneEnvs - 1) / kLaneEnvs), body);
}

// Fused evaluation with the level-parallel bodies: blockIdx.y is the role.
__global__ void __launch_bounds__(256) eval_level_kernel(ModelView mv, int64_t B, EvalArgs a) {
  const int role = a.roles[blockIdx.y];
  const int F = role == ROLE_ABA ? kAbaState : role == ROLE_CRBA ? kCrbaState : role == ROLE_RNEA ? kRneaState : kFkState;
  // tiles are sized for the largest role (ABA), as the launch allocates them
  FST_LEVEL_PROLOGUE_S(mv.nq + 2 * mv.nv, F, (mv.nq + 2 * mv.nv + kAbaState * mv.n) * kLaneEnvs);
  stage_block_rows(tile, a.q, mv.nq, B, e);
  if (role == ROLE_RNEA) {
    stage_block_rows(tile + mv.nq * kLaneEnvs, a.qd, mv.nv, B, e);
    stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, a.qdd, mv.nv, B, e);
  } else if (role == ROLE_ABA) {
    stage_block_rows(tile + mv.nq * kLaneEnvs, a.qd, mv.nv, B, e);
    stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, a.tau, mv.nv, B, e);
  }
  FST_LEVEL_READY;
  const Col cq{tile + lane, kLaneEnvs};
  const Col c1{tile + mv.nq * kLaneEnvs + lane, kLaneEnvs};
  const Col c2{tile + (mv.nq + mv.nv) * kLaneEnvs + lane, kLaneEnvs};
  switch (role) {
    case ROLE_ABA:
      aba_level(sm, world_accel(mv), cq, c1, c2, S, a.qdd_out, B, e, act);
      break;
    case ROLE_CRBA:
      crba_level(sm, cq, mv.nv, S, a.M, B, e, act);
      break;
    case ROLE_RNEA:
      rnea_level(sm, world_accel(mv), cq, c1, c2, S, a.tau_out, B, e, act);
      break;
    default:
      kin_level(sm, cq, mv.nv, a.links, S, a.poses, a.J, B, e, act);
      break;
  }
}

// bytes of shared memory of one tile: input rows and per-body state
size_t level_tile_bytes(const ModelView& mv, int rows, int F) {
  return (size_t)rows * kLaneEnvs * sizeof(float) + (size_t)F * mv.n * kLaneEnvs * sizeof(float);
}

// `block` threads (a multiple of 32 T) as `tiles` tiles of block / (32 T)
// warps each: a 1-D block for one tile, (32, T, W) for several.
template <typename K, typename... A>
cudaError_t go(K* kernel, const ModelView& mv, int64_t B, size_t sh, int block, int tiles, unsigned gy,
               cudaStream_t s, A... args) {
  if (sh > kLevelSmemLimit || tiles < 1 || block < 32 * tiles || block % (32 * tiles))
    return cudaErrorInvalidConfiguration;
  prepare(kernel, sh);
  const int64_t envs = (int64_t)kLaneEnvs * tiles;
  const dim3 blk = tiles == 1 ? dim3(block) : dim3(32, tiles, block / (32 * tiles));
  kernel<<<dim3((unsigned)((B + envs - 1) / envs), gy), blk, sh, s>>>(mv, B, args...);
  return cudaGetLastError();
}

}  // namespace

size_t model_smem_bytes(int n) { return smem_bytes(n); }

size_t level_smem_needed(const ModelView& mv, int kind, int tiles) {
  size_t t;
  switch (kind) {
    case LEVEL_FK:
    case LEVEL_JAC:
      t = level_tile_bytes(mv, mv.nq, kFkState);
      break;
    case LEVEL_RNEA:
      t = level_tile_bytes(mv, mv.nq + 2 * mv.nv, kRneaState);
      break;
    case LEVEL_CRBA:
      t = level_tile_bytes(mv, mv.nq, kCrbaState);
      break;
    default:  // ABA, and eval (its tiles are sized for the ABA role)
      t = level_tile_bytes(mv, mv.nq + 2 * mv.nv, kAbaState);
      break;
  }
  return smem_bytes(mv.n) + (size_t)tiles * t;
}

cudaError_t launch_fk_level(const ModelView& mv, int64_t B, const float* q, float* poses, int block, int tiles,
                            cudaStream_t s) {
  return go(fk_level_kernel, mv, B, level_smem_needed(mv, LEVEL_FK, tiles), block, tiles, 1, s, q, poses);
}
cudaError_t launch_jac_level(const ModelView& mv, int64_t B, const float* q, const LinkList& links, float* J,
                             int block, int tiles, cudaStream_t s) {
  return go(jac_level_kernel, mv, B, level_smem_needed(mv, LEVEL_JAC, tiles), block, tiles, 1, s, q, links,
            (float*)nullptr, J);
}
cudaError_t launch_rnea_level(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                              float* tau, int block, int tiles, cudaStream_t s) {
  return go(rnea_level_kernel, mv, B, level_smem_needed(mv, LEVEL_RNEA, tiles), block, tiles, 1, s, q, qd, qdd, tau);
}
cudaError_t launch_crba_level(const ModelView& mv, int64_t B, const float* q, float* M, int block, int tiles,
                              cudaStream_t s) {
  return go(crba_level_kernel, mv, B, level_smem_needed(mv, LEVEL_CRBA, tiles), block, tiles, 1, s, q, M);
}
cudaError_t launch_aba_level(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                             float* qdd, int block, int tiles, cudaStream_t s) {
  return go(aba_level_kernel, mv, B, level_smem_needed(mv, LEVEL_ABA, tiles), block, tiles, 1, s, q, qd, tau, qdd);
}
size_t aba_lean_smem_needed(const ModelView& mv, int maxw, int tiles) {
  const size_t t = level_tile_bytes(mv, mv.nq + 2 * mv.nv, kAbaLeanBodyFloats) +
                   (size_t)2 * kAbaLeanRingFloats * maxw * kLaneEnvs * sizeof(float);
  return smem_bytes(mv.n) + (size_t)tiles * t;
}
cudaError_t launch_aba_level_lean(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                                  float* qdd, int block, int maxw, cudaStream_t s) {
  return go(aba_lean_kernel, mv, B, aba_lean_smem_needed(mv, maxw, 1), block, 1, 1, s, q, qd, tau, qdd, maxw);
}
size_t crba_lean_smem_needed(const ModelView& mv, int maxw) {
  return smem_bytes(mv.n) +
         (size_t)(kCrbaLeanBodyFloats * mv.n + 2 * kCrbaLeanRingFloats * maxw) * kLaneEnvs * sizeof(float);
}
cudaError_t launch_crba_level_lean(const ModelView& mv, int64_t B, const float* q, float* M, int block, int maxw,
                                   cudaStream_t s) {
  return go(crba_lean_kernel, mv, B, crba_lean_smem_needed(mv, maxw), block, 1, 1, s, q, M, maxw);
}
cudaError_t launch_aba_level_pinned(const ModelView& mv, int64_t B, const float* q, const float* qd,
                                    const float* tau, float* qdd, int block, const PinArgs& p, cudaStream_t s) {
  const size_t sh = level_smem_needed(mv, LEVEL_ABA);
  if (sh > kLevelSmemLimit) return cudaErrorInvalidConfiguration;
  prepare(aba_level_pin_kernel, sh);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  aba_level_pin_kernel<<<2 * (sms > 0 ? sms : 1), block, sh, s>>>(mv, B, q, qd, tau, qdd, p);
  return cudaGetLastError();
}

cudaError_t launch_eval_level(const ModelView& mv, int64_t B, const EvalArgs& a, int block, int tiles,
                              cudaStream_t s) {
  return go(eval_level_kernel, mv, B, level_smem_needed(mv, LEVEL_EVAL, tiles), block, tiles, (unsigned)a.n_roles, s,
            a);
}

}  // namespace fst
