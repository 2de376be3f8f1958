// Kernels specialised for one fixed tree, compiled at run time by NVRTC.
//
// The host generator (jit.cpp) writes a prelude that defines FST_N (the
// number of bodies), the model constants kC/kI as initialised device
// constants, one FST_JIT_* macro selecting the kernel to build and
// FST_JIT_NAME, its exported name, then includes this file. The kernels call the same operator templates as the
// generic kernels, with a compile-time topology: every body loop is fully
// unrolled, every parent index is a constant, and the per-body sweep state
// lives in registers instead of per-thread local memory. Only the inertial
// parameters are read at run time (from the override or the model's device
// copy), so one compiled module serves every parameter set.
#pragma once

#include "adjoint.cuh"
#include "derivs.cuh"
#include "level.cuh"
#include "pathpar.cuh"

namespace fst {

struct FixedTopo {
  const float* th;  // inertial parameters of body k at th + k * ts
  int ts;
  __device__ __forceinline__ static constexpr int n() { return FST_N; }
  __device__ __forceinline__ const BodyC& C(int k) const { return kC[k]; }
  __device__ __forceinline__ BodyI I(int k) const { return kI[k]; }
  __device__ __forceinline__ const float* theta(int k) const { return th + k * ts; }
  __device__ __forceinline__ static constexpr int depth() { return FST_DEPTH; }
  __device__ __forceinline__ int level_begin(int l) const { return kLevelStart[l]; }
  __device__ __forceinline__ int level_body(int k) const { return kLevelBody[k]; }
  __device__ __forceinline__ int child_begin(int k) const { return kChildStart[k]; }
  __device__ __forceinline__ int child(int k) const { return kChild[k]; }
#if FST_PATH_G > 0
  // root-to-leaf paths, one per lane (path-parallel variant)
  __device__ __forceinline__ int path(int g, int t) const { return kPath[g * FST_DEPTH + t]; }
  __device__ __forceinline__ int seg(int g, int t) const { return kSeg[g * FST_DEPTH + t]; }
  __device__ __forceinline__ unsigned lead_mask(int g) const { return kLead[g]; }
  __device__ __forceinline__ bool red(int t) const { return kRed[t] != 0; }
  __device__ __forceinline__ int owner(int i) const { return kOwner[i]; }
  __device__ __forceinline__ int depth_of(int i) const { return kDepthOf[i]; }
#endif
};

__device__ __forceinline__ FixedTopo fixed_topo(const ModelView& mv) {
  if (mv.theta) return FixedTopo{mv.theta, 10};
  return FixedTopo{mv.c[0].theta, (int)(sizeof(BodyC) / sizeof(float))};
}

__device__ __forceinline__ Col jit_stage_or_zero(float* tile, const float* __restrict__ src, int rows, int64_t B,
                                                 int64_t e, bool act) {
  if (act) return stage_rows(tile, src, rows, B, e);
  float* dst = tile + threadIdx.x;
  for (int k = 0; k < rows; ++k) dst[k * blockDim.x] = 0.f;
  return Col{dst, (int)blockDim.x};
}

__device__ __forceinline__ void jit_write_partial(const float* slots, int P, float* partial) {
  const int warps = blockDim.x / 32;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < warps; ++w) s += slots[w * P + p];
    partial[(int64_t)blockIdx.x * P + p] = s;
  }
}

}  // namespace fst

using namespace fst;

#define FST_JIT_PROLOGUE                                              \
  extern __shared__ float4 smem[];                                    \
  float* tile = reinterpret_cast<float*>(smem);                       \
  const int T = blockDim.x;                                           \
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;            \
  const bool act = e < B;                                             \
  (void)T;                                                            \
  (void)act

#ifdef FST_JIT_FK
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 float* __restrict__ poses) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  cp_async_wait_all();
  fk_env<FST_N>(fixed_topo(mv), cq, poses, B, e);
}
#endif

#ifdef FST_JIT_JACOBIAN
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 LinkList links, float* __restrict__ J) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  cp_async_wait_all();
  jac_env<FST_N>(fixed_topo(mv), cq, mv.nv, links, nullptr, J, B, e);
}
#endif

#ifdef FST_JIT_RNEA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ qdd,
                                                                 float* __restrict__ tau) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  const Col cqd = stage_rows(tile + mv.nq * T, qd, mv.nv, B, e);
  const Col cqdd = stage_rows(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e);
  cp_async_wait_all();
  rnea_env<FST_N>(fixed_topo(mv), world_accel(mv), cq, cqd, cqdd, tau, B, e);
}
#endif

#ifdef FST_JIT_CRBA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 float* __restrict__ M) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  cp_async_wait_all();
  crba_env<FST_N>(fixed_topo(mv), cq, mv.nv, M, B, e);
}
#endif

#ifdef FST_JIT_ABA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ tau,
                                                                 float* __restrict__ qdd) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  const Col cqd = stage_rows(tile + mv.nq * T, qd, mv.nv, B, e);
  const Col ctau = stage_rows(tile + (mv.nq + mv.nv) * T, tau, mv.nv, B, e);
  cp_async_wait_all();
  aba_env<FST_N>(fixed_topo(mv), world_accel(mv), cq, cqd, ctau, qdd, B, e);
}
#endif

#ifdef FST_JIT_EVAL
// The fused evaluation: blockIdx.y is the role (one operator per group of
// blocks), one environment per thread.
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, EvalArgs a) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const int role = a.roles[blockIdx.y];
  const Col cq = stage_rows(tile, a.q, mv.nq, B, e);
  Col c1{}, c2{};
  if (role == ROLE_RNEA) {
    c1 = stage_rows(tile + mv.nq * T, a.qd, mv.nv, B, e);
    c2 = stage_rows(tile + (mv.nq + mv.nv) * T, a.qdd, mv.nv, B, e);
  } else if (role == ROLE_ABA) {
    c1 = stage_rows(tile + mv.nq * T, a.qd, mv.nv, B, e);
    c2 = stage_rows(tile + (mv.nq + mv.nv) * T, a.tau, mv.nv, B, e);
  }
  cp_async_wait_all();
  const FixedTopo tp = fixed_topo(mv);
  switch (role) {
    case ROLE_ABA:
      aba_env<FST_N>(tp, world_accel(mv), cq, c1, c2, a.qdd_out, B, e);
      break;
    case ROLE_CRBA:
      crba_env<FST_N>(tp, cq, mv.nv, a.M, B, e);
      break;
    case ROLE_RNEA:
      rnea_env<FST_N>(tp, world_accel(mv), cq, c1, c2, a.tau_out, B, e);
      break;
    default:
      if (a.J)
        jac_env<FST_N>(tp, cq, mv.nv, a.links, a.poses, a.J, B, e);
      else
        fk_env<FST_N>(tp, cq, a.poses, B, e);
      break;
  }
}

// The extended fused evaluation (a separate kernel, so that the plain one
// above keeps its registers and code size): the RNEA role with the adjoint
// and/or the kinematics from its own sweep (a.rnea_flags), and M and J in
// the packed layouts (a.packed). The rows past q, qd and qdd hold tau_bar.
extern "C" __global__ void __launch_bounds__(256) FST_JIT_EXT_NAME(ModelView mv, int64_t B, EvalArgs a) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const int role = a.roles[blockIdx.y];
  const Col cq = stage_rows(tile, a.q, mv.nq, B, e);
  Col c1{}, c2{};
  if (role == ROLE_RNEA) {
    c1 = stage_rows(tile + mv.nq * T, a.qd, mv.nv, B, e);
    c2 = stage_rows(tile + (mv.nq + mv.nv) * T, a.qdd, mv.nv, B, e);
    if ((a.rnea_flags & EVAL_RNEA_VJP) && !(a.rnea_flags & EVAL_TBAR_IS_TAU))
      stage_rows(tile + (mv.nq + 2 * mv.nv) * T, a.tau_bar, mv.nv, B, e);
  } else if (role == ROLE_ABA) {
    c1 = stage_rows(tile + mv.nq * T, a.qd, mv.nv, B, e);
    c2 = stage_rows(tile + (mv.nq + mv.nv) * T, a.tau, mv.nv, B, e);
  }
  cp_async_wait_all();
  const FixedTopo tp = fixed_topo(mv);
  switch (role) {
    case ROLE_ABA:
      aba_env<FST_N>(tp, world_accel(mv), cq, c1, c2, a.qdd_out, B, e);
      break;
    case ROLE_CRBA:
      if (a.packed)
        crba_env<FST_N, true>(tp, cq, mv.nv, a.M, B, e);
      else
        crba_env<FST_N>(tp, cq, mv.nv, a.M, B, e);
      break;
    case ROLE_RNEA:
      if (a.rnea_flags)
        rnea_role_env<FST_N>(tp, world_accel(mv), cq, c1, c2, tile + (mv.nq + 2 * mv.nv) * T + threadIdx.x, T,
                             mv.nv, a, B, e);
      else
        rnea_env<FST_N>(tp, world_accel(mv), cq, c1, c2, a.tau_out, B, e);
      break;
    default:
      if (a.J)
        jac_env<FST_N>(tp, cq, mv.nv, a.links, a.poses, a.J, B, e, a.packed ? &a.pj : nullptr);
      else
        fk_env<FST_N>(tp, cq, a.poses, B, e);
      break;
  }
}
#endif

#ifdef FST_JIT_EVAL
// SM-pinned fused step (FST_VARIANT_PINNED): ONE launch of one block per SM,
// each block serving the role its SM is pinned to (pinned_role), tile after
// tile (pinned_tiles), so that an SM runs the same straight-line code from
// launch to launch and finds it in its instruction caches: when consecutive
// launches hand an SM another role's code, it refetches that code and the
// launch takes about twice as long. Blocks are (32, 2, 4): 256 threads, as
// two tiles of 32 environments with four warps each.
//  * KIN, RNEA and CRBA: one environment per thread, p.envs[slot] (<= 256)
//    environments per tile;
//  * ABA: level-parallel (level.cuh), 64 environments per tile as two tiles
//    of 32, each tile's four warps splitting every level.
// Dynamic shared memory: the model, then two ABA tiles (input rows and
// per-body state) or the staged input rows of 256 environments, whichever is
// larger.
extern "C" __global__ void __launch_bounds__(256) FST_JIT_PIN_NAME(ModelView mv, int64_t B, EvalArgs a, PinArgs p) {
  extern __shared__ float4 smem[];
  // ABA runs the level-parallel bodies over the model staged in shared memory
  // (compact loops: the fully unrolled form of the compiled-in tree runs about
  // twice as long here)
  const SmemModel sm = stage_model(mv, smem);
  float* base = smem_tile(smem, mv.n);
  const int tid = threadIdx.x + 32 * (threadIdx.y + 2 * threadIdx.z);
  const int code = pinned_role(p);
  int my = -1;
  for (int r = 0; r < a.n_roles; ++r)
    if (a.roles[r] == code) my = r;
  const FixedTopo tp = fixed_topo(mv);
  const int rows = mv.nq + 2 * mv.nv;
  auto body = [&](int slot, int t) {
    const int role = a.roles[slot];
    if (role == ROLE_ABA) {
      const int lane = threadIdx.x;
      float* tile = base + (size_t)threadIdx.y * (rows + kAbaState * mv.n) * kLaneEnvs;
      const LaneState S{tile + rows * kLaneEnvs, kAbaState};
      const int64_t e = ((int64_t)t * 2 + threadIdx.y) * kLaneEnvs + lane;
      stage_block_rows(tile, a.q, mv.nq, B, e);
      stage_block_rows(tile + mv.nq * kLaneEnvs, a.qd, mv.nv, B, e);
      stage_block_rows(tile + (mv.nq + mv.nv) * kLaneEnvs, a.tau, mv.nv, B, e);
      cp_async_wait_all();
      __syncthreads();
      aba_level(sm, world_accel(mv), Col{tile + lane, kLaneEnvs}, Col{tile + mv.nq * kLaneEnvs + lane, kLaneEnvs},
                Col{tile + (mv.nq + mv.nv) * kLaneEnvs + lane, kLaneEnvs}, S, a.qdd_out, B, e, e < B);
    } else {
      const int E = p.envs[slot];
      const int64_t e = (int64_t)t * E + tid;
      if (tid < E && e < B) {
        float* col = base + tid;
        for (int k = 0; k < mv.nq; ++k) cp_async4(col + k * 256, a.q + (int64_t)k * B + e);
        if (role == ROLE_RNEA) {
          for (int k = 0; k < mv.nv; ++k) {
            cp_async4(col + (mv.nq + k) * 256, a.qd + (int64_t)k * B + e);
            cp_async4(col + (mv.nq + mv.nv + k) * 256, a.qdd + (int64_t)k * B + e);
          }
        }
        cp_async_wait_all();
        const Col cq{col, 256}, c1{col + mv.nq * 256, 256}, c2{col + (mv.nq + mv.nv) * 256, 256};
        switch (role) {
          case ROLE_CRBA:
            crba_env<FST_N>(tp, cq, mv.nv, a.M, B, e);
            break;
          case ROLE_RNEA:
            rnea_env<FST_N>(tp, world_accel(mv), cq, c1, c2, a.tau_out, B, e);
            break;
          default:
            if (a.J)
              jac_env<FST_N>(tp, cq, mv.nv, a.links, a.poses, a.J, B, e);
            else
              fk_env<FST_N>(tp, cq, a.poses, B, e);
            break;
        }
      }
    }
    __syncthreads();  // the next tile reuses the shared memory
  };
  pinned_tiles(p, my, a.n_roles, p.tiles, body);
}
#endif

#ifdef FST_JIT_EVAL_MIXED
// Roles in a.level_mask run level-parallel (32 environments per block, the
// block's warps splitting each tree level); the others one environment per
// thread. The grid's x extent covers the larger of the two; blocks past a
// role's last environment leave at once (block-uniform, before any barrier).
// A level-parallel role runs on a copy of the model staged in shared memory
// (run-time topology), as the operator's own level-parallel kernel does: its
// per-level loops are compact code that every warp shares, where the
// compiled-in tree would unroll every body of every level into each warp's
// instruction stream; its tile follows the model copy.
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, EvalArgs a) {
  extern __shared__ float4 smem[];
  float* tile = reinterpret_cast<float*>(smem);
  const int role = a.roles[blockIdx.y];
  const FixedTopo tp = fixed_topo(mv);
  if ((a.level_mask >> role) & 1) {
    if ((int64_t)blockIdx.x * kLaneEnvs >= B) return;
    const int lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * kLaneEnvs + lane;
    const bool act = e < B;
    float* ltile = smem_tile(smem, mv.n);
    const int F = role == ROLE_ABA ? kAbaState : role == ROLE_CRBA ? kCrbaState : role == ROLE_RNEA ? kRneaState : kFkState;
    const LaneState S{ltile + (mv.nq + 2 * mv.nv) * kLaneEnvs, F};
    stage_block_rows(ltile, a.q, mv.nq, B, e);
    if (role == ROLE_RNEA) {
      stage_block_rows(ltile + mv.nq * kLaneEnvs, a.qd, mv.nv, B, e);
      stage_block_rows(ltile + (mv.nq + mv.nv) * kLaneEnvs, a.qdd, mv.nv, B, e);
    } else if (role == ROLE_ABA) {
      stage_block_rows(ltile + mv.nq * kLaneEnvs, a.qd, mv.nv, B, e);
      stage_block_rows(ltile + (mv.nq + mv.nv) * kLaneEnvs, a.tau, mv.nv, B, e);
    }
    const SmemModel sm = stage_model(mv, smem);  // also waits for the staged rows, and synchronises
    const Col cq{ltile + lane, kLaneEnvs};
    const Col c1{ltile + mv.nq * kLaneEnvs + lane, kLaneEnvs};
    const Col c2{ltile + (mv.nq + mv.nv) * kLaneEnvs + lane, kLaneEnvs};
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
    return;
  }
  const int T = blockDim.x;
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  if (e >= B) return;
  const Col cq = stage_rows(tile, a.q, mv.nq, B, e);
  Col c1{}, c2{};
  if (role == ROLE_RNEA) {
    c1 = stage_rows(tile + mv.nq * T, a.qd, mv.nv, B, e);
    c2 = stage_rows(tile + (mv.nq + mv.nv) * T, a.qdd, mv.nv, B, e);
  } else if (role == ROLE_ABA) {
    c1 = stage_rows(tile + mv.nq * T, a.qd, mv.nv, B, e);
    c2 = stage_rows(tile + (mv.nq + mv.nv) * T, a.tau, mv.nv, B, e);
  }
  cp_async_wait_all();
  switch (role) {
    case ROLE_ABA:
      aba_env<FST_N>(tp, world_accel(mv), cq, c1, c2, a.qdd_out, B, e);
      break;
    case ROLE_CRBA:
      crba_env<FST_N>(tp, cq, mv.nv, a.M, B, e);
      break;
    case ROLE_RNEA:
      rnea_env<FST_N>(tp, world_accel(mv), cq, c1, c2, a.tau_out, B, e);
      break;
    default:
      if (a.J)
        jac_env<FST_N>(tp, cq, mv.nv, a.links, a.poses, a.J, B, e);
      else
        fk_env<FST_N>(tp, cq, a.poses, B, e);
      break;
  }
}
#endif

#ifdef FST_JIT_FK_VJP
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ pbar,
                                                                 float* __restrict__ qbar) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  const Col cpb = stage_rows(tile + mv.nq * T, pbar, mv.n * 12, B, e);
  cp_async_wait_all();
  fk_vjp_env<FST_N>(fixed_topo(mv), cq, cpb, qbar, B, e);
}
#endif

#ifdef FST_JIT_RNEA_VJP
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ qdd,
                                                                 const float* __restrict__ tbar, float* qbar,
                                                                 float* qdbar, float* qddbar, float* partial) {
  FST_JIT_PROLOGUE;
  const int rows = mv.nq + 3 * mv.nv;
  const Col cq = jit_stage_or_zero(tile, q, mv.nq, B, e, act);
  const Col cqd = jit_stage_or_zero(tile + mv.nq * T, qd, mv.nv, B, e, act);
  const Col cqdd = jit_stage_or_zero(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e, act);
  const Col ctb = jit_stage_or_zero(tile + (mv.nq + 2 * mv.nv) * T, tbar, mv.nv, B, e, act);
  const int P = FST_N * 10;
  float* slots = partial ? tile + rows * T : nullptr;
  if (slots)
    for (int k = threadIdx.x; k < (T / 32) * P; k += T) slots[k] = 0.f;
  cp_async_wait_all();
  __syncthreads();
  VjpOut o{qbar, qdbar, qddbar, slots ? slots + (threadIdx.x / 32) * P : nullptr, 1.f, act};
  rnea_vjp_env<FST_N>(fixed_topo(mv), world_accel(mv), cq, cqd, cqdd, ctb, o, B, e);
  if (partial) {
    __syncthreads();
    jit_write_partial(slots, P, partial);
  }
}
#endif

#ifdef FST_JIT_RNEA_STORE
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ qdd, float* __restrict__ tau,
                                                                 float* __restrict__ tape) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  const Col cqd = stage_rows(tile + mv.nq * T, qd, mv.nv, B, e);
  const Col cqdd = stage_rows(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e);
  cp_async_wait_all();
  rnea_store_env<FST_N>(fixed_topo(mv), world_accel(mv), cq, cqd, cqdd, tau, tape, B, e);
}
#endif

#ifdef FST_JIT_RNEA_VJP_STORED
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ tape,
                                                                 const float* __restrict__ tbar, float* qbar,
                                                                 float* qdbar, float* qddbar, float* partial) {
  FST_JIT_PROLOGUE;
  const int rows = mv.nq + 2 * mv.nv;
  const Col cq = jit_stage_or_zero(tile, q, mv.nq, B, e, act);
  const Col cqd = jit_stage_or_zero(tile + mv.nq * T, qd, mv.nv, B, e, act);
  const Col ctb = jit_stage_or_zero(tile + (mv.nq + mv.nv) * T, tbar, mv.nv, B, e, act);
  const int P = FST_N * 10;
  float* slots = partial ? tile + rows * T : nullptr;
  if (slots)
    for (int k = threadIdx.x; k < (T / 32) * P; k += T) slots[k] = 0.f;
  cp_async_wait_all();
  __syncthreads();
  VjpOut o{qbar, qdbar, qddbar, slots ? slots + (threadIdx.x / 32) * P : nullptr, 1.f, act};
  rnea_vjp_stored_env<FST_N>(fixed_topo(mv), world_accel(mv), cq, cqd, tape, ctb, o, B, e);
  if (partial) {
    __syncthreads();
    jit_write_partial(slots, P, partial);
  }
}
#endif

#ifdef FST_JIT_RNEA_DERIVS
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ qdd, float* __restrict__ dq,
                                                                 float* __restrict__ dqd) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  const Col cqd = stage_rows(tile + mv.nq * T, qd, mv.nv, B, e);
  const Col cqdd = stage_rows(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e);
  cp_async_wait_all();
  rnea_derivs_env<FST_N>(fixed_topo(mv), world_accel(mv), cq, cqd, cqdd, mv.nv, dq, dqd, B, e);
}
#endif

#ifdef FST_JIT_ABA_DERIVS
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ tau, float* __restrict__ qdd,
                                                                 float* __restrict__ dq, float* __restrict__ dqd,
                                                                 float* __restrict__ Minv) {
  FST_JIT_PROLOGUE;
  if (!act) return;
  const Col cq = stage_rows(tile, q, mv.nq, B, e);
  const Col cqd = stage_rows(tile + mv.nq * T, qd, mv.nv, B, e);
  const Col ctau = stage_rows(tile + (mv.nq + mv.nv) * T, tau, mv.nv, B, e);
  float* col = tile + (mv.nq + 2 * mv.nv) * T + threadIdx.x;
  cp_async_wait_all();
  aba_derivs_env<FST_N>(fixed_topo(mv), world_accel(mv), cq, cqd, ctau, mv.nv, col, T, dq, dqd, Minv, B, e);
  if (qdd)
    for (int k = 0; k < mv.nv; ++k) qdd[(int64_t)k * B + e] = col[k * T];
}
#endif

#ifdef FST_JIT_ABA_VJP
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ qdd,
                                                                 const float* __restrict__ qddbar, float* qbar,
                                                                 float* qdbar, float* taubar, float* partial) {
  FST_JIT_PROLOGUE;
  const int rows = mv.nq + 4 * mv.nv;
  const Col cq = jit_stage_or_zero(tile, q, mv.nq, B, e, act);
  const Col cqd = jit_stage_or_zero(tile + mv.nq * T, qd, mv.nv, B, e, act);
  const Col cqdd = jit_stage_or_zero(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e, act);
  const Col cqb = jit_stage_or_zero(tile + (mv.nq + 2 * mv.nv) * T, qddbar, mv.nv, B, e, act);
  float* lam = tile + (mv.nq + 3 * mv.nv) * T + threadIdx.x;
  const int P = FST_N * 10;
  float* slots = partial ? tile + rows * T : nullptr;
  if (slots)
    for (int k = threadIdx.x; k < (T / 32) * P; k += T) slots[k] = 0.f;
  cp_async_wait_all();
  __syncthreads();
  const FixedTopo tp = fixed_topo(mv);
  aba_env<FST_N>(tp, sv_zero(), cq, cqd, cqb, nullptr, B, e, true, lam, T);
  const Col clam{lam, T};
  if (taubar && act)
    for (int k = 0; k < mv.nv; ++k) taubar[(int64_t)k * B + e] = clam[k];
  VjpOut o{qbar, qdbar, nullptr, slots ? slots + (threadIdx.x / 32) * P : nullptr, -1.f, act};
  rnea_vjp_env<FST_N>(tp, world_accel(mv), cq, cqd, cqdd, clam, o, B, e);
  if (partial) {
    __syncthreads();
    jit_write_partial(slots, P, partial);
  }
}
#endif

#ifdef FST_JIT_LOSS_GRAD
extern "C" __global__ void __launch_bounds__(256) FST_JIT_NAME(ModelView mv, int64_t B, const float* __restrict__ q,
                                                                 const float* __restrict__ qd,
                                                                 const float* __restrict__ qdd,
                                                                 const float* __restrict__ tau_meas, float* qbar,
                                                                 float* qdbar, float* partial) {
  FST_JIT_PROLOGUE;
  const int rows = mv.nq + 3 * mv.nv;
  const Col cq = jit_stage_or_zero(tile, q, mv.nq, B, e, act);
  const Col cqd = jit_stage_or_zero(tile + mv.nq * T, qd, mv.nv, B, e, act);
  const Col cqdd = jit_stage_or_zero(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e, act);
  jit_stage_or_zero(tile + (mv.nq + 2 * mv.nv) * T, tau_meas, mv.nv, B, e, act);
  const int P = FST_N * 10 + 1;
  float* slots = tile + rows * T;
  for (int k = threadIdx.x; k < (T / 32) * P; k += T) slots[k] = 0.f;
  cp_async_wait_all();
  __syncthreads();
  const FixedTopo tp = fixed_topo(mv);
  const SV a0 = world_accel(mv);
  Xf X[FST_N];
  SV v[FST_N], a[FST_N], F[FST_N];
  rnea_forward<FST_N>(tp, a0, cq, cqd, cqdd, X, v, a, F);
  rnea_backward<FST_N>(tp, X, F, nullptr, B, e);
  float* tb = tile + (mv.nq + 2 * mv.nv) * T + threadIdx.x;
  float loss = 0.f;
#pragma unroll
  for (int i = 0; i < FST_N; ++i) {
    const BodyI bi = tp.I(i);
    const int nvi = nv_of(bi.type);
    if (nvi == 0) continue;
    float tau6[6];
    if (nvi == 1) {
      tau6[0] = dot(S_of(tp.C(i)), F[i]);
    } else {
      tau6[0] = F[i].v.x; tau6[1] = F[i].v.y; tau6[2] = F[i].v.z;
      tau6[3] = F[i].w.x; tau6[4] = F[i].w.y; tau6[5] = F[i].w.z;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      if (r >= nvi) break;
      const float res = tau6[r] - tb[(bi.vi + r) * T];
      loss = fmaf(res, res, loss);
      tb[(bi.vi + r) * T] = 2.f * res;
    }
  }
  float* wslot = slots + (threadIdx.x / 32) * P;
  float lg = act ? loss : 0.f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, off);
  if ((threadIdx.x & 31) == 0) wslot[P - 1] += lg;
  VjpOut o{qbar, qdbar, nullptr, wslot, 1.f, act};
  rnea_vjp_reverse<FST_N>(tp, a0, cq, cqd, X, v, a, F, Col{tb, T}, o, B, e);
  __syncthreads();
  jit_write_partial(slots, P, partial);
}
#endif

// ---- path-parallel kernels (FST_VARIANT_PATH), one per operator module ------
#if FST_PATH_G > 0
#define FST_PATH_PROLOGUE                                                  \
  extern __shared__ float4 smem[];                                        \
  float* tile = reinterpret_cast<float*>(smem);                           \
  constexpr int G = FST_PATH_G;                                           \
  constexpr int D = FST_DEPTH;                                            \
  PathLane<G> L;                                                          \
  const int EPB = (int)(blockDim.x >> 5) * PathLane<G>::E;                \
  const int eb = (int)(threadIdx.x >> 5) * PathLane<G>::E + L.es;         \
  const int64_t e0 = (int64_t)blockIdx.x * EPB;                           \
  const int64_t e = e0 + eb;                                              \
  const bool act = e < B;                                                 \
  const FixedTopo tp = fixed_topo(mv);                                    \
  const LanePath<D> lp = lane_path<G, D>(tp, L.g)

#define FST_PATH_READY \
  cp_async_wait_all(); \
  __syncthreads()

#define FST_PATH_COL(r) (Col{tile + (r)*EPB + eb, EPB})

#ifdef FST_JIT_FK
extern "C" __global__ void __launch_bounds__(256) FST_JIT_PATH_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q,
                                                                      float* __restrict__ poses) {
  FST_PATH_PROLOGUE;
  path_stage(tile, q, mv.nq, B, e0, EPB);
  FST_PATH_READY;
  Xf P[D];
  fk_path<D>(tp, lp, FST_PATH_COL(0), P, poses, B, e, act);
}
#endif

#ifdef FST_JIT_JACOBIAN
extern "C" __global__ void __launch_bounds__(256) FST_JIT_PATH_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q, LinkList links,
                                                                      float* __restrict__ J) {
  FST_PATH_PROLOGUE;
  path_stage(tile, q, mv.nq, B, e0, EPB);
  FST_PATH_READY;
  Xf P[D];
  fk_path<D>(tp, lp, FST_PATH_COL(0), P, nullptr, B, e, act);
  jac_path<D>(tp, lp, P, mv.nv, links, J, B, e, act);
}
#endif

#ifdef FST_JIT_RNEA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_PATH_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q,
                                                                      const float* __restrict__ qd,
                                                                      const float* __restrict__ qdd,
                                                                      float* __restrict__ tau) {
  FST_PATH_PROLOGUE;
  path_stage(tile, q, mv.nq, B, e0, EPB);
  path_stage(tile + mv.nq * EPB, qd, mv.nv, B, e0, EPB);
  path_stage(tile + (mv.nq + mv.nv) * EPB, qdd, mv.nv, B, e0, EPB);
  FST_PATH_READY;
  rnea_path<D>(tp, L, lp, world_accel(mv), FST_PATH_COL(0), FST_PATH_COL(mv.nq), FST_PATH_COL(mv.nq + mv.nv),
                  tau, B, e, act);
}
#endif

#ifdef FST_JIT_CRBA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_PATH_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q,
                                                                      float* __restrict__ M) {
  FST_PATH_PROLOGUE;
  path_stage(tile, q, mv.nq, B, e0, EPB);
  FST_PATH_READY;
  crba_path<D>(tp, L, lp, FST_PATH_COL(0), mv.nv, M, B, e, act);
}
#endif

#ifdef FST_JIT_ABA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_PATH_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q,
                                                                      const float* __restrict__ qd,
                                                                      const float* __restrict__ tau,
                                                                      float* __restrict__ qdd) {
  FST_PATH_PROLOGUE;
  path_stage(tile, q, mv.nq, B, e0, EPB);
  path_stage(tile + mv.nq * EPB, qd, mv.nv, B, e0, EPB);
  path_stage(tile + (mv.nq + mv.nv) * EPB, tau, mv.nv, B, e0, EPB);
  FST_PATH_READY;
  aba_path<D>(tp, L, lp, world_accel(mv), FST_PATH_COL(0), FST_PATH_COL(mv.nq), FST_PATH_COL(mv.nq + mv.nv), qdd,
                 B, e, act);
}
#endif

#ifdef FST_JIT_EVAL
// Roles on blockIdx.y, each path-parallel.
extern "C" __global__ void __launch_bounds__(256) FST_JIT_PATH_NAME(ModelView mv, int64_t B, EvalArgs a) {
  FST_PATH_PROLOGUE;
  const int role = a.roles[blockIdx.y];
  path_stage(tile, a.q, mv.nq, B, e0, EPB);
  if (role == ROLE_RNEA) {
    path_stage(tile + mv.nq * EPB, a.qd, mv.nv, B, e0, EPB);
    path_stage(tile + (mv.nq + mv.nv) * EPB, a.qdd, mv.nv, B, e0, EPB);
  } else if (role == ROLE_ABA) {
    path_stage(tile + mv.nq * EPB, a.qd, mv.nv, B, e0, EPB);
    path_stage(tile + (mv.nq + mv.nv) * EPB, a.tau, mv.nv, B, e0, EPB);
  }
  FST_PATH_READY;
  const Col cq = FST_PATH_COL(0), c1 = FST_PATH_COL(mv.nq), c2 = FST_PATH_COL(mv.nq + mv.nv);
  switch (role) {
    case ROLE_ABA:
      aba_path<D>(tp, L, lp, world_accel(mv), cq, c1, c2, a.qdd_out, B, e, act);
      break;
    case ROLE_CRBA:
      crba_path<D>(tp, L, lp, cq, mv.nv, a.M, B, e, act);
      break;
    case ROLE_RNEA:
      rnea_path<D>(tp, L, lp, world_accel(mv), cq, c1, c2, a.tau_out, B, e, act);
      break;
    default: {
      Xf P[D];
      fk_path<D>(tp, lp, cq, P, a.poses, B, e, act);
      if (a.J) jac_path<D>(tp, lp, P, mv.nv, a.links, a.J, B, e, act);
      break;
    }
  }
}
#endif
#endif  // FST_PATH_G > 0

// ---- path-per-warp kernels (FST_VARIANT_PATH_WARP) ----------------------------
// A block of FST_PATH_NP warps serves 32 environments (one per lane); warp g
// sweeps path g with code compiled for that path (every body constant folds),
// and the paths meet through the shared-memory merge of SmemMerge.
#if FST_PATH_G > 0
template <int g>
struct WarpPath {
  __device__ __forceinline__ int body(int t) const { return kPath[g * FST_DEPTH + t]; }
  __device__ __forceinline__ bool leads(int t) const { return (kLead[g] >> t) & 1u; }
  __device__ __forceinline__ int lo(int t) const { return kSeg[g * FST_DEPTH + t] & 0xff; }
  __device__ __forceinline__ int hi(int t) const { return kSeg[g * FST_DEPTH + t] >> 8; }
  __device__ __forceinline__ int index() const { return g; }
};

template <int K>
struct IC {
  static constexpr int value = K;
};

// Calls f(IC<w>) with this warp's index as a compile-time constant.
template <int K, int NP, class F>
__device__ __forceinline__ void for_warp(int w, F& f) {
  if constexpr (K < NP) {
    if (w == K)
      f(IC<K>{});
    else
      for_warp<K + 1, NP>(w, f);
  }
}

constexpr int kWarpXch = 27;  // floats per lane and warp in one merge (Sym6 + force)

#define FST_WARP_PROLOGUE(rows)                                  \
  extern __shared__ float4 smem[];                              \
  float* tile = reinterpret_cast<float*>(smem);                 \
  constexpr int D = FST_DEPTH;                                  \
  constexpr int NP = FST_PATH_NP;                               \
  const int lane = (int)(threadIdx.x & 31);                     \
  const int warp = (int)(threadIdx.x >> 5);                     \
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;            \
  const bool act = e < B;                                       \
  const FixedTopo tp = fixed_topo(mv);                          \
  SmemMerge<NP, kWarpXch> mg{tile + (rows) * 32, warp, lane, 0}

#define FST_WARP_READY \
  cp_async_wait_all(); \
  __syncthreads()

#define FST_WARP_COL(r) (Col{tile + (r)*32 + lane, 32})

#ifdef FST_JIT_FK
extern "C" __global__ void __launch_bounds__(256) FST_JIT_WARP_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q,
                                                                      float* __restrict__ poses) {
  FST_WARP_PROLOGUE(mv.nq);
  stage_block_rows(tile, q, mv.nq, B, e);
  FST_WARP_READY;
  auto f = [&](auto kc) {
    Xf P[D];
    fk_path<D>(tp, WarpPath<decltype(kc)::value>{}, FST_WARP_COL(0), P, poses, B, e, act);
  };
  for_warp<0, NP>(warp, f);
}
#endif

#ifdef FST_JIT_JACOBIAN
extern "C" __global__ void __launch_bounds__(256) FST_JIT_WARP_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q, LinkList links,
                                                                      float* __restrict__ J) {
  FST_WARP_PROLOGUE(mv.nq);
  stage_block_rows(tile, q, mv.nq, B, e);
  FST_WARP_READY;
  auto f = [&](auto kc) {
    const WarpPath<decltype(kc)::value> lp{};
    Xf P[D];
    fk_path<D>(tp, lp, FST_WARP_COL(0), P, nullptr, B, e, act);
    jac_path<D>(tp, lp, P, mv.nv, links, J, B, e, act);
  };
  for_warp<0, NP>(warp, f);
}
#endif

#ifdef FST_JIT_RNEA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_WARP_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q,
                                                                      const float* __restrict__ qd,
                                                                      const float* __restrict__ qdd,
                                                                      float* __restrict__ tau) {
  FST_WARP_PROLOGUE(mv.nq + 2 * mv.nv);
  stage_block_rows(tile, q, mv.nq, B, e);
  stage_block_rows(tile + mv.nq * 32, qd, mv.nv, B, e);
  stage_block_rows(tile + (mv.nq + mv.nv) * 32, qdd, mv.nv, B, e);
  FST_WARP_READY;
  auto f = [&](auto kc) {
    rnea_path<D>(tp, mg, WarpPath<decltype(kc)::value>{}, world_accel(mv), FST_WARP_COL(0), FST_WARP_COL(mv.nq),
                 FST_WARP_COL(mv.nq + mv.nv), tau, B, e, act);
  };
  for_warp<0, NP>(warp, f);
}
#endif

#ifdef FST_JIT_CRBA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_WARP_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q,
                                                                      float* __restrict__ M) {
  FST_WARP_PROLOGUE(mv.nq);
  stage_block_rows(tile, q, mv.nq, B, e);
  FST_WARP_READY;
  auto f = [&](auto kc) {
    crba_path<D>(tp, mg, WarpPath<decltype(kc)::value>{}, FST_WARP_COL(0), mv.nv, M, B, e, act);
  };
  for_warp<0, NP>(warp, f);
}
#endif

#ifdef FST_JIT_ABA
extern "C" __global__ void __launch_bounds__(256) FST_JIT_WARP_NAME(ModelView mv, int64_t B,
                                                                      const float* __restrict__ q,
                                                                      const float* __restrict__ qd,
                                                                      const float* __restrict__ tau,
                                                                      float* __restrict__ qdd) {
  FST_WARP_PROLOGUE(mv.nq + 2 * mv.nv);
  stage_block_rows(tile, q, mv.nq, B, e);
  stage_block_rows(tile + mv.nq * 32, qd, mv.nv, B, e);
  stage_block_rows(tile + (mv.nq + mv.nv) * 32, tau, mv.nv, B, e);
  FST_WARP_READY;
  auto f = [&](auto kc) {
    aba_path<D>(tp, mg, WarpPath<decltype(kc)::value>{}, world_accel(mv), FST_WARP_COL(0), FST_WARP_COL(mv.nq),
                FST_WARP_COL(mv.nq + mv.nv), qdd, B, e, act);
  };
  for_warp<0, NP>(warp, f);
}
#endif

#ifdef FST_JIT_EVAL
extern "C" __global__ void __launch_bounds__(256) FST_JIT_WARP_NAME(ModelView mv, int64_t B, EvalArgs a) {
  FST_WARP_PROLOGUE(mv.nq + 2 * mv.nv);
  const int role = a.roles[blockIdx.y];
  stage_block_rows(tile, a.q, mv.nq, B, e);
  if (role == ROLE_RNEA) {
    stage_block_rows(tile + mv.nq * 32, a.qd, mv.nv, B, e);
    stage_block_rows(tile + (mv.nq + mv.nv) * 32, a.qdd, mv.nv, B, e);
  } else if (role == ROLE_ABA) {
    stage_block_rows(tile + mv.nq * 32, a.qd, mv.nv, B, e);
    stage_block_rows(tile + (mv.nq + mv.nv) * 32, a.tau, mv.nv, B, e);
  }
  FST_WARP_READY;
  const Col cq = FST_WARP_COL(0), c1 = FST_WARP_COL(mv.nq), c2 = FST_WARP_COL(mv.nq + mv.nv);
  auto f = [&](auto kc) {
    const WarpPath<decltype(kc)::value> lp{};
    switch (role) {
      case ROLE_ABA:
        aba_path<D>(tp, mg, lp, world_accel(mv), cq, c1, c2, a.qdd_out, B, e, act);
        break;
      case ROLE_CRBA:
        crba_path<D>(tp, mg, lp, cq, mv.nv, a.M, B, e, act);
        break;
      case ROLE_RNEA:
        rnea_path<D>(tp, mg, lp, world_accel(mv), cq, c1, c2, a.tau_out, B, e, act);
        break;
      default: {
        Xf P[D];
        fk_path<D>(tp, lp, cq, P, a.poses, B, e, act);
        if (a.J) jac_path<D>(tp, lp, P, mv.nv, a.links, a.J, B, e, act);
        break;
      }
    }
  };
  for_warp<0, NP>(warp, f);
}
#endif
#endif  // FST_PATH_G > 0
