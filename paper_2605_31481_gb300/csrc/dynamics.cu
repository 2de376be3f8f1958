// RNEA, CRBA and ABA kernels, one environment per thread (bodies in ops.cuh).
//
// Each thread sweeps its environment's tree in body order (parents first)
// and back; per-body state lives in per-thread arrays (local memory, cached
// in L1), model constants in shared memory where every lane of a warp reads
// the same word (a broadcast), and the environment's inputs are staged into
// shared memory with asynchronous copies before the sweep starts.
#include "ops.cuh"
#include "launch.h"

namespace fst {
namespace {

template <int NB>
__global__ void __launch_bounds__(256) rnea_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                   const float* __restrict__ qd, const float* __restrict__ qdd,
                                                   float* __restrict__ tau) {
  extern __shared__ float4 smem[];
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = e < B;
  Col cq{}, cqd{}, cqdd{};
  if (act) {
    cq = stage_rows(tile, q, mv.nq, B, e);
    cqd = stage_rows(tile + mv.nq * blockDim.x, qd, mv.nv, B, e);
    cqdd = stage_rows(tile + (mv.nq + mv.nv) * blockDim.x, qdd, mv.nv, B, e);
  }
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  rnea_env<NB>(sm, world_accel(mv), cq, cqd, cqdd, tau, B, e);
}

template <int NB>
__global__ void __launch_bounds__(256) crba_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                   float* __restrict__ M) {
  extern __shared__ float4 smem[];
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = e < B;
  Col cq{};
  if (act) cq = stage_rows(tile, q, mv.nq, B, e);
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  crba_env<NB>(sm, cq, mv.nv, M, B, e);
}

template <int NB>
__global__ void __launch_bounds__(256) aba_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                  const float* __restrict__ qd, const float* __restrict__ tau,
                                                  float* __restrict__ qdd) {
  extern __shared__ float4 smem[];
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = e < B;
  Col cq{}, cqd{}, ctau{};
  if (act) {
    cq = stage_rows(tile, q, mv.nq, B, e);
    cqd = stage_rows(tile + mv.nq * blockDim.x, qd, mv.nv, B, e);
    ctau = stage_rows(tile + (mv.nq + mv.nv) * blockDim.x, tau, mv.nv, B, e);
  }
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  aba_env<NB>(sm, world_accel(mv), cq, cqd, ctau, qdd, B, e);
}

}  // namespace

cudaError_t launch_rnea(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                        float* tau, const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq + 2 * mv.nv, L.block);
  FST_NB_DISPATCH(mv.n, prepare(rnea_kernel<NB>, sh); rnea_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, qd, qdd, tau));
  return cudaGetLastError();
}

cudaError_t launch_crba(const ModelView& mv, int64_t B, const float* q, float* M, const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq, L.block);
  FST_NB_DISPATCH(mv.n, prepare(crba_kernel<NB>, sh); crba_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, M));
  return cudaGetLastError();
}

cudaError_t launch_aba(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                       float* qdd, const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq + 2 * mv.nv, L.block);
  FST_NB_DISPATCH(mv.n, prepare(aba_kernel<NB>, sh); aba_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, qd, tau, qdd));
  return cudaGetLastError();
}

}  // namespace fst
