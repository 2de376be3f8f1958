// Dense dynamics-derivative kernels (bodies in derivs.cuh): one environment
// per thread, inputs staged in shared memory, outputs [nv][nv][B].
#include "derivs.cuh"
#include "launch.h"

namespace fst {
namespace {

template <int NB>
__global__ void __launch_bounds__(256) rnea_derivs_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                          const float* __restrict__ qd,
                                                          const float* __restrict__ qdd, float* __restrict__ dq,
                                                          float* __restrict__ dqd) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  Col cq{}, cqd{}, cqdd{};
  if (act) {
    cq = stage_rows(tile, q, mv.nq, B, e);
    cqd = stage_rows(tile + mv.nq * T, qd, mv.nv, B, e);
    cqdd = stage_rows(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e);
  }
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  rnea_derivs_env<NB>(sm, world_accel(mv), cq, cqd, cqdd, mv.nv, dq, dqd, B, e);
}

template <int NB>
__global__ void __launch_bounds__(256) aba_derivs_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                         const float* __restrict__ qd, const float* __restrict__ tau,
                                                         float* __restrict__ qdd, float* __restrict__ dq,
                                                         float* __restrict__ dqd, float* __restrict__ Minv) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  Col cq{}, cqd{}, ctau{};
  if (act) {
    cq = stage_rows(tile, q, mv.nq, B, e);
    cqd = stage_rows(tile + mv.nq * T, qd, mv.nv, B, e);
    ctau = stage_rows(tile + (mv.nq + mv.nv) * T, tau, mv.nv, B, e);
  }
  float* col = tile + (mv.nq + 2 * mv.nv) * T + threadIdx.x;
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  aba_derivs_env<NB>(sm, world_accel(mv), cq, cqd, ctau, mv.nv, col, T, dq, dqd, Minv, B, e);
  if (qdd)
    for (int k = 0; k < mv.nv; ++k) qdd[(int64_t)k * B + e] = col[k * T];
}

}  // namespace

cudaError_t launch_rnea_derivs(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                               float* dq, float* dqd, const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq + 2 * mv.nv, L.block);
  FST_NB_DISPATCH(mv.n, prepare(rnea_derivs_kernel<NB>, sh);
                  rnea_derivs_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, qd, qdd, dq, dqd));
  return cudaGetLastError();
}

cudaError_t launch_aba_derivs(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                              float* qdd, float* dq, float* dqd, float* Minv, const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq + 3 * mv.nv, L.block);
  FST_NB_DISPATCH(mv.n, prepare(aba_derivs_kernel<NB>, sh);
                  aba_derivs_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, qd, tau, qdd, dq,
                                                                                         dqd, Minv));
  return cudaGetLastError();
}

}  // namespace fst
