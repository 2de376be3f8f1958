// Forward kinematics and geometric Jacobian kernels, one environment per
// thread (bodies in ops.cuh).
#include "ops.cuh"
#include "launch.h"

namespace fst {
namespace {

template <int NB>
__global__ void __launch_bounds__(256) fk_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                 float* __restrict__ poses) {
  extern __shared__ float4 smem[];
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = e < B;
  Col cq{};
  if (act) cq = stage_rows(tile, q, mv.nq, B, e);
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  fk_env<NB>(sm, cq, poses, B, e);
}

template <int NB>
__global__ void __launch_bounds__(256) jac_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                  LinkList links, float* __restrict__ J) {
  extern __shared__ float4 smem[];
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = e < B;
  Col cq{};
  if (act) cq = stage_rows(tile, q, mv.nq, B, e);
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  jac_env<NB>(sm, cq, mv.nv, links, nullptr, J, B, e);
}

}  // namespace

cudaError_t launch_fk(const ModelView& mv, int64_t B, const float* q, float* poses, const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq, L.block);
  FST_NB_DISPATCH(mv.n, prepare(fk_kernel<NB>, sh); fk_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, poses));
  return cudaGetLastError();
}

cudaError_t launch_jacobian(const ModelView& mv, int64_t B, const float* q, const LinkList& links, float* J,
                            const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq, L.block);
  FST_NB_DISPATCH(mv.n, prepare(jac_kernel<NB>, sh); jac_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, links, J));
  return cudaGetLastError();
}

}  // namespace fst
