// Fused evaluation: every requested operator in one launch.
//
// The paper shares kinematic quantities across operators through a tiered
// lazy cache and computes only the tiers a query needs (Sec. 3.1). Here the
// operators are independent given (q, qd, qdd, tau), so one launch runs them
// side by side: blockIdx.y picks the operator ("role") of a block, and only
// the operators whose outputs were requested get a role. At B = 4096 one
// operator alone fills only a fraction of the GPU's 152 SMs; the roles
// together fill it, and the launch takes as long as its slowest role rather
// than the sum of all of them.
#include "adjoint.cuh"
#include "launch.h"

namespace fst {
namespace {

// EXT: the extended form (a separate kernel, so that the plain one keeps its
// registers and code size): the RNEA role with the adjoint and/or the
// kinematics from its own sweep (a.rnea_flags), and M and J in the packed
// layouts (a.packed). Its input rows past q, qd and qdd hold tau_bar.
template <int NB, bool EXT>
__global__ void __launch_bounds__(256) eval_kernel(ModelView mv, int64_t B, EvalArgs a) {
  extern __shared__ float4 smem[];
  float* tile = smem_tile(smem, mv.n);
  const int role = a.roles[blockIdx.y];
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = e < B;
  const int T = blockDim.x;
  Col cq{}, c1{}, c2{};
  if (act) {
    cq = stage_rows(tile, a.q, mv.nq, B, e);
    if (role == ROLE_RNEA) {
      c1 = stage_rows(tile + mv.nq * T, a.qd, mv.nv, B, e);
      c2 = stage_rows(tile + (mv.nq + mv.nv) * T, a.qdd, mv.nv, B, e);
      if (EXT && (a.rnea_flags & EVAL_RNEA_VJP) && !(a.rnea_flags & EVAL_TBAR_IS_TAU))
        stage_rows(tile + (mv.nq + 2 * mv.nv) * T, a.tau_bar, mv.nv, B, e);
    } else if (role == ROLE_ABA) {
      c1 = stage_rows(tile + mv.nq * T, a.qd, mv.nv, B, e);
      c2 = stage_rows(tile + (mv.nq + mv.nv) * T, a.tau, mv.nv, B, e);
    }
  }
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  switch (role) {
    case ROLE_ABA:
      aba_env<NB>(sm, world_accel(mv), cq, c1, c2, a.qdd_out, B, e);
      break;
    case ROLE_CRBA:
      if (EXT && a.packed)
        crba_env<NB, true>(sm, cq, mv.nv, a.M, B, e);
      else
        crba_env<NB>(sm, cq, mv.nv, a.M, B, e);
      break;
    case ROLE_RNEA:
      if (EXT && a.rnea_flags)
        rnea_role_env<NB>(sm, world_accel(mv), cq, c1, c2, tile + (mv.nq + 2 * mv.nv) * T + threadIdx.x, T, mv.nv, a,
                          B, e);
      else
        rnea_env<NB>(sm, world_accel(mv), cq, c1, c2, a.tau_out, B, e);
      break;
    default:
      if (a.J)
        jac_env<NB>(sm, cq, mv.nv, a.links, a.poses, a.J, B, e, EXT && a.packed ? &a.pj : nullptr);
      else
        fk_env<NB>(sm, cq, a.poses, B, e);
      break;
  }
}

}  // namespace

cudaError_t launch_eval(const ModelView& mv, int64_t B, const EvalArgs& a, const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq + (a.rnea_flags & EVAL_RNEA_VJP ? 3 : 2) * mv.nv, L.block);
  const dim3 grid(grid_for(B, L.block), a.n_roles);
  if (a.rnea_flags || a.packed)
    FST_NB_DISPATCH(mv.n, prepare(eval_kernel<NB, true>, sh);
                    eval_kernel<NB, true><<<grid, L.block, sh, L.stream>>>(mv, B, a));
  else
    FST_NB_DISPATCH(mv.n, prepare(eval_kernel<NB, false>, sh);
                    eval_kernel<NB, false><<<grid, L.block, sh, L.stream>>>(mv, B, a));
  return cudaGetLastError();
}

}  // namespace fst
