// Forward kinematics and geometric Jacobians, one environment per thread.
//
// FK is tier 3 of the paper's kinematic state (Sec. 3.1): world poses by
// propagating each joint's Rodrigues transform (Eq. 4-5) from the root. The
// Jacobian builds each column directly from the world pose of the joint's
// body (Sec. 3.4, Eq. 6): w = R_k S_w, v = R_k S_v + p_k x w, which for a
// revolute joint is [o_k x z_k; z_k] with o_k on the axis.
#include "fst_device.cuh"
#include "launch.h"

namespace fst {
namespace {

template <int NB>
__global__ void __launch_bounds__(128) fk_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                 float* __restrict__ poses) {
  extern __shared__ float4 smem[];
  const SmemModel sm = stage_model(mv, smem);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  float Rw[NB][9];
  float pw[NB][3];
  for (int i = 0; i < sm.n; ++i) {
    const BodyC& c = sm.c[i];
    const BodyI bi = sm.i[i];
    const Xf X = joint_X(c, bi, q, B, e);
    float R[9], p[3];
    if (bi.parent < 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) R[k] = X.R[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) p[k] = X.t[k];
    } else {
      const float* Rp = Rw[bi.parent];
      const float* pp = pw[bi.parent];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
          R[3 * r + cc] = fmaf(Rp[3 * r], X.R[cc], fmaf(Rp[3 * r + 1], X.R[3 + cc], Rp[3 * r + 2] * X.R[6 + cc]));
        p[r] = fmaf(Rp[3 * r], X.t[0], fmaf(Rp[3 * r + 1], X.t[1], fmaf(Rp[3 * r + 2], X.t[2], pp[r])));
      }
    }
    float* out = poses + (int64_t)i * 12 * B + e;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      Rw[i][k] = R[k];
      out[(int64_t)k * B] = R[k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      pw[i][k] = p[k];
      out[(int64_t)(9 + k) * B] = p[k];
    }
  }
}

template <int NB>
__global__ void __launch_bounds__(128) jac_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                  LinkList links, float* __restrict__ J) {
  extern __shared__ float4 smem[];
  const SmemModel sm = stage_model(mv, smem);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  float Rw[NB][9];
  float pw[NB][3];
  for (int i = 0; i < sm.n; ++i) {
    const BodyC& c = sm.c[i];
    const BodyI bi = sm.i[i];
    const Xf X = joint_X(c, bi, q, B, e);
    if (bi.parent < 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Rw[i][k] = X.R[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) pw[i][k] = X.t[k];
    } else {
      const float* Rp = Rw[bi.parent];
      const float* pp = pw[bi.parent];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
          Rw[i][3 * r + cc] =
              fmaf(Rp[3 * r], X.R[cc], fmaf(Rp[3 * r + 1], X.R[3 + cc], Rp[3 * r + 2] * X.R[6 + cc]));
        pw[i][r] = fmaf(Rp[3 * r], X.t[0], fmaf(Rp[3 * r + 1], X.t[1], fmaf(Rp[3 * r + 2], X.t[2], pp[r])));
      }
    }
  }
  const int nv = mv.nv;
  for (int l = 0; l < links.n; ++l) {
    const unsigned long long mask = sm.c[links.idx[l]].anc;
    float* Jl = J + (int64_t)l * 6 * nv * B + e;
    for (int k = 0; k < sm.n; ++k) {
      const BodyI bk = sm.i[k];
      const int nvk = nv_of(bk.type);
      if (nvk == 0) continue;
      const bool on_path = (mask >> k) & 1ull;
      const f3 p = f3{pw[k][0], pw[k][1], pw[k][2]};
      if (nvk == 1) {
        float col[6] = {0, 0, 0, 0, 0, 0};
        if (on_path) {
          const SV s = S_of(sm.c[k]);
          const f3 w = Rmul(Rw[k], s.w);
          const f3 v = Rmul(Rw[k], s.v) + cross(p, w);
          col[0] = v.x; col[1] = v.y; col[2] = v.z;
          col[3] = w.x; col[4] = w.y; col[5] = w.z;
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) Jl[((int64_t)r * nv + bk.vi) * B] = col[r];
      } else {  // free base: velocity [v; w] in body coordinates
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          float col[6] = {0, 0, 0, 0, 0, 0};
          if (on_path) {
            const int a = j % 3;
            const f3 Re = f3{Rw[k][a], Rw[k][3 + a], Rw[k][6 + a]};  // R e_a
            if (j < 3) {
              col[0] = Re.x; col[1] = Re.y; col[2] = Re.z;
            } else {
              const f3 v = cross(p, Re);
              col[0] = v.x; col[1] = v.y; col[2] = v.z;
              col[3] = Re.x; col[4] = Re.y; col[5] = Re.z;
            }
          }
#pragma unroll
          for (int r = 0; r < 6; ++r) Jl[((int64_t)r * nv + bk.vi + j) * B] = col[r];
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_fk(const ModelView& mv, int64_t B, const float* q, float* poses, const Launch& L) {
  const size_t sh = smem_bytes(mv.n);
  FST_NB_DISPATCH(mv.n, fk_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, poses));
  return cudaGetLastError();
}

cudaError_t launch_jacobian(const ModelView& mv, int64_t B, const float* q, const LinkList& links, float* J,
                            const Launch& L) {
  const size_t sh = smem_bytes(mv.n);
  FST_NB_DISPATCH(mv.n, jac_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, links, J));
  return cudaGetLastError();
}

}  // namespace fst
