// RNEA, CRBA and ABA, one environment per thread.
//
// Each thread sweeps its environment's tree in body order (parents first)
// and back; the per-body state lives in per-thread arrays (local memory,
// cached in L1), the model constants in shared memory where every lane of a
// warp reads the same word (a broadcast). Sibling bodies are independent, so
// the paper's level-parallel grouping (Sec. 3.3) is not needed to expose
// parallelism here: all B environments already run concurrently.
#include "fst_device.cuh"
#include "launch.h"

namespace fst {
namespace {

__device__ __forceinline__ SV world_accel(const ModelView& mv) {
  return SV{f3{0.f, 0.f, 0.f}, f3{mv.a0[0], mv.a0[1], mv.a0[2]}};
}

// Recursive Newton-Euler (paper Sec. 3.3, Eq. 7 for the velocity sweep):
//   v_i = X_i v_p + S_i qd_i
//   a_i = X_i a_p + S_i qdd_i + v_i x S_i qd_i     (a of the world = -g)
//   f_i = I_i a_i + v_i x* I_i v_i
// then leaf to root: tau_i = S_i^T f_i, f_p += X_i^T f_i.
template <int NB>
__global__ void __launch_bounds__(128) rnea_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                   const float* __restrict__ qd, const float* __restrict__ qdd,
                                                   float* __restrict__ tau) {
  extern __shared__ float4 smem[];
  const SmemModel sm = stage_model(mv, smem);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  Xf X[NB];
  SV v[NB], a[NB], f[NB];
  const SV a0 = world_accel(mv);
  for (int i = 0; i < sm.n; ++i) {
    const BodyC& c = sm.c[i];
    const BodyI bi = sm.i[i];
    X[i] = joint_X(c, bi, q, B, e);
    const SV vJ = S_times(c, bi, qd, B, e);
    const SV aJ = S_times(c, bi, qdd, B, e);
    SV vi, ai;
    if (bi.parent < 0) {
      vi = vJ;
      ai = X_motion(X[i], a0) + aJ;
    } else {
      vi = X_motion(X[i], v[bi.parent]) + vJ;
      ai = X_motion(X[i], a[bi.parent]) + aJ + crm(vi, vJ);
    }
    const In10 I = in_load(c.theta);
    v[i] = vi;
    a[i] = ai;
    f[i] = in_mul(I, ai) + crf(vi, in_mul(I, vi));
  }
  for (int i = sm.n - 1; i >= 0; --i) {
    const BodyI bi = sm.i[i];
    ST_store(sm.c[i], bi, f[i], tau, B, e);
    if (bi.parent >= 0) f[bi.parent] = f[bi.parent] + XT_force(X[i], f[i]);
  }
}

// Composite-rigid-body algorithm: composite inertias leaf to root
// (I^c_p += X_i^T I^c_i X_i, kept as 10 parameters because a sum of rigid
// bodies is a rigid body), then F = I^c_i S_i carried up the support path:
// M_ij = S_j^T F.
template <int NB>
__global__ void __launch_bounds__(128) crba_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                   float* __restrict__ M) {
  extern __shared__ float4 smem[];
  const SmemModel sm = stage_model(mv, smem);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  Xf X[NB];
  In10 Ic[NB];
  const int nv = mv.nv;
  for (int i = 0; i < sm.n; ++i) {
    X[i] = joint_X(sm.c[i], sm.i[i], q, B, e);
    Ic[i] = in_load(sm.c[i].theta);
  }
  for (int i = sm.n - 1; i > 0; --i) {
    const int p = sm.i[i].parent;
    if (p >= 0) in_add(Ic[p], in_to_parent(X[i], Ic[i]));
  }
  float* Me = M + e;
  for (int i = 0; i < sm.n; ++i) {
    const BodyI bi = sm.i[i];
    if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
      SV F = in_mul(Ic[i], S_of(sm.c[i]));
      Me[((int64_t)bi.vi * nv + bi.vi) * B] = dot(S_of(sm.c[i]), F);
      int j = i;
      while (sm.i[j].parent >= 0) {
        F = XT_force(X[j], F);
        j = sm.i[j].parent;
        const BodyI bj = sm.i[j];
        if (bj.type == FST_JOINT_REVOLUTE || bj.type == FST_JOINT_PRISMATIC) {
          const float mij = dot(S_of(sm.c[j]), F);
          Me[((int64_t)bi.vi * nv + bj.vi) * B] = mij;
          Me[((int64_t)bj.vi * nv + bi.vi) * B] = mij;
        } else if (bj.type == FST_JOINT_FREE) {
          const float col[6] = {F.v.x, F.v.y, F.v.z, F.w.x, F.w.y, F.w.z};
#pragma unroll
          for (int r = 0; r < 6; ++r) {
            Me[((int64_t)(bj.vi + r) * nv + bi.vi) * B] = col[r];
            Me[((int64_t)bi.vi * nv + bj.vi + r) * B] = col[r];
          }
        }
      }
    } else if (bi.type == FST_JOINT_FREE) {
      // base block: the composite inertia with rows/cols ordered [v; w]
      const In10& I = Ic[i];
      const float blk[6][6] = {
          {I.m, 0.f, 0.f, 0.f, I.h.z, -I.h.y},
          {0.f, I.m, 0.f, -I.h.z, 0.f, I.h.x},
          {0.f, 0.f, I.m, I.h.y, -I.h.x, 0.f},
          {0.f, -I.h.z, I.h.y, I.I[0], I.I[1], I.I[3]},
          {I.h.z, 0.f, -I.h.x, I.I[1], I.I[2], I.I[4]},
          {-I.h.y, I.h.x, 0.f, I.I[3], I.I[4], I.I[5]},
      };
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) Me[((int64_t)(bi.vi + r) * nv + bi.vi + cc) * B] = blk[r][cc];
    }
  }
  // structural zeros: DOF pairs whose bodies are not on one support path
  for (int i = 1; i < sm.n; ++i) {
    const BodyI bi = sm.i[i];
    const int ni = nv_of(bi.type);
    if (ni == 0) continue;
    const unsigned long long anc_i = sm.c[i].anc;
    for (int j = 0; j < i; ++j) {
      const BodyI bj = sm.i[j];
      const int nj = nv_of(bj.type);
      if (nj == 0 || ((anc_i >> j) & 1ull)) continue;
      for (int r = 0; r < ni; ++r)
        for (int cc = 0; cc < nj; ++cc) {
          Me[((int64_t)(bi.vi + r) * nv + bj.vi + cc) * B] = 0.f;
          Me[((int64_t)(bj.vi + cc) * nv + bi.vi + r) * B] = 0.f;
        }
    }
  }
}

// Cholesky solve of a symmetric positive-definite 6x6 spatial system.
__device__ __forceinline__ SV sym6_solve(const Sym6& s, SV rhs) {
  float A[6][6];
  const float Af[9] = {s.A[0], s.A[1], s.A[3], s.A[1], s.A[2], s.A[4], s.A[3], s.A[4], s.A[5]};
  const float Cf[9] = {s.C[0], s.C[1], s.C[3], s.C[1], s.C[2], s.C[4], s.C[3], s.C[4], s.C[5]};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A[r][c] = Af[3 * r + c];
      A[r][3 + c] = s.Bk[3 * r + c];
      A[3 + r][c] = s.Bk[3 * c + r];
      A[3 + r][3 + c] = Cf[3 * r + c];
    }
  float L[6][6];
  float inv[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float d = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d = fmaf(-L[j][k], L[j][k], d);
    const float ljj = sqrtf(d);
    inv[j] = 1.0f / ljj;
    L[j][j] = ljj;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      float x = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) x = fmaf(-L[i][k], L[j][k], x);
      L[i][j] = x * inv[j];
    }
  }
  float y[6] = {rhs.w.x, rhs.w.y, rhs.w.z, rhs.v.x, rhs.v.y, rhs.v.z};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int k = 0; k < i; ++k) y[i] = fmaf(-L[i][k], y[k], y[i]);
    y[i] *= inv[i];
  }
#pragma unroll
  for (int i = 5; i >= 0; --i) {
#pragma unroll
    for (int k = i + 1; k < 6; ++k) y[i] = fmaf(-L[k][i], y[k], y[i]);
    y[i] *= inv[i];
  }
  return SV{f3{y[0], y[1], y[2]}, f3{y[3], y[4], y[5]}};
}

// Articulated-body algorithm, three passes (paper Sec. 4.1):
//  1. root to leaf: v_i, bias acceleration c_i = v_i x S_i qd_i,
//     I^A_i = I_i, p^A_i = v_i x* I_i v_i
//  2. leaf to root: U = I^A S, D = S^T U, u = tau - S^T p^A,
//     I^a = I^A - U U^T / D, p^a = p^A + I^a c + U u / D,
//     I^A_p += X^T I^a X, p^A_p += X^T p^a
//  3. root to leaf: a' = X a_p + c, qdd = (u - U^T a') / D, a = a' + S qdd
// A free base solves its 6x6 articulated inertia directly.
template <int NB>
__global__ void __launch_bounds__(128) aba_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                  const float* __restrict__ qd, const float* __restrict__ tau,
                                                  float* __restrict__ qdd) {
  extern __shared__ float4 smem[];
  const SmemModel sm = stage_model(mv, smem);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  Xf X[NB];
  SV va[NB];  // velocity in pass 1, acceleration in pass 3
  SV cb[NB], pA[NB], U[NB];
  Sym6 IA[NB];
  float invD[NB], u[NB];
  for (int i = 0; i < sm.n; ++i) {
    const BodyC& c = sm.c[i];
    const BodyI bi = sm.i[i];
    X[i] = joint_X(c, bi, q, B, e);
    const SV vJ = S_times(c, bi, qd, B, e);
    SV vi;
    if (bi.parent < 0) {
      vi = vJ;
      cb[i] = sv_zero();
    } else {
      vi = X_motion(X[i], va[bi.parent]) + vJ;
      cb[i] = crm(vi, vJ);
    }
    va[i] = vi;
    const In10 I = in_load(c.theta);
    IA[i] = sym6_from_in(I);
    pA[i] = crf(vi, in_mul(I, vi));
  }
  for (int i = sm.n - 1; i >= 0; --i) {
    const BodyI bi = sm.i[i];
    if (bi.type == FST_JOINT_FREE) continue;  // the root: solved in pass 3
    Sym6 Ia = IA[i];
    SV pa = pA[i];
    if (bi.type != FST_JOINT_FIXED) {
      const SV S = S_of(sm.c[i]);
      const SV Ui = sym6_mul(IA[i], S);
      const float iD = 1.0f / dot(S, Ui);
      const float ui = __ldg(tau + (int64_t)bi.vi * B + e) - dot(S, pA[i]);
      U[i] = Ui;
      invD[i] = iD;
      u[i] = ui;
      if (bi.parent < 0) continue;
      sym6_rank1_sub(Ia, Ui, iD);
      pa = pa + sym6_mul(Ia, cb[i]) + (ui * iD) * Ui;
    } else {
      if (bi.parent < 0) continue;
      pa = pa + sym6_mul(Ia, cb[i]);
    }
    sym6_add(IA[bi.parent], sym6_to_parent(X[i], Ia));
    pA[bi.parent] = pA[bi.parent] + XT_force(X[i], pa);
  }
  const SV a0 = world_accel(mv);
  for (int i = 0; i < sm.n; ++i) {
    const BodyI bi = sm.i[i];
    const SV ap = bi.parent < 0 ? a0 : va[bi.parent];
    SV ai = X_motion(X[i], ap) + cb[i];
    if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
      const float qi = (u[i] - dot(U[i], ai)) * invD[i];
      qdd[(int64_t)bi.vi * B + e] = qi;
      ai = ai + qi * S_of(sm.c[i]);
    } else if (bi.type == FST_JOINT_FREE) {
      const float* tp = tau + (int64_t)bi.vi * B + e;
      const SV tf = SV{f3{__ldg(tp + 3 * B), __ldg(tp + 4 * B), __ldg(tp + 5 * B)},
                       f3{__ldg(tp), __ldg(tp + B), __ldg(tp + 2 * B)}};
      const SV anew = sym6_solve(IA[i], tf - pA[i]);
      const SV x = anew - ai;
      float* o = qdd + (int64_t)bi.vi * B + e;
      o[0] = x.v.x;
      o[B] = x.v.y;
      o[2 * B] = x.v.z;
      o[3 * B] = x.w.x;
      o[4 * B] = x.w.y;
      o[5 * B] = x.w.z;
      ai = anew;
    }
    va[i] = ai;
  }
}

}  // namespace

cudaError_t launch_rnea(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                        float* tau, const Launch& L) {
  const size_t sh = smem_bytes(mv.n);
  FST_NB_DISPATCH(mv.n, rnea_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, qd, qdd, tau));
  return cudaGetLastError();
}

cudaError_t launch_crba(const ModelView& mv, int64_t B, const float* q, float* M, const Launch& L) {
  const size_t sh = smem_bytes(mv.n);
  FST_NB_DISPATCH(mv.n, crba_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, M));
  return cudaGetLastError();
}

cudaError_t launch_aba(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tau,
                       float* qdd, const Launch& L) {
  const size_t sh = smem_bytes(mv.n);
  FST_NB_DISPATCH(mv.n, aba_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, qd, tau, qdd));
  return cudaGetLastError();
}

}  // namespace fst
