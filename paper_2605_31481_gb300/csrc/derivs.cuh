// Dense derivatives of inverse and forward dynamics, one environment per
// thread, by forward-mode (tangent) sweeps through RNEA.
//
// The paper names analytical derivatives of the dynamics as the next step
// after its autograd gradients (Sec. 3.5 and the conclusion). For every
// degree of freedom j (motion subspace column S_j of body b) a tangent runs
// through the two RNEA sweeps:
//
//   q-tangent:  X_b moves as d(X m) = -S_j x (X m), so at b
//                 dv_b = -S_j x (X_b v_p),  da_b = -S_j x (X_b a_p) + dv_b x vJ_b
//               and below b dv_i = X_i dv_p, da_i = X_i da_p + dv_i x vJ_i;
//               on the way back d(X_b^T F_b) = X_b^T (S_j x* F_b) joins
//               dF_p = sum X_c^T dF_c.
//   qd-tangent: dv_b = S_j, da_b = S_j x ... (v_b x S_j), below b as above.
//   Both:       df_i = I da_i + dv_i x* (I v_i) + v_i x* (I dv_i),
//               dtau_i = S_i^T dF_i.
//
// Only b's subtree carries a forward tangent and only its ancestors receive
// a backward one. A free joint's q-tangent is the displacement of its moving
// frame expressed in that frame (6 directions, [dp; dw] in the velocity
// order [v; w]), the same formula with S_j = that unit twist.
//
// Forward dynamics: qdd = M^-1 (tau - C(q, qd)), so at qdd = ABA(q, qd, tau)
// d qdd / d q = -M^-1 d tau / d q, d qdd / d qd = -M^-1 d tau / d qd and
// d qdd / d tau = M^-1; M comes from CRBA and is factorised per environment
// (Cholesky, FP32) in the output buffer itself.
#pragma once

#include "ops.cuh"

namespace fst {

// Column c of body b's motion subspace, spatial [w; v]; the free joint's
// velocity order is [v; w].
__device__ __forceinline__ SV dof_S(const BodyC& c, const BodyI& b, int col) {
  if (b.type == FST_JOINT_FREE) {
    SV s = sv_zero();
    if (col < 3)
      (col == 0 ? s.v.x : col == 1 ? s.v.y : s.v.z) = 1.f;
    else
      (col == 3 ? s.w.x : col == 4 ? s.w.y : s.w.z) = 1.f;
    return s;
  }
  return S_of(c);
}

// Row r of the joint-space projection S_i^T F for body i (r < nv_of(type)).
__device__ __forceinline__ float proj_row(const BodyC& c, const BodyI& b, SV F, int r) {
  if (b.type == FST_JOINT_FREE) {
    const float o[6] = {F.v.x, F.v.y, F.v.z, F.w.x, F.w.y, F.w.z};
    return o[r];
  }
  return dot(S_of(c), F);
}

// d tau / d q (tangent directions) and d tau / d qd, [nv][nv][B] each (row =
// tau component, column = direction); either output may be null.
template <int NB, class TP>
__device__ __forceinline__ void rnea_derivs_env(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& qdd,
                                                int nv, float* __restrict__ dq, float* __restrict__ dqd, int64_t B,
                                                int64_t e) {
  Xf X[NB];
  SV v[NB], a[NB], F[NB];
  rnea_forward<NB>(tp, a0, q, qd, qdd, X, v, a, F);
  rnea_backward<NB>(tp, X, F, nullptr, B, e);  // F: accumulated forces
  const bool want_q = dq != nullptr, want_qd = dqd != nullptr;
  for (int b = 0; b < tp.n(); ++b) {
    const BodyI bb = tp.I(b);
    const int nvb = nv_of(bb.type);
    for (int col = 0; col < nvb; ++col) {
      const SV Sj = dof_S(tp.C(b), bb, col);
      const int jcol = bb.vi + col;
      SV tv[NB], ta[NB], tF[NB], uv[NB], ua[NB], uF[NB];
      FST_UNROLL
      for (int i = 0; i < tp.n(); ++i) {
        tF[i] = sv_zero();
        uF[i] = sv_zero();
        if (!((tp.C(i).anc >> b) & 1ull)) continue;  // not in b's subtree
        const BodyC& ci = tp.C(i);
        const BodyI bi = tp.I(i);
        const SV vJ = S_times(ci, bi, qd);
        SV dv, da, ev, ea;
        if (i == b) {
          const SV Xv = bi.parent < 0 ? sv_zero() : X_motion(X[i], v[bi.parent]);
          const SV Xa = X_motion(X[i], bi.parent < 0 ? a0 : a[bi.parent]);
          dv = -1.f * crm(Sj, Xv);
          da = crm(dv, vJ) - crm(Sj, Xa);
          ev = Sj;
          ea = crm(ev, vJ) + crm(v[i], Sj);
        } else {
          dv = X_motion(X[i], tv[bi.parent]);
          da = X_motion(X[i], ta[bi.parent]) + crm(dv, vJ);
          ev = X_motion(X[i], uv[bi.parent]);
          ea = X_motion(X[i], ua[bi.parent]) + crm(ev, vJ);
        }
        tv[i] = dv;
        ta[i] = da;
        uv[i] = ev;
        ua[i] = ea;
        const In10 I = in_load(tp.theta(i));
        const SV h = in_mul(I, v[i]);
        if (want_q) tF[i] = in_mul(I, da) + crf(dv, h) + crf(v[i], in_mul(I, dv));
        if (want_qd) uF[i] = in_mul(I, ea) + crf(ev, h) + crf(v[i], in_mul(I, ev));
      }
      FST_UNROLL
      for (int i = tp.n() - 1; i >= 0; --i) {
        const BodyC& ci = tp.C(i);
        const BodyI bi = tp.I(i);
        const int nvi = nv_of(bi.type);
        for (int r = 0; r < nvi; ++r) {
          const int64_t off = ((int64_t)(bi.vi + r) * nv + jcol) * B + e;
          if (want_q) dq[off] = proj_row(ci, bi, tF[i], r);
          if (want_qd) dqd[off] = proj_row(ci, bi, uF[i], r);
        }
        if (bi.parent >= 0) {
          SV t = tF[i];
          if (i == b) t = t + crf(Sj, F[i]);
          tF[bi.parent] = tF[bi.parent] + XT_force(X[i], t);
          uF[bi.parent] = uF[bi.parent] + XT_force(X[i], uF[i]);
        }
      }
    }
  }
}

// Element (r, c) of an environment's [n][n][B] matrix.
struct EnvMat {
  float* p;
  int n;
  int64_t B;
  __device__ __forceinline__ float& operator()(int r, int c) const { return p[((int64_t)r * n + c) * B]; }
};

// In-place Cholesky M = L L^T (lower triangle); returns false if a pivot is
// not positive (the matrix is then left partly factorised).
__device__ __forceinline__ bool chol_inplace(const EnvMat& M) {
  bool ok = true;
  for (int j = 0; j < M.n; ++j) {
    float d = M(j, j);
    for (int k = 0; k < j; ++k) d = fmaf(-M(j, k), M(j, k), d);
    ok = ok && d > 0.f;
    const float l = sqrtf(fmaxf(d, 1e-30f));
    M(j, j) = l;
    const float il = 1.0f / l;
    for (int i = j + 1; i < M.n; ++i) {
      float s = M(i, j);
      for (int k = 0; k < j; ++k) s = fmaf(-M(i, k), M(j, k), s);
      M(i, j) = s * il;
    }
  }
  return ok;
}

// x := -(L L^T)^-1 x for one column x (stride `ld` floats).
__device__ __forceinline__ void chol_solve_neg(const EnvMat& L, float* x, int64_t ld) {
  const int n = L.n;
  for (int i = 0; i < n; ++i) {
    float s = x[i * ld];
    for (int k = 0; k < i; ++k) s = fmaf(-L(i, k), x[k * ld], s);
    x[i * ld] = s / L(i, i);
  }
  for (int i = n - 1; i >= 0; --i) {
    float s = x[i * ld];
    for (int k = i + 1; k < n; ++k) s = fmaf(-L(k, i), x[k * ld], s);
    x[i * ld] = s / L(i, i);
  }
  for (int i = 0; i < n; ++i) x[i * ld] = -x[i * ld];
}

// M^-1 from its Cholesky factor, in place: L^-1 (lower, in place), then the
// lower triangle of L^-T L^-1 row by row (each entry only reads rows at or
// below its own, which are still L^-1), then the upper triangle by symmetry.
__device__ __forceinline__ void chol_inverse_inplace(const EnvMat& M) {
  const int n = M.n;
  for (int j = 0; j < n; ++j) {
    M(j, j) = 1.0f / M(j, j);
    for (int i = j + 1; i < n; ++i) {
      float s = 0.f;
      for (int k = j; k < i; ++k) s = fmaf(M(i, k), M(k, j), s);
      M(i, j) = -s / M(i, i);
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      float s = 0.f;
      for (int k = i; k < n; ++k) s = fmaf(M(k, i), M(k, j), s);
      M(i, j) = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) M(i, j) = M(j, i);
}

// Forward-dynamics derivatives at qdd = ABA(q, qd, tau): d qdd / d q,
// d qdd / d qd (either may be null) and M^-1 (required: it is the
// factorisation's workspace). qdd_col: this thread's staged column (stride
// ld) that receives qdd. Returns false when M was not positive definite.
template <int NB, class TP>
__device__ __forceinline__ bool aba_derivs_env(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& tau,
                                               int nv, float* qdd_col, int ld, float* __restrict__ dq,
                                               float* __restrict__ dqd, float* __restrict__ Minv, int64_t B,
                                               int64_t e) {
  aba_env<NB>(tp, a0, q, qd, tau, nullptr, B, e, false, qdd_col, ld);
  rnea_derivs_env<NB>(tp, a0, q, qd, Col{qdd_col, ld}, nv, dq, dqd, B, e);
  crba_env<NB>(tp, q, nv, Minv, B, e);
  const EnvMat L{Minv + e, nv, B};
  const bool ok = chol_inplace(L);
  for (int c = 0; c < nv; ++c) {
    if (dq) chol_solve_neg(L, dq + e + (int64_t)c * B, (int64_t)nv * B);
    if (dqd) chol_solve_neg(L, dqd + e + (int64_t)c * B, (int64_t)nv * B);
  }
  chol_inverse_inplace(L);
  return ok;
}

}  // namespace fst
