// Per-environment bodies of the five operators. Each runs in one thread,
// reads its environment's inputs from a staged shared-memory column and
// writes its outputs straight to global memory (coalesced across the warp:
// consecutive threads hold consecutive environments of a [field][B] array).
//
// Every body is a template over the topology accessor TP (n(), C(i), I(i)):
// the generic kernels pass the run-time model in shared memory, a kernel
// compiled for one fixed tree passes compile-time constants. The per-op
// kernels and the fused evaluation kernel call the same bodies, so every
// launch form computes bit-identical results.
#pragma once

#include "fst_device.cuh"

namespace fst {

__device__ __forceinline__ SV world_accel(const ModelView& mv) {
  return SV{f3{0.f, 0.f, 0.f}, f3{mv.a0[0], mv.a0[1], mv.a0[2]}};
}

// world pose of a body from its parent's world pose and its local transform
__device__ __forceinline__ void compose(const float* Rp, const float* pp, const Xf& X, float* R, float* p) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      R[3 * r + cc] = fmaf(Rp[3 * r], X.R[cc], fmaf(Rp[3 * r + 1], X.R[3 + cc], Rp[3 * r + 2] * X.R[6 + cc]));
    p[r] = fmaf(Rp[3 * r], X.t[0], fmaf(Rp[3 * r + 1], X.t[1], fmaf(Rp[3 * r + 2], X.t[2], pp[r])));
  }
}

// Forward kinematics (tier 3 of the paper's cache, Sec. 3.1); world poses
// are kept in Rw/pw for the caller (the Jacobian reuses them) and written to
// `poses` when it is not null.
template <int NB, class TP>
__device__ __forceinline__ void world_poses(const TP& tp, const Col& q, float (&Rw)[NB][9], float (&pw)[NB][3],
                                            float* __restrict__ poses, int64_t B, int64_t e) {
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    const BodyI bi = tp.I(i);
    const Xf X = joint_X(tp.C(i), bi, q);
    if (bi.parent < 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Rw[i][k] = X.R[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) pw[i][k] = X.t[k];
    } else {
      compose(Rw[bi.parent], pw[bi.parent], X, Rw[i], pw[i]);
    }
    if (poses) {
      float* out = poses + (int64_t)i * 12 * B + e;
#pragma unroll
      for (int k = 0; k < 9; ++k) out[(int64_t)k * B] = Rw[i][k];
#pragma unroll
      for (int k = 0; k < 3; ++k) out[(int64_t)(9 + k) * B] = pw[i][k];
    }
  }
}

template <int NB, class TP>
__device__ __forceinline__ void fk_env(const TP& tp, const Col& q, float* __restrict__ poses, int64_t B, int64_t e) {
  float Rw[NB][9];
  float pw[NB][3];
  world_poses<NB>(tp, q, Rw, pw, poses, B, e);
}

// Body k's columns of one link's Jacobian straight from its world pose
// (paper Sec. 3.4, Eq. 6): w = R_k S_w, v = R_k S_v + p_k x w, i.e.
// [o_k x z_k; z_k] for a revolute joint with o_k on its axis. Rows are
// [v; w]; a DOF off the link's support path gets a zero column. Jl points at
// the link's [6][stride] block for this environment and the body's first
// column is `col`.
template <class TP>
__device__ __forceinline__ void jac_column(const TP& tp, int k, const float* Rk, const float* pk, bool on_path,
                                           int stride, int col, float* __restrict__ Jl, int64_t B) {
  const BodyI bk = tp.I(k);
  const int nvk = nv_of(bk.type);
  if (nvk == 0) return;
  const f3 p = f3{pk[0], pk[1], pk[2]};
  if (nvk == 1) {
    float c6[6] = {0, 0, 0, 0, 0, 0};
    if (on_path) {
      const SV s = S_of(tp.C(k));
      const f3 w = Rmul(Rk, s.w);
      const f3 v = Rmul(Rk, s.v) + cross(p, w);
      c6[0] = v.x; c6[1] = v.y; c6[2] = v.z;
      c6[3] = w.x; c6[4] = w.y; c6[5] = w.z;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) Jl[((int64_t)r * stride + col) * B] = c6[r];
  } else {  // free base: velocity [v; w] in body coordinates
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float c6[6] = {0, 0, 0, 0, 0, 0};
      if (on_path) {
        const int a = j % 3;
        const f3 Re = f3{Rk[a], Rk[3 + a], Rk[6 + a]};  // R e_a
        if (j < 3) {
          c6[0] = Re.x; c6[1] = Re.y; c6[2] = Re.z;
        } else {
          const f3 v = cross(p, Re);
          c6[0] = v.x; c6[1] = v.y; c6[2] = v.z;
          c6[3] = Re.x; c6[4] = Re.y; c6[5] = Re.z;
        }
      }
#pragma unroll
      for (int r = 0; r < 6; ++r) Jl[((int64_t)r * stride + col + j) * B] = c6[r];
    }
  }
}

// Every link's Jacobian from the world poses Rw/pw. Full layout: link l's
// [6][nv] block at l * 6 nv, structural zeros included. Packed (PK non-null,
// see PackedJ): only the columns of the DOFs on link l's support path.

template <int NB, class TP>
__device__ __forceinline__ void jac_from_world(const TP& tp, const float (&Rw)[NB][9], const float (&pw)[NB][3], int nv,
                                               const LinkList& links, const PackedJ* PK, float* __restrict__ J,
                                               int64_t B, int64_t e) {
  for (int l = 0; l < links.n; ++l) {
    const unsigned long long mask = tp.C(links.idx[l]).anc;
    if (!PK) {
      float* Jl = J + (int64_t)l * 6 * nv * B + e;
      FST_UNROLL
      for (int k = 0; k < tp.n(); ++k) jac_column(tp, k, Rw[k], pw[k], (mask >> k) & 1ull, nv, tp.I(k).vi, Jl, B);
    } else {
      float* Jl = J + (int64_t)PK->off[l] * B + e;
      int col = 0;
      FST_UNROLL
      for (int k = 0; k < tp.n(); ++k) {
        if (!((mask >> k) & 1ull)) continue;
        jac_column(tp, k, Rw[k], pw[k], true, PK->cols[l], col, Jl, B);
        col += nv_of(tp.I(k).type);
      }
    }
  }
}

template <int NB, class TP>
__device__ __forceinline__ void jac_env(const TP& tp, const Col& q, int nv, const LinkList& links,
                                        float* __restrict__ poses, float* __restrict__ J, int64_t B, int64_t e,
                                        const PackedJ* PK = nullptr) {
  float Rw[NB][9];
  float pw[NB][3];
  world_poses<NB>(tp, q, Rw, pw, poses, B, e);
  jac_from_world<NB>(tp, Rw, pw, nv, links, PK, J, B, e);
}

// World poses (and, when J is set, the Jacobian columns) from joint
// transforms already computed by a dynamics sweep, so a fused kernel
// evaluates each joint's transform (paper Eq. 4-5) once for all of its
// operators. The same compositions as world_poses, so the results are
// bit-identical to fk_env / jac_env.
template <int NB, class TP>
__device__ __forceinline__ void kin_from_X(const TP& tp, const Xf (&X)[NB], int nv, const LinkList& links,
                                           float* __restrict__ poses, float* __restrict__ J, int64_t B, int64_t e,
                                           const PackedJ* PK = nullptr) {
  float Rw[NB][9];
  float pw[NB][3];
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    const int par = tp.I(i).parent;
    if (par < 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Rw[i][k] = X[i].R[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) pw[i][k] = X[i].t[k];
    } else {
      compose(Rw[par], pw[par], X[i], Rw[i], pw[i]);
    }
    if (poses) {
      float* out = poses + (int64_t)i * 12 * B + e;
#pragma unroll
      for (int k = 0; k < 9; ++k) out[(int64_t)k * B] = Rw[i][k];
#pragma unroll
      for (int k = 0; k < 3; ++k) out[(int64_t)(9 + k) * B] = pw[i][k];
    }
  }
  if (J) jac_from_world<NB>(tp, Rw, pw, nv, links, PK, J, B, e);
}

// Forward sweep of RNEA (paper Sec. 3.3, Eq. 7 for the velocities):
//   v_i = X_i v_p + S_i qd_i
//   a_i = X_i a_p + S_i qdd_i + v_i x S_i qd_i     (a of the world = -g)
//   f_i = I_i a_i + v_i x* I_i v_i
template <int NB, class TP>
__device__ __forceinline__ void rnea_forward(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& qdd,
                                             Xf (&X)[NB], SV (&v)[NB], SV (&a)[NB], SV (&f)[NB]) {
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    const BodyC& c = tp.C(i);
    const BodyI bi = tp.I(i);
    X[i] = joint_X(c, bi, q);
    const SV vJ = S_times(c, bi, qd);
    const SV aJ = S_times(c, bi, qdd);
    SV vi, ai;
    if (bi.parent < 0) {
      vi = vJ;
      ai = X_motion(X[i], a0) + aJ;
    } else {
      vi = X_motion(X[i], v[bi.parent]) + vJ;
      ai = X_motion(X[i], a[bi.parent]) + aJ + crm(vi, vJ);
    }
    const In10 I = in_load(tp.theta(i));
    v[i] = vi;
    a[i] = ai;
    f[i] = in_mul(I, ai) + crf(vi, in_mul(I, vi));
  }
}

// Backward sweep of RNEA, leaf to root: F_i = f_i + sum_children X_c^T F_c,
// tau_i = S_i^T F_i. f is accumulated in place into F.
template <int NB, class TP>
__device__ __forceinline__ void rnea_backward(const TP& tp, const Xf (&X)[NB], SV (&f)[NB], float* __restrict__ tau,
                                              int64_t B, int64_t e) {
  FST_UNROLL
  for (int i = tp.n() - 1; i >= 0; --i) {
    const BodyI bi = tp.I(i);
    if (tau) ST_store(tp.C(i), bi, f[i], tau, B, e);
    if (bi.parent >= 0) f[bi.parent] = f[bi.parent] + XT_force(X[i], f[i]);
  }
}

template <int NB, class TP>
__device__ __forceinline__ void rnea_env(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& qdd,
                                         float* __restrict__ tau, int64_t B, int64_t e) {
  Xf X[NB];
  SV v[NB], a[NB], f[NB];
  rnea_forward<NB>(tp, a0, q, qd, qdd, X, v, a, f);
  rnea_backward<NB>(tp, X, f, tau, B, e);
}

// Where CRBA writes M for one environment: the full symmetric [nv][nv]
// matrix, or (PACKED) its upper triangle row by row, element (r, c), r <= c,
// at row r nv - r (r - 1) / 2 + c - r of a [nv (nv + 1) / 2][B] array.
template <bool PACKED>
struct MOut {
  float* p;  // M + e
  int nv;
  int64_t B;
  __device__ __forceinline__ int64_t row(int r, int c) const {
    if (!PACKED) return (int64_t)r * nv + c;
    return (int64_t)r * nv - (int64_t)r * (r - 1) / 2 + (c - r);
  }
  // M_rc = M_cr = x
  __device__ __forceinline__ void sym(int r, int c, float x) const {
    if (PACKED) {
      p[row(r < c ? r : c, r < c ? c : r) * B] = x;
    } else {
      p[row(r, c) * B] = x;
      p[row(c, r) * B] = x;
    }
  }
  // M_rc = x where the caller also stores M_cr (a diagonal block)
  __device__ __forceinline__ void one(int r, int c, float x) const {
    if (!PACKED || r <= c) p[row(r, c) * B] = x;
  }
};

// Composite-rigid-body algorithm: composite inertias leaf to root
// (I^c_p += X_i^T I^c_i X_i, kept as 10 parameters because a sum of rigid
// bodies is a rigid body), then F = I^c_i S_i carried up the support path:
// M_ij = S_j^T F. Ancestors have smaller indices than their descendants, so
// walking j = i-1 .. 0 over the support-path bitmask visits the path from i
// to the root in order. Structural zeros are written too.
template <int NB, bool PACKED = false, class TP>
__device__ __forceinline__ void crba_env(const TP& tp, const Col& q, int nv, float* __restrict__ M, int64_t B,
                                         int64_t e) {
  Xf X[NB];
  In10 Ic[NB];
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    X[i] = joint_X(tp.C(i), tp.I(i), q);
    Ic[i] = in_load(tp.theta(i));
  }
  FST_UNROLL
  for (int i = tp.n() - 1; i > 0; --i) {
    const int p = tp.I(i).parent;
    if (p >= 0) in_add(Ic[p], in_to_parent(X[i], Ic[i]));
  }
  const MOut<PACKED> Me{M + e, nv, B};
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    const BodyI bi = tp.I(i);
    if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
      SV F = in_mul(Ic[i], S_of(tp.C(i)));
      Me.one(bi.vi, bi.vi, dot(S_of(tp.C(i)), F));
      const unsigned long long anc = tp.C(i).anc;
      int k = i;
      FST_UNROLL
      for (int j = i - 1; j >= 0; --j) {
        if (!((anc >> j) & 1ull)) continue;
        F = XT_force(X[k], F);
        k = j;
        const BodyI bj = tp.I(j);
        if (bj.type == FST_JOINT_REVOLUTE || bj.type == FST_JOINT_PRISMATIC) {
          Me.sym(bi.vi, bj.vi, dot(S_of(tp.C(j)), F));
        } else if (bj.type == FST_JOINT_FREE) {
          const float col[6] = {F.v.x, F.v.y, F.v.z, F.w.x, F.w.y, F.w.z};
#pragma unroll
          for (int r = 0; r < 6; ++r) Me.sym(bj.vi + r, bi.vi, col[r]);
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
        for (int cc = 0; cc < 6; ++cc) Me.one(bi.vi + r, bi.vi + cc, blk[r][cc]);
    }
  }
  FST_UNROLL
  for (int i = 1; i < tp.n(); ++i) {
    const BodyI bi = tp.I(i);
    const int ni = nv_of(bi.type);
    if (ni == 0) continue;
    const unsigned long long anc_i = tp.C(i).anc;
    FST_UNROLL
    for (int j = 0; j < i; ++j) {
      const BodyI bj = tp.I(j);
      const int nj = nv_of(bj.type);
      if (nj == 0 || ((anc_i >> j) & 1ull)) continue;
      for (int r = 0; r < ni; ++r)
        for (int cc = 0; cc < nj; ++cc) Me.sym(bi.vi + r, bj.vi + cc, 0.f);
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
// With qd_zero set, qd is taken as 0 (no velocity terms at all); the adjoint
// of ABA uses that with a0 = 0 to apply M(q)^-1.
// The result is written to qdd (global, [nv][B]) and, if qdd_col is not
// null, also to that shared-memory column.
template <int NB, class TP>
__device__ __forceinline__ void aba_env(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& tau,
                                        float* __restrict__ qdd, int64_t B, int64_t e, bool qd_zero = false,
                                        float* qdd_col = nullptr, int qdd_ld = 0) {
  Xf X[NB];
  SV va[NB];  // velocity in pass 1, acceleration in pass 3
  SV cb[NB], pA[NB], U[NB];
  Sym6 IA[NB];
  float invD[NB], u[NB];
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    const BodyC& c = tp.C(i);
    const BodyI bi = tp.I(i);
    X[i] = joint_X(c, bi, q);
    const In10 I = in_load(tp.theta(i));
    IA[i] = sym6_from_in(I);
    if (qd_zero) {
      va[i] = sv_zero();
      cb[i] = sv_zero();
      pA[i] = sv_zero();
      continue;
    }
    const SV vJ = S_times(c, bi, qd);
    SV vi;
    if (bi.parent < 0) {
      vi = vJ;
      cb[i] = sv_zero();
    } else {
      vi = X_motion(X[i], va[bi.parent]) + vJ;
      cb[i] = crm(vi, vJ);
    }
    va[i] = vi;
    pA[i] = crf(vi, in_mul(I, vi));
  }
  FST_UNROLL
  for (int i = tp.n() - 1; i >= 0; --i) {
    const BodyI bi = tp.I(i);
    if (bi.type == FST_JOINT_FREE) continue;  // the root: solved in pass 3
    Sym6 Ia = IA[i];
    SV pa = pA[i];
    if (bi.type != FST_JOINT_FIXED) {
      const SV S = S_of(tp.C(i));
      const SV Ui = sym6_mul(IA[i], S);
      const float iD = 1.0f / dot(S, Ui);
      const float ui = tau[bi.vi] - dot(S, pA[i]);
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
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    const BodyI bi = tp.I(i);
    const SV ap = bi.parent < 0 ? a0 : va[bi.parent];
    SV ai = X_motion(X[i], ap) + cb[i];
    if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
      const float qi = (u[i] - dot(U[i], ai)) * invD[i];
      if (qdd) qdd[(int64_t)bi.vi * B + e] = qi;
      if (qdd_col) qdd_col[bi.vi * qdd_ld] = qi;
      ai = ai + qi * S_of(tp.C(i));
    } else if (bi.type == FST_JOINT_FREE) {
      const SV tf = SV{f3{tau[bi.vi + 3], tau[bi.vi + 4], tau[bi.vi + 5]}, f3{tau[bi.vi], tau[bi.vi + 1], tau[bi.vi + 2]}};
      const SV anew = sym6_solve(IA[i], tf - pA[i]);
      const SV x = anew - ai;
      const float xo[6] = {x.v.x, x.v.y, x.v.z, x.w.x, x.w.y, x.w.z};
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        if (qdd) qdd[(int64_t)(bi.vi + r) * B + e] = xo[r];
        if (qdd_col) qdd_col[(bi.vi + r) * qdd_ld] = xo[r];
      }
      ai = anew;
    }
    va[i] = ai;
  }
}

}  // namespace fst
