// Hand-written reverse-mode (vector-Jacobian) bodies of FK, RNEA and ABA.
//
// The paper differentiates its operators with PyTorch autograd (Sec. 3.5)
// and uses the RNEA gradient for system identification (Sec. 4.3). These
// bodies compute the same vector-Jacobian products directly, one environment
// per thread, by running each sweep backwards:
//
//   RNEA: F_i = f_i + sum_children X_c^T F_c, tau_i = S_i^T F_i, so the
//   cotangent runs root to leaf, Fbar_i = S_i taubar_i + X_i Fbar_p; then the
//   forward sweep's cotangents (vbar, abar) run leaf to root. A joint
//   transform depends on its q through d(X m)/dq = -S x (X m) and
//   d(X^T F)/dq = X^T (S x* F). The 10 inertial parameters enter linearly,
//   f = I a + v x* (I v), so thetabar is a contraction y^T (dI/dtheta) x.
//
//   ABA: qdd solves RNEA(q, qd, qdd) = tau, so for the cotangent qddbar,
//   lambda = M^-1 qddbar, taubar = lambda and
//   {qbar, qdbar, thetabar} = -RNEA-VJP(q, qd, qdd; taubar = lambda).
//   lambda comes from an ABA sweep with qd = 0, gravity 0 and tau = qddbar.
//
//   FK: world poses R_i = R_p R_pc, p_i = p_p + R_p t_pc run backwards leaf
//   to root; each joint's transform (paper Eq. 4-5) is differentiated in q.
#pragma once

#include "ops.cuh"

namespace fst {

// g += y^T (dI/dtheta) x for I * (w, u) = (I_o w + h x u, m u - h x w).
__device__ __forceinline__ void theta_contract(SV y, SV x, float* g) {
  const f3 w = x.w, u = x.v, y1 = y.w, y2 = y.v;
  g[0] += dot(y2, u);
  const f3 dh = cross(u, y1) - cross(w, y2);
  g[1] += dh.x;
  g[2] += dh.y;
  g[3] += dh.z;
  g[4] += y1.x * w.x;
  g[5] += fmaf(y1.x, w.y, y1.y * w.x);
  g[6] += y1.y * w.y;
  g[7] += fmaf(y1.x, w.z, y1.z * w.x);
  g[8] += fmaf(y1.y, w.z, y1.z * w.y);
  g[9] += y1.z * w.z;
}

// Cotangent of the unnormalised quaternion (x, y, z, w) for L = sum G_ij R_ij,
// R the rotation of the normalised quaternion (the same formula quat_R uses).
__device__ __forceinline__ void quat_grad(float x, float y, float z, float w, const float* G, float* out) {
  const float n2 = fmaf(x, x, fmaf(y, y, fmaf(z, z, w * w)));
  const float inv = rsqrtf(n2);
  x *= inv;
  y *= inv;
  z *= inv;
  w *= inv;
  float gx = 2.f * (y * (G[1] + G[3]) + z * (G[2] + G[6]) + w * (G[7] - G[5])) - 4.f * x * (G[4] + G[8]);
  float gy = 2.f * (x * (G[1] + G[3]) + z * (G[5] + G[7]) + w * (G[2] - G[6])) - 4.f * y * (G[0] + G[8]);
  float gz = 2.f * (x * (G[2] + G[6]) + y * (G[5] + G[7]) + w * (G[3] - G[1])) - 4.f * z * (G[0] + G[4]);
  float gw = 2.f * (x * (G[7] - G[5]) + y * (G[2] - G[6]) + z * (G[3] - G[1]));
  // through the normalisation q_hat = p / |p|
  const float d = x * gx + y * gy + z * gz + w * gw;
  out[0] = (gx - x * d) * inv;
  out[1] = (gy - y * d) * inv;
  out[2] = (gz - z * d) * inv;
  out[3] = (gw - w * d) * inv;
}

// Reduces the 10 per-thread values g over the warp and adds lane 0's sum
// into acc (a per-warp slot in shared memory). All 32 lanes must call it.
__device__ __forceinline__ void warp_reduce_add10(const float* g, float* acc) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    float x = g[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) acc[k] += x;
  }
}

// Where the reverse sweeps put their results.
struct VjpOut {
  float* qbar;       // [nq][B] or null
  float* qdbar;      // [nv][B] or null
  float* qddbar;     // [nv][B] or null
  float* th_warp;    // shared memory [n][10] slot of this warp, or null (no thetabar)
  float sign;        // +1 for RNEA, -1 for the ABA adjoint
  bool active;       // false for padding threads past B: they add nothing
  bool accumulate = false;  // add to q/qd/qdd bar instead of overwriting them
};

__device__ __forceinline__ void store_if(float* base, int row, int64_t B, int64_t e, float val, bool active,
                                         bool acc = false) {
  if (base && active) {
    float* p = base + (int64_t)row * B + e;
    *p = acc ? *p + val : val;
  }
}

// Reverse sweeps of the RNEA vector-Jacobian product, given the forward
// state: joint transforms X, velocities v, accelerations a and the
// accumulated forces F of every body.
template <int NB, class TP>
__device__ __forceinline__ void rnea_vjp_reverse(const TP& tp, SV a0, const Col& q, const Col& qd, const Xf (&X)[NB],
                                                 const SV (&v)[NB], const SV (&a)[NB], const SV (&F)[NB],
                                                 const Col& tbar, const VjpOut& o, int64_t B, int64_t e) {
  // root to leaf: Fbar_i = S_i taubar_i + X_i Fbar_p
  SV Fb[NB];
  float qb[NB];
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    const BodyC& c = tp.C(i);
    const BodyI bi = tp.I(i);
    SV fb = S_times(c, bi, tbar);
    qb[i] = 0.f;
    if (bi.parent >= 0) {
      const SV w = X_motion(X[i], Fb[bi.parent]);
      fb = fb + w;
      if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) qb[i] = dot(w, crf(S_of(c), F[i]));
    }
    Fb[i] = fb;
  }

  // leaf to root through the forward sweep
  SV vb[NB], ab[NB];
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    vb[i] = sv_zero();
    ab[i] = sv_zero();
  }
  FST_UNROLL
  for (int i = tp.n() - 1; i >= 0; --i) {
    const BodyC& c = tp.C(i);
    const BodyI bi = tp.I(i);
    const In10 I = in_load(tp.theta(i));
    const SV fb = Fb[i];
    // f = I a + v x* h,  h = I v
    const SV h = in_mul(I, v[i]);
    ab[i] = ab[i] + in_mul(I, fb);
    const SV hb = SV{cross(fb.w, v[i].w), cross(fb.w, v[i].v) + cross(fb.v, v[i].w)};
    vb[i] = vb[i] + SV{cross(h.w, fb.w) + cross(h.v, fb.v), cross(h.v, fb.w)} + in_mul(I, hb);
    if (o.th_warp) {
      float g[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      if (o.active) {
        theta_contract(fb, a[i], g);
        theta_contract(hb, v[i], g);
#pragma unroll
        for (int k = 0; k < 10; ++k) g[k] *= o.sign;
      }
      warp_reduce_add10(g, o.th_warp + 10 * i);
    }
    const bool one = bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC;
    float qbi = qb[i], qdbi = 0.f;
    const SV S = one ? S_of(c) : sv_zero();
    if (bi.parent >= 0) {
      // a = X a_p + S qdd + v x vJ
      const SV vJ = S_times(c, bi, qd);
      const SV cb = ab[i];
      vb[i] = vb[i] + SV{cross(vJ.w, cb.w) + cross(vJ.v, cb.v), cross(vJ.w, cb.v)};
      const SV sb = SV{cross(cb.w, v[i].w) + cross(cb.v, v[i].v), cross(cb.v, v[i].w)};
      qdbi += one ? dot(S, sb) : 0.f;
      ab[bi.parent] = ab[bi.parent] + XT_force(X[i], ab[i]);
      if (one) qbi -= dot(ab[i], crm(S, X_motion(X[i], a[bi.parent])));
      // v = X v_p + S qd
      vb[bi.parent] = vb[bi.parent] + XT_force(X[i], vb[i]);
      if (one) qbi -= dot(vb[i], crm(S, X_motion(X[i], v[bi.parent])));
    } else if (one) {
      qbi -= dot(ab[i], crm(S, X_motion(X[i], a0)));
    }
    if (one) {
      qdbi += dot(S, vb[i]);
      store_if(o.qbar, bi.qi, B, e, o.sign * qbi, o.active, o.accumulate);
      store_if(o.qdbar, bi.vi, B, e, o.sign * qdbi, o.active, o.accumulate);
      store_if(o.qddbar, bi.vi, B, e, o.sign * dot(S, ab[i]), o.active, o.accumulate);
    } else if (bi.type == FST_JOINT_FREE) {
      // a = X a0 + S qdd, v = S qd (no parent): only gravity moves with q
      const f3 g1 = RTmul(c.R0, a0.v);  // R_joint^T a0
      const float G[9] = {g1.x * ab[i].v.x, g1.x * ab[i].v.y, g1.x * ab[i].v.z,
                          g1.y * ab[i].v.x, g1.y * ab[i].v.y, g1.y * ab[i].v.z,
                          g1.z * ab[i].v.x, g1.z * ab[i].v.y, g1.z * ab[i].v.z};
      float gq[4];
      quat_grad(q[bi.qi + 3], q[bi.qi + 4], q[bi.qi + 5], q[bi.qi + 6], G, gq);
      const float qo[7] = {0.f, 0.f, 0.f, gq[0], gq[1], gq[2], gq[3]};
      const float vo[6] = {vb[i].v.x, vb[i].v.y, vb[i].v.z, vb[i].w.x, vb[i].w.y, vb[i].w.z};
      const float ao[6] = {ab[i].v.x, ab[i].v.y, ab[i].v.z, ab[i].w.x, ab[i].w.y, ab[i].w.z};
#pragma unroll
      for (int r = 0; r < 7; ++r) store_if(o.qbar, bi.qi + r, B, e, o.sign * qo[r], o.active, o.accumulate);
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        store_if(o.qdbar, bi.vi + r, B, e, o.sign * vo[r], o.active, o.accumulate);
        store_if(o.qddbar, bi.vi + r, B, e, o.sign * ao[r], o.active, o.accumulate);
      }
    }
  }
}

// RNEA vector-Jacobian product with the forward state recomputed.
template <int NB, class TP>
__device__ __forceinline__ void rnea_vjp_env(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& qdd,
                                             const Col& tbar, const VjpOut& o, int64_t B, int64_t e) {
  Xf X[NB];
  SV v[NB], a[NB], F[NB];
  rnea_forward<NB>(tp, a0, q, qd, qdd, X, v, a, F);
  rnea_backward<NB>(tp, X, F, nullptr, B, e);  // F now holds the accumulated forces
  rnea_vjp_reverse<NB>(tp, a0, q, qd, X, v, a, F, tbar, o, B, e);
}

// The RNEA role of the fused evaluation (fst_eval): ONE forward sweep whose
// joint transforms, velocities, accelerations and forces feed, as
// a.rnea_flags requests, the world poses and Jacobians, tau, and the reverse
// sweeps of the RNEA adjoint for the cotangent in column tb (staged from
// a.tau_bar, or filled here with the computed tau when EVAL_TBAR_IS_TAU).
// This is the controller step the paper times in its RL experiment (FK,
// Jacobians and RNEA each step, Sec. 4.4) with the gradient of RNEA added,
// in one pass instead of one launch per operator. Each output is
// bit-identical to the separate operator's (fk_env, jac_env, rnea_env,
// rnea_vjp_env run the same arithmetic in the same order).
template <int NB, class TP>
__device__ __forceinline__ void rnea_role_env(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& qdd,
                                              float* tb, int tb_ld, int nv, const EvalArgs& a, int64_t B,
                                              int64_t e) {
  Xf X[NB];
  SV v[NB], acc[NB], F[NB];
  rnea_forward<NB>(tp, a0, q, qd, qdd, X, v, acc, F);
  if (a.rnea_flags & EVAL_KIN_IN_RNEA)
    kin_from_X<NB>(tp, X, nv, a.links, a.poses, a.J, B, e, a.packed ? &a.pj : nullptr);
  rnea_backward<NB>(tp, X, F, a.tau_out, B, e);
  if (!(a.rnea_flags & EVAL_RNEA_VJP)) return;
  if (a.rnea_flags & EVAL_TBAR_IS_TAU) {
    FST_UNROLL
    for (int i = 0; i < tp.n(); ++i) {
      const BodyI bi = tp.I(i);
      if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
        tb[bi.vi * tb_ld] = dot(S_of(tp.C(i)), F[i]);
      } else if (bi.type == FST_JOINT_FREE) {
        const float f6[6] = {F[i].v.x, F[i].v.y, F[i].v.z, F[i].w.x, F[i].w.y, F[i].w.z};
#pragma unroll
        for (int r = 0; r < 6; ++r) tb[(bi.vi + r) * tb_ld] = f6[r];
      }
    }
  }
  const VjpOut o{a.qbar, a.qdbar, a.qddbar, nullptr, 1.f, true};
  rnea_vjp_reverse<NB>(tp, a0, q, qd, X, v, acc, F, Col{tb, tb_ld}, o, B, e);
}

// ---- store variant: the forward state on a tape -----------------------------
// Instead of recomputing the forward sweep inside the adjoint kernel, the
// forward kernel can leave, per body, the quantities the reverse sweeps read:
// the joint transform X (R row-major 9, t 3), velocity v and acceleration a
// ([w; v] each) and the accumulated force F ([n; f]). Tape layout
// [n][kTapeFloats][B], environment index fastest (coalesced).
constexpr int kTapeFloats = 30;

template <int NB, class TP>
__device__ __forceinline__ void tape_store(const TP& tp, const Xf (&X)[NB], const SV (&v)[NB], const SV (&a)[NB],
                                           const SV (&F)[NB], float* __restrict__ tape, int64_t B, int64_t e) {
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    float* p = tape + (int64_t)i * kTapeFloats * B + e;
    const float r[kTapeFloats] = {X[i].R[0], X[i].R[1], X[i].R[2], X[i].R[3], X[i].R[4], X[i].R[5], X[i].R[6],
                                  X[i].R[7], X[i].R[8], X[i].t[0], X[i].t[1], X[i].t[2], v[i].w.x, v[i].w.y,
                                  v[i].w.z,  v[i].v.x,  v[i].v.y,  v[i].v.z,  a[i].w.x,  a[i].w.y,  a[i].w.z,
                                  a[i].v.x,  a[i].v.y,  a[i].v.z,  F[i].w.x,  F[i].w.y,  F[i].w.z,  F[i].v.x,
                                  F[i].v.y,  F[i].v.z};
#pragma unroll
    for (int k = 0; k < kTapeFloats; ++k) p[(int64_t)k * B] = r[k];
  }
}

// Reads one environment's forward state back (zeros for a padding thread).
template <int NB, class TP>
__device__ __forceinline__ void tape_load(const TP& tp, const float* __restrict__ tape, int64_t B, int64_t e, bool act,
                                          Xf (&X)[NB], SV (&v)[NB], SV (&a)[NB], SV (&F)[NB]) {
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    float r[kTapeFloats];
    const float* p = tape + (int64_t)i * kTapeFloats * B + e;
#pragma unroll
    for (int k = 0; k < kTapeFloats; ++k) r[k] = act ? __ldg(p + (int64_t)k * B) : 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) X[i].R[k] = r[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) X[i].t[k] = r[9 + k];
    v[i] = SV{f3{r[12], r[13], r[14]}, f3{r[15], r[16], r[17]}};
    a[i] = SV{f3{r[18], r[19], r[20]}, f3{r[21], r[22], r[23]}};
    F[i] = SV{f3{r[24], r[25], r[26]}, f3{r[27], r[28], r[29]}};
  }
}

// RNEA forward that also writes the tape (tau optional).
template <int NB, class TP>
__device__ __forceinline__ void rnea_store_env(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& qdd,
                                               float* __restrict__ tau, float* __restrict__ tape, int64_t B,
                                               int64_t e) {
  Xf X[NB];
  SV v[NB], a[NB], F[NB];
  rnea_forward<NB>(tp, a0, q, qd, qdd, X, v, a, F);
  rnea_backward<NB>(tp, X, F, tau, B, e);
  tape_store<NB>(tp, X, v, a, F, tape, B, e);
}

// RNEA vector-Jacobian product from a tape written by rnea_store_env.
template <int NB, class TP>
__device__ __forceinline__ void rnea_vjp_stored_env(const TP& tp, SV a0, const Col& q, const Col& qd,
                                                    const float* __restrict__ tape, const Col& tbar,
                                                    const VjpOut& o, int64_t B, int64_t e) {
  Xf X[NB];
  SV v[NB], a[NB], F[NB];
  tape_load<NB>(tp, tape, B, e, o.active, X, v, a, F);
  rnea_vjp_reverse<NB>(tp, a0, q, qd, X, v, a, F, tbar, o, B, e);
}

// S_i^T f into a staged column (tau of one environment).
template <class TP>
__device__ __forceinline__ void ST_col(const TP& tp, int i, SV f, float* col, int ld) {
  const BodyI bi = tp.I(i);
  if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
    col[bi.vi * ld] = dot(S_of(tp.C(i)), f);
  } else if (bi.type == FST_JOINT_FREE) {
    const float o[6] = {f.v.x, f.v.y, f.v.z, f.w.x, f.w.y, f.w.z};
#pragma unroll
    for (int r = 0; r < 6; ++r) col[(bi.vi + r) * ld] = o[r];
  }
}

// World poses of every body (R row-major, p) and the joint transforms.
template <int NB, class TP>
__device__ __forceinline__ void fk_world(const TP& tp, const Col& q, Xf (&X)[NB], float (&Rw)[NB][9],
                                         float (&pw)[NB][3]) {
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
    const BodyI bi = tp.I(i);
    X[i] = joint_X(tp.C(i), bi, q);
    if (bi.parent < 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Rw[i][k] = X[i].R[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) pw[i][k] = X[i].t[k];
    } else {
      compose(Rw[bi.parent], pw[bi.parent], X[i], Rw[i], pw[i]);
    }
  }
}

// Reverse of fk_world: world-pose cotangents (Rb, pb; consumed) -> q_bar.
template <int NB, class TP>
__device__ __forceinline__ void fk_vjp_core(const TP& tp, const Col& q, const Xf (&X)[NB], const float (&Rw)[NB][9],
                                            float (&Rb)[NB][9], float (&pb)[NB][3], float* __restrict__ qbar,
                                            int64_t B, int64_t e) {
  FST_UNROLL
  for (int i = tp.n() - 1; i >= 0; --i) {
    const BodyC& c = tp.C(i);
    const BodyI bi = tp.I(i);
    float Rl[9], tl[3];  // cotangents of the local transform (R_pc, t_pc)
    if (bi.parent >= 0) {
      const float* Rp = Rw[bi.parent];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
          Rl[3 * a + b] = fmaf(Rp[a], Rb[i][b], fmaf(Rp[3 + a], Rb[i][3 + b], Rp[6 + a] * Rb[i][6 + b]));
        tl[a] = fmaf(Rp[a], pb[i][0], fmaf(Rp[3 + a], pb[i][1], Rp[6 + a] * pb[i][2]));
      }
      float* Rbp = Rb[bi.parent];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
          Rbp[3 * a + b] += fmaf(Rb[i][3 * a], X[i].R[3 * b],
                                 fmaf(Rb[i][3 * a + 1], X[i].R[3 * b + 1],
                                      fmaf(Rb[i][3 * a + 2], X[i].R[3 * b + 2], pb[i][a] * X[i].t[b])));
        pb[bi.parent][a] += pb[i][a];
      }
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) Rl[k] = Rb[i][k];
#pragma unroll
      for (int k = 0; k < 3; ++k) tl[k] = pb[i][k];
    }
    if (bi.type == FST_JOINT_REVOLUTE) {
      float sh, ch;
      sincosf(0.5f * q[bi.qi], &sh, &ch);
      const float s = 2.f * sh * ch;
      const float co = fmaf(-2.f * sh, sh, 1.f);
      float g = 0.f;
#pragma unroll
      for (int k = 0; k < 9; ++k) g = fmaf(Rl[k], fmaf(co, c.A[k], s * c.Bm[k]), g);
#pragma unroll
      for (int k = 0; k < 3; ++k) g = fmaf(tl[k], fmaf(co, c.a[k], s * c.b[k]), g);
      qbar[(int64_t)bi.qi * B + e] = g;
    } else if (bi.type == FST_JOINT_PRISMATIC) {
      qbar[(int64_t)bi.qi * B + e] = fmaf(tl[0], c.a[0], fmaf(tl[1], c.a[1], tl[2] * c.a[2]));
    } else if (bi.type == FST_JOINT_FREE) {
      // R = R0 Rq, t = R0 p + t0
      const f3 pg = RTmul(c.R0, f3{tl[0], tl[1], tl[2]});
      float G[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) G[3 * a + b] = fmaf(c.R0[a], Rl[b], fmaf(c.R0[3 + a], Rl[3 + b], c.R0[6 + a] * Rl[6 + b]));
      float gq[4];
      quat_grad(q[bi.qi + 3], q[bi.qi + 4], q[bi.qi + 5], q[bi.qi + 6], G, gq);
      const float out[7] = {pg.x, pg.y, pg.z, gq[0], gq[1], gq[2], gq[3]};
#pragma unroll
      for (int r = 0; r < 7; ++r) qbar[(int64_t)(bi.qi + r) * B + e] = out[r];
    }
  }
}


// FK vector-Jacobian product: poses_bar (staged [n][12] column) -> q_bar.
template <int NB, class TP>
__device__ __forceinline__ void fk_vjp_env(const TP& tp, const Col& q, const Col& pbar, float* __restrict__ qbar,
                                           int64_t B, int64_t e) {
  float Rw[NB][9];
  float pw[NB][3];
  Xf X[NB];
  fk_world<NB>(tp, q, X, Rw, pw);
  float Rb[NB][9];
  float pb[NB][3];
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
#pragma unroll
    for (int k = 0; k < 9; ++k) Rb[i][k] = pbar[12 * i + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) pb[i][k] = pbar[12 * i + 9 + k];
  }
  fk_vjp_core<NB>(tp, q, X, Rw, Rb, pb, qbar, B, e);
}

// Jacobian vector-Jacobian product: Jbar [n_links][6][nv][B] (rows [v; w])
// -> q_bar. Each column of link l's Jacobian is the world twist of a motion
// subspace column on l's support path, w = R s_w, v = R s_v + p x w (a free
// joint: R e_j, and p x R e_a with R e_a); its cotangents (vbar, wbar) give
// world-pose cotangents wbar' = wbar + vbar x p, pbar += w x vbar,
// Rbar += vbar s_v^T + wbar' s_w^T, which the FK reverse sweep takes to q.
template <int NB, class TP>
__device__ __forceinline__ void jac_vjp_env(const TP& tp, const Col& q, int nv, const LinkList& links,
                                            const float* __restrict__ Jbar, float* __restrict__ qbar, int64_t B,
                                            int64_t e) {
  float Rw[NB][9];
  float pw[NB][3];
  Xf X[NB];
  fk_world<NB>(tp, q, X, Rw, pw);
  float Rb[NB][9];
  float pb[NB][3];
  FST_UNROLL
  for (int i = 0; i < tp.n(); ++i) {
#pragma unroll
    for (int k = 0; k < 9; ++k) Rb[i][k] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) pb[i][k] = 0.f;
  }
  for (int l = 0; l < links.n; ++l) {
    const unsigned long long anc = tp.C(links.idx[l]).anc;
    const float* Jl = Jbar + (int64_t)l * 6 * nv * B + e;
    FST_UNROLL
    for (int k = 0; k < tp.n(); ++k) {
      if (!((anc >> k) & 1ull)) continue;
      const BodyI bk = tp.I(k);
      const int nvk = nv_of(bk.type);
      const f3 p = f3{pw[k][0], pw[k][1], pw[k][2]};
      for (int j = 0; j < nvk; ++j) {
        const int c = bk.vi + j;
        const f3 vb = f3{__ldg(Jl + ((int64_t)0 * nv + c) * B), __ldg(Jl + ((int64_t)1 * nv + c) * B),
                         __ldg(Jl + ((int64_t)2 * nv + c) * B)};
        const f3 wb = f3{__ldg(Jl + ((int64_t)3 * nv + c) * B), __ldg(Jl + ((int64_t)4 * nv + c) * B),
                         __ldg(Jl + ((int64_t)5 * nv + c) * B)};
        f3 sw, sv;
        if (bk.type == FST_JOINT_FREE) {
          sw = f3{0.f, 0.f, 0.f};
          sv = sw;
          if (j < 3) {
            (j == 0 ? sv.x : j == 1 ? sv.y : sv.z) = 1.f;
          } else {
            (j == 3 ? sw.x : j == 4 ? sw.y : sw.z) = 1.f;
          }
        } else {
          const SV s = S_of(tp.C(k));
          sw = s.w;
          sv = s.v;
        }
        const f3 w = f3{fmaf(Rw[k][0], sw.x, fmaf(Rw[k][1], sw.y, Rw[k][2] * sw.z)),
                        fmaf(Rw[k][3], sw.x, fmaf(Rw[k][4], sw.y, Rw[k][5] * sw.z)),
                        fmaf(Rw[k][6], sw.x, fmaf(Rw[k][7], sw.y, Rw[k][8] * sw.z))};
        const bool free_lin = bk.type == FST_JOINT_FREE && j < 3;
        const f3 wb2 = free_lin ? wb : wb + cross(vb, p);
        if (!free_lin) {
          const f3 dp = cross(w, vb);
          pb[k][0] += dp.x;
          pb[k][1] += dp.y;
          pb[k][2] += dp.z;
        }
        const float va[3] = {vb.x, vb.y, vb.z}, wa[3] = {wb2.x, wb2.y, wb2.z};
        const float svb[3] = {sv.x, sv.y, sv.z}, swb[3] = {sw.x, sw.y, sw.z};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) Rb[k][3 * a + b] += fmaf(va[a], svb[b], wa[a] * swb[b]);
      }
    }
  }
  fk_vjp_core<NB>(tp, q, X, Rw, Rb, pb, qbar, B, e);
}

}  // namespace fst
