// Path-parallel operator bodies (FST_VARIANT_PATH): G lanes of one warp per
// environment, lane g sweeping the g-th root-to-leaf path of the tree.
//
// The paper's level-parallel propagation (Sec. 3.3) runs all bodies of one
// depth at once, which costs a synchronisation per level and a scatter into
// the parents on the way back. Here every lane owns one root-to-leaf path
// (in depth-first order, so a subtree's paths are adjacent lanes), and runs
// its path's bodies in depth order with the per-depth sweep state in
// registers:
//   * root-to-leaf passes need no communication at all: a body shared by
//     several paths (the spine of a legged robot) is computed by each of its
//     lanes, redundantly and identically;
//   * leaf-to-root passes need the sum over a body's children. Each lane
//     carries the contribution of the child on its own path; where a depth
//     has a body with more than one child, the lanes sharing that body
//     exchange contributions with warp shuffles (each child counted once,
//     through its leader lane, summed in lane order so that every lane of
//     the segment gets the bitwise same value).
// The serial chain of an environment shrinks from the number of bodies to
// the tree depth, and the warps per environment grow by G.
//
// Lane geometry: E = 32 / G environments per warp, lane = g * E + es.
// The topology provider TP adds, per lane g and depth t: path(g, t) (body or
// -1 past the path's end), lead_mask(g) (bit t: g is the first lane whose
// path holds that body, so it writes the body's outputs), seg(g, t) (lanes
// [lo, hi) sharing that body, lo | hi << 8), red(t) (a body at depth t has
// several children on different paths), owner(i) (leader lane of body i)
// and depth_of(i).
#pragma once

#include "ops.cuh"

namespace fst {

template <int G>
struct PathLane {
  static constexpr int E = 32 / G;
  int g, es;
  __device__ __forceinline__ PathLane() : g((int)(threadIdx.x & 31) / E), es((int)(threadIdx.x & 31) % E) {}

  // Sum of x over this environment's lanes g in [lo, hi), in lane order.
  // Every lane of the warp must call it.
  __device__ __forceinline__ float sum(float x, int lo, int hi) const {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const float y = __shfl_sync(0xffffffffu, x, k * E + es);
      if (k >= lo && k < hi) s += y;
    }
    return s;
  }
  __device__ __forceinline__ f3 sum(f3 x, int lo, int hi) const {
    return f3{sum(x.x, lo, hi), sum(x.y, lo, hi), sum(x.z, lo, hi)};
  }
  __device__ __forceinline__ SV sum(SV x, int lo, int hi) const { return SV{sum(x.w, lo, hi), sum(x.v, lo, hi)}; }
  __device__ __forceinline__ Sym6 sum(const Sym6& x, int lo, int hi) const {
    Sym6 s;
#pragma unroll
    for (int k = 0; k < 6; ++k) s.A[k] = sum(x.A[k], lo, hi);
#pragma unroll
    for (int k = 0; k < 9; ++k) s.Bk[k] = sum(x.Bk[k], lo, hi);
#pragma unroll
    for (int k = 0; k < 6; ++k) s.C[k] = sum(x.C[k], lo, hi);
    return s;
  }
  __device__ __forceinline__ In10 sum(const In10& x, int lo, int hi) const {
    In10 s;
    s.m = sum(x.m, lo, hi);
    s.h = sum(x.h, lo, hi);
#pragma unroll
    for (int k = 0; k < 6; ++k) s.I[k] = sum(x.I[k], lo, hi);
    return s;
  }
  __device__ __forceinline__ void sum2(const Sym6& x, SV y, int lo, int hi, Sym6& xo, SV& yo) const {
    xo = sum(x, lo, hi);
    yo = sum(y, lo, hi);
  }
};

// A lane's path with run-time tables (lane-group mapping): bodies per depth,
// leader bits, sharing segments.
template <int D>
struct LanePath {
  int b[D];
  int l[D], h[D];
  unsigned lead;
  int g;
  __device__ __forceinline__ int body(int t) const { return b[t]; }
  __device__ __forceinline__ bool leads(int t) const { return (lead >> t) & 1u; }
  __device__ __forceinline__ int lo(int t) const { return l[t]; }
  __device__ __forceinline__ int hi(int t) const { return h[t]; }
  __device__ __forceinline__ int index() const { return g; }
};

template <int G, int D, class TP>
__device__ __forceinline__ LanePath<D> lane_path(const TP& tp, int g) {
  LanePath<D> p;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    p.b[t] = tp.path(g, t);
    const int s = tp.seg(g, t);
    p.l[t] = s & 0xff;
    p.h[t] = s >> 8;
  }
  p.lead = tp.lead_mask(g);
  p.g = g;
  return p;
}

// Merge across the shared-memory exchange of a path-per-warp block: warp g
// holds path g of the block's 32 environments (one per lane). A merge
// writes each warp's contribution to buf[phase parity][warp][field][lane],
// waits at one block barrier and sums the segment's slots in warp order.
// Two alternating buffers make one barrier per merge enough: a warp can
// only overwrite a buffer after the next merge's barrier, which every warp
// reaches after finishing its reads of that buffer.
template <int NP, int NF>
struct SmemMerge {
  float* buf;  // 2 * NP * NF * 32 floats
  int g, lane, phase;
  template <int N>
  __device__ __forceinline__ void sum_arr(const float (&x)[N], float (&out)[N], int lo, int hi) {
    static_assert(N <= NF, "exchange slot too small");
    float* b = buf + (phase & 1) * NP * NF * 32;
#pragma unroll
    for (int f = 0; f < N; ++f) b[(g * NF + f) * 32 + lane] = x[f];
    // The warps run different (per-path) code, so this is the non-aligned
    // form of the block barrier, on its own barrier id; every warp passes
    // the same number of merges.
    asm volatile("barrier.sync 1, %0;" ::"r"(NP * 32) : "memory");
#pragma unroll
    for (int f = 0; f < N; ++f) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < NP; ++k)
        if (k >= lo && k < hi) s += b[(k * NF + f) * 32 + lane];
      out[f] = s;
    }
    ++phase;
  }
  __device__ __forceinline__ SV sum(SV x, int lo, int hi) {
    const float a[6] = {x.w.x, x.w.y, x.w.z, x.v.x, x.v.y, x.v.z};
    float o[6];
    sum_arr(a, o, lo, hi);
    return SV{f3{o[0], o[1], o[2]}, f3{o[3], o[4], o[5]}};
  }
  __device__ __forceinline__ In10 sum(const In10& x, int lo, int hi) {
    const float a[10] = {x.m, x.h.x, x.h.y, x.h.z, x.I[0], x.I[1], x.I[2], x.I[3], x.I[4], x.I[5]};
    float o[10];
    sum_arr(a, o, lo, hi);
    return in_load(o);
  }
  __device__ __forceinline__ void sum2(const Sym6& x, SV y, int lo, int hi, Sym6& xo, SV& yo) {
    float a[27], o[27];
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = x.A[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) a[6 + k] = x.Bk[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) a[15 + k] = x.C[k];
    a[21] = y.w.x; a[22] = y.w.y; a[23] = y.w.z; a[24] = y.v.x; a[25] = y.v.y; a[26] = y.v.z;
    sum_arr(a, o, lo, hi);
#pragma unroll
    for (int k = 0; k < 6; ++k) xo.A[k] = o[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) xo.Bk[k] = o[6 + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) xo.C[k] = o[15 + k];
    yo = SV{f3{o[21], o[22], o[23]}, f3{o[24], o[25], o[26]}};
  }
};

__device__ __forceinline__ Sym6 sym6_zero() {
  Sym6 s;
#pragma unroll
  for (int k = 0; k < 6; ++k) s.A[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) s.Bk[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) s.C[k] = 0.f;
  return s;
}

__device__ __forceinline__ In10 in_zero() {
  In10 s;
  s.m = 0.f;
  s.h = f3{0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 6; ++k) s.I[k] = 0.f;
  return s;
}

// ---- FK: world poses along the path ------------------------------------------
template <int D, class TP, class LP>
__device__ __forceinline__ void fk_path(const TP& tp, const LP& lp, const Col& q, Xf (&P)[D],
                                        float* __restrict__ poses, int64_t B, int64_t e, bool act) {
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const int i = lp.body(t);
    if (i < 0) continue;
    const Xf X = joint_X(tp.C(i), tp.I(i), q);
    if (t == 0)
      P[t] = X;
    else
      compose(P[t - 1].R, P[t - 1].t, X, P[t].R, P[t].t);
    if (poses && act && lp.leads(t)) {
      float* out = poses + (int64_t)i * 12 * B + e;
#pragma unroll
      for (int c = 0; c < 9; ++c) out[(int64_t)c * B] = P[t].R[c];
#pragma unroll
      for (int c = 0; c < 3; ++c) out[(int64_t)(9 + c) * B] = P[t].t[c];
    }
  }
}

// ---- Jacobians: each lane takes the links whose leader it is -------------------
template <int D, class TP, class LP>
__device__ __forceinline__ void jac_path(const TP& tp, const LP& lp, const Xf (&P)[D], int nv,
                                         const LinkList& links, float* __restrict__ J, int64_t B, int64_t e,
                                         bool act) {
  for (int r = 0; r < links.n; ++r) {
    int l = -1;
    for (int k = 0, cnt = 0; k < links.n; ++k)
      if (tp.owner(links.idx[k]) == lp.index()) {
        if (cnt == r) l = k;
        ++cnt;
      }
    if (!__any_sync(0xffffffffu, l >= 0)) break;
    if (l < 0 || !act) continue;
    const unsigned long long anc = tp.C(links.idx[l]).anc;
    float* Jl = J + (int64_t)l * 6 * nv * B + e;
    FST_UNROLL
    for (int k = 0; k < tp.n(); ++k) {
      const BodyI bk = tp.I(k);
      const int nvk = nv_of(bk.type);
      if (nvk == 0) continue;
      const bool on = (anc >> k) & 1ull;
      const Xf& Pk = P[tp.depth_of(k)];  // this lane's path holds every ancestor of its links
      const f3 p = tvec(Pk);
      if (nvk == 1) {
        float col[6] = {0, 0, 0, 0, 0, 0};
        if (on) {
          const SV s = S_of(tp.C(k));
          const f3 wv = Rmul(Pk.R, s.w);
          const f3 v = Rmul(Pk.R, s.v) + cross(p, wv);
          col[0] = v.x; col[1] = v.y; col[2] = v.z;
          col[3] = wv.x; col[4] = wv.y; col[5] = wv.z;
        }
#pragma unroll
        for (int rr = 0; rr < 6; ++rr) Jl[((int64_t)rr * nv + bk.vi) * B] = col[rr];
      } else {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          float col[6] = {0, 0, 0, 0, 0, 0};
          if (on) {
            const int a = j % 3;
            const f3 Re = f3{Pk.R[a], Pk.R[3 + a], Pk.R[6 + a]};
            if (j < 3) {
              col[0] = Re.x; col[1] = Re.y; col[2] = Re.z;
            } else {
              const f3 v = cross(p, Re);
              col[0] = v.x; col[1] = v.y; col[2] = v.z;
              col[3] = Re.x; col[4] = Re.y; col[5] = Re.z;
            }
          }
#pragma unroll
          for (int rr = 0; rr < 6; ++rr) Jl[((int64_t)rr * nv + bk.vi + j) * B] = col[rr];
        }
      }
    }
  }
}

// ---- RNEA -------------------------------------------------------------------------
template <int D, class TP, class LP, class MG>
__device__ __forceinline__ void rnea_path(const TP& tp, MG& L, const LP& lp, SV a0,
                                          const Col& q, const Col& qd, const Col& qdd, float* __restrict__ tau,
                                          int64_t B, int64_t e, bool act) {
  Xf X[D];
  SV f[D];
  SV vp = sv_zero(), ap = a0;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const int i = lp.body(t);
    if (i < 0) continue;
    const BodyC& c = tp.C(i);
    const BodyI bi = tp.I(i);
    X[t] = joint_X(c, bi, q);
    const SV vJ = S_times(c, bi, qd);
    const SV aJ = S_times(c, bi, qdd);
    SV v, a;
    if (t == 0) {
      v = vJ;
      a = X_motion(X[t], a0) + aJ;
    } else {
      v = X_motion(X[t], vp) + vJ;
      a = X_motion(X[t], ap) + aJ + crm(v, vJ);
    }
    const In10 I = in_load(tp.theta(i));
    f[t] = in_mul(I, a) + crf(v, in_mul(I, v));
    vp = v;
    ap = a;
  }
  SV cc = sv_zero();  // X_c^T F_c of the child on this lane's path
#pragma unroll
  for (int t = D - 1; t >= 0; --t) {
    const int i = lp.body(t);
    SV s = cc;
    if (t + 1 < D && tp.red(t)) s = L.sum(lp.leads(t + 1) ? cc : sv_zero(), lp.lo(t), lp.hi(t));
    if (i < 0) {
      cc = sv_zero();
      continue;
    }
    const SV F = f[t] + s;
    if (tau && act && lp.leads(t)) ST_store(tp.C(i), tp.I(i), F, tau, B, e);
    cc = t > 0 ? XT_force(X[t], F) : sv_zero();
  }
}

// ---- CRBA -------------------------------------------------------------------------
template <int D, class TP, class LP, class MG>
__device__ __forceinline__ void crba_path(const TP& tp, MG& L, const LP& lp, const Col& q,
                                          int nv, float* __restrict__ M, int64_t B, int64_t e, bool act) {
  Xf X[D];
  In10 Ic[D];
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const int i = lp.body(t);
    if (i >= 0) X[t] = joint_X(tp.C(i), tp.I(i), q);
  }
  In10 cc = in_zero();
#pragma unroll
  for (int t = D - 1; t >= 0; --t) {
    const int i = lp.body(t);
    In10 s = cc;
    if (t + 1 < D && tp.red(t)) s = L.sum(lp.leads(t + 1) ? cc : in_zero(), lp.lo(t), lp.hi(t));
    if (i < 0) {
      cc = in_zero();
      continue;
    }
    In10 I = in_load(tp.theta(i));
    in_add(I, s);
    Ic[t] = I;
    cc = t > 0 ? in_to_parent(X[t], I) : in_zero();
  }
  if (!act) return;
  float* Me = M + e;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const int i = lp.body(t);
    if (i < 0 || !lp.leads(t)) continue;
    const BodyI bi = tp.I(i);
    if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
      const SV Si = S_of(tp.C(i));
      SV F = in_mul(Ic[t], Si);
      Me[((int64_t)bi.vi * nv + bi.vi) * B] = dot(Si, F);
#pragma unroll
      for (int u = t - 1; u >= 0; --u) {
        F = XT_force(X[u + 1], F);
        const int j = lp.body(u);
        const BodyI bj = tp.I(j);
        if (bj.type == FST_JOINT_REVOLUTE || bj.type == FST_JOINT_PRISMATIC) {
          const float mij = dot(S_of(tp.C(j)), F);
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
      const In10& I = Ic[t];
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
        for (int cc2 = 0; cc2 < 6; ++cc2) Me[((int64_t)(bi.vi + r) * nv + bi.vi + cc2) * B] = blk[r][cc2];
    }
    // structural zeros of row block i against earlier bodies off its path
    const int ni = nv_of(bi.type);
    if (ni == 0) continue;
    const unsigned long long anc_i = tp.C(i).anc;
    for (int j = 0; j < i; ++j) {
      const BodyI bj = tp.I(j);
      const int nj = nv_of(bj.type);
      if (nj == 0 || ((anc_i >> j) & 1ull)) continue;
      for (int r = 0; r < ni; ++r)
        for (int c2 = 0; c2 < nj; ++c2) {
          Me[((int64_t)(bi.vi + r) * nv + bj.vi + c2) * B] = 0.f;
          Me[((int64_t)(bj.vi + c2) * nv + bi.vi + r) * B] = 0.f;
        }
    }
  }
}

// ---- ABA --------------------------------------------------------------------------
template <int D, class TP, class LP, class MG>
__device__ __forceinline__ void aba_path(const TP& tp, MG& L, const LP& lp, SV a0,
                                         const Col& q, const Col& qd, const Col& tau, float* __restrict__ qdd,
                                         int64_t B, int64_t e, bool act) {
  Xf X[D];
  SV cb[D], pA[D], U[D];
  float iD[D], uu[D];
  // 1. root to leaf: velocities, bias accelerations, bias forces
  SV vp = sv_zero();
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const int i = lp.body(t);
    if (i < 0) continue;
    const BodyC& c = tp.C(i);
    const BodyI bi = tp.I(i);
    X[t] = joint_X(c, bi, q);
    const SV vJ = S_times(c, bi, qd);
    SV v;
    if (t == 0) {
      v = vJ;
      cb[t] = sv_zero();
    } else {
      v = X_motion(X[t], vp) + vJ;
      cb[t] = crm(v, vJ);
    }
    const In10 I = in_load(tp.theta(i));
    pA[t] = crf(v, in_mul(I, v));
    vp = v;
  }
  // 2. leaf to root: articulated inertias; cI/cp carry the contribution of
  //    the child on this lane's path to its parent
  Sym6 cI = sym6_zero(), IAr = sym6_zero();
  SV cp = sv_zero(), pAr = sv_zero();
#pragma unroll
  for (int t = D - 1; t >= 0; --t) {
    const int i = lp.body(t);
    Sym6 sI = cI;
    SV sp = cp;
    if (t + 1 < D && tp.red(t)) {
      const bool mine = lp.leads(t + 1);
      L.sum2(mine ? cI : sym6_zero(), mine ? cp : sv_zero(), lp.lo(t), lp.hi(t), sI, sp);
    }
    cI = sym6_zero();
    cp = sv_zero();
    if (i < 0) continue;
    const BodyI bi = tp.I(i);
    Sym6 IA = sym6_from_in(in_load(tp.theta(i)));
    sym6_add(IA, sI);
    const SV pAi = pA[t] + sp;
    if (bi.type == FST_JOINT_FREE) {  // the root only
      IAr = IA;
      pAr = pAi;
      continue;
    }
    Sym6 Ia = IA;
    SV pa = pAi;
    if (bi.type != FST_JOINT_FIXED) {
      const SV Sv = S_of(tp.C(i));
      const SV Ui = sym6_mul(IA, Sv);
      const float invD = 1.0f / dot(Sv, Ui);
      const float ui = tau[bi.vi] - dot(Sv, pAi);
      U[t] = Ui;
      iD[t] = invD;
      uu[t] = ui;
      if (t == 0) continue;
      sym6_rank1_sub(Ia, Ui, invD);
      pa = pa + sym6_mul(Ia, cb[t]) + (ui * invD) * Ui;
    } else {
      if (t == 0) continue;
      pa = pa + sym6_mul(Ia, cb[t]);
    }
    cI = sym6_to_parent(X[t], Ia);
    cp = XT_force(X[t], pa);
  }
  // 3. root to leaf: accelerations
  SV ap = a0;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const int i = lp.body(t);
    if (i < 0) continue;
    const BodyI bi = tp.I(i);
    SV ai = X_motion(X[t], ap) + cb[t];
    if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
      const float qi = (uu[t] - dot(U[t], ai)) * iD[t];
      if (act && lp.leads(t)) qdd[(int64_t)bi.vi * B + e] = qi;
      ai = ai + qi * S_of(tp.C(i));
    } else if (bi.type == FST_JOINT_FREE) {
      const SV tf = SV{f3{tau[bi.vi + 3], tau[bi.vi + 4], tau[bi.vi + 5]}, f3{tau[bi.vi], tau[bi.vi + 1], tau[bi.vi + 2]}};
      const SV anew = sym6_solve(IAr, tf - pAr);
      const SV x = anew - ai;
      if (act && lp.leads(t)) {
        const float xo[6] = {x.v.x, x.v.y, x.v.z, x.w.x, x.w.y, x.w.z};
#pragma unroll
        for (int r = 0; r < 6; ++r) qdd[(int64_t)(bi.vi + r) * B + e] = xo[r];
      }
      ai = anew;
    }
    ap = ai;
  }
}

// Stages `rows` rows of the block's EPB environments (starting at e0) into
// tile[r * EPB + j] (zeros past B); every thread of the block takes part.
__device__ __forceinline__ void path_stage(float* tile, const float* __restrict__ src, int rows, int64_t B,
                                           int64_t e0, int EPB) {
  for (int idx = threadIdx.x; idx < rows * EPB; idx += blockDim.x) {
    const int r = idx / EPB, j = idx - r * EPB;
    const int64_t env = e0 + j;
    if (env < B)
      cp_async4(tile + idx, src + (int64_t)r * B + env);
    else
      tile[idx] = 0.f;
  }
}

}  // namespace fst
