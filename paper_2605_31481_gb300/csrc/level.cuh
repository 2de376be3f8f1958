// Level-parallel operator bodies: one block serves 32 environments (one per
// lane) and its W warps split the bodies of each tree level between them.
//
// This is the paper's level-parallel propagation (Sec. 3.3: all bodies of
// one depth are independent given their parents) mapped onto warps instead
// of batched tensor ops: warp w handles bodies level_body[k] with
// k = level_start[l] + w, + W, ... and the block synchronises once per level.
// The per-body sweep state lives in shared memory as [body][field][lane]
// (lane-contiguous, so every access is conflict-free), because a body's
// parent or children may belong to another warp. Leaf-to-root passes are
// gathers, not scatters: each body leaves its contribution to the parent in
// its own slots and the parent adds its children's after the level barrier,
// so no atomics are needed (the paper keeps these passes sequential for the
// same reason, Sec. 3.3).
//
// Every warp runs the same loops with the same trip counts, so all warps
// meet every __syncthreads(); padding lanes (environments past B) compute on
// zeros and store nothing to global memory.
#pragma once

#include "ops.cuh"

namespace fst {

constexpr int kLaneEnvs = 32;

struct LaneState {
  float* base;  // [body][F][32]
  int F;
  __device__ __forceinline__ float* at(int i, int f) const {
    return base + ((i * F + f) << 5) + (threadIdx.x & 31);
  }
  __device__ __forceinline__ SV sv(int i, int f) const {
    const float* p = at(i, f);
    return SV{f3{p[0], p[32], p[64]}, f3{p[96], p[128], p[160]}};
  }
  __device__ __forceinline__ void put(int i, int f, SV v) const {
    float* p = at(i, f);
    p[0] = v.w.x;
    p[32] = v.w.y;
    p[64] = v.w.z;
    p[96] = v.v.x;
    p[128] = v.v.y;
    p[160] = v.v.z;
  }
  __device__ __forceinline__ void get_n(int i, int f, float* out, int n) const {
    const float* p = at(i, f);
    for (int k = 0; k < n; ++k) out[k] = p[k << 5];
  }
  __device__ __forceinline__ void put_n(int i, int f, const float* in, int n) const {
    float* p = at(i, f);
    for (int k = 0; k < n; ++k) p[k << 5] = in[k];
  }
  __device__ __forceinline__ Xf X(int i, int f) const {
    Xf x;
    const float* p = at(i, f);
#pragma unroll
    for (int k = 0; k < 9; ++k) x.R[k] = p[k << 5];
#pragma unroll
    for (int k = 0; k < 3; ++k) x.t[k] = p[(9 + k) << 5];
    return x;
  }
  __device__ __forceinline__ void putX(int i, int f, const Xf& x) const {
    float* p = at(i, f);
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k << 5] = x.R[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) p[(9 + k) << 5] = x.t[k];
  }
  __device__ __forceinline__ Sym6 sym(int i, int f) const {
    Sym6 s;
    const float* p = at(i, f);
#pragma unroll
    for (int k = 0; k < 6; ++k) s.A[k] = p[k << 5];
#pragma unroll
    for (int k = 0; k < 9; ++k) s.Bk[k] = p[(6 + k) << 5];
#pragma unroll
    for (int k = 0; k < 6; ++k) s.C[k] = p[(15 + k) << 5];
    return s;
  }
  __device__ __forceinline__ void putsym(int i, int f, const Sym6& s) const {
    float* p = at(i, f);
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k << 5] = s.A[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) p[(6 + k) << 5] = s.Bk[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) p[(15 + k) << 5] = s.C[k];
  }
  __device__ __forceinline__ In10 in10(int i, int f) const {
    float t[10];
    get_n(i, f, t, 10);
    return in_load(t);
  }
  __device__ __forceinline__ void putin(int i, int f, const In10& I) const {
    const float t[10] = {I.m, I.h.x, I.h.y, I.h.z, I.I[0], I.I[1], I.I[2], I.I[3], I.I[4], I.I[5]};
    put_n(i, f, t, 10);
  }
};

// floats of per-body state per environment
constexpr int kFkState = kFkStateFloats;
constexpr int kRneaState = kRneaStateFloats;   // X 12 | v 6 | a 6 | f 6
constexpr int kCrbaState = kCrbaStateFloats;   // X 12 | Ic 10 | contribution 10
constexpr int kAbaState = kAbaStateFloats;    // X 12 | va 6 | c 6 | IA 21 | pA 6 | U 6 | invD | u

// Warps of one tile of 32 environments (lane = threadIdx.x & 31). A 1-D
// block of 32 W threads is one tile of W warps. A 3-D block (32, T, W) holds
// T tiles (threadIdx.y) of W warps (threadIdx.z) each; its hardware warp k
// belongs to tile k mod T, so each tile's first warp (the one that owns the
// first body of every level, the busiest) sits on its own SM sub-partition.
__device__ __forceinline__ int warp_id() { return (threadIdx.x >> 5) + (blockDim.x >> 5) * threadIdx.z; }
__device__ __forceinline__ int n_warps() { return (blockDim.x >> 5) * blockDim.z; }

// Stages `rows` rows of this tile's 32 environments (zeros past B);
// call from every thread, then cp_async_wait_all() and __syncthreads().
__device__ __forceinline__ void stage_block_rows(float* tile, const float* __restrict__ src, int rows, int64_t B,
                                                 int64_t e) {
  const int W = n_warps(), w = warp_id(), lane = threadIdx.x & 31;
  for (int r = w; r < rows; r += W) {
    float* d = tile + (r << 5) + lane;
    if (e < B)
      cp_async4(d, src + (int64_t)r * B + e);
    else
      *d = 0.f;
  }
}

// Loop over the bodies of level l that belong to this warp (every W-th one,
// starting at the warp's index). With a run-time topology this is a strided
// loop; with a compile-time one it is unrolled over the whole level with a
// cheap round-robin ownership test, so each body's constants fold into its
// code and each warp executes only its own bodies.
#ifdef FST_FIXED_TOPOLOGY
#define FST_FOR_MY_BODIES(tp, l, k)                                                          \
  _Pragma("unroll") for (int k = (tp).level_begin(l), own_ = 0; k < (tp).level_begin((l) + 1); \
                         ++k, own_ = (own_ + 1 == W ? 0 : own_ + 1)) if (own_ == w)
#else
#define FST_FOR_MY_BODIES(tp, l, k) for (int k = (tp).level_begin(l) + w; k < (tp).level_begin((l) + 1); k += W)
#endif


// ---- forward kinematics -------------------------------------------------------
template <class TP>
__device__ __forceinline__ void fk_level(const TP& tp, const Col& q, const LaneState& S, float* __restrict__ poses,
                                         int64_t B, int64_t e, bool act) {
  const int W = n_warps(), w = warp_id();
  FST_UNROLL
  for (int l = 0; l < tp.depth(); ++l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyI bi = tp.I(i);
      const Xf X = joint_X(tp.C(i), bi, q);
      Xf P;
      if (bi.parent < 0) {
        P = X;
      } else {
        const Xf Pp = S.X(bi.parent, 0);
        compose(Pp.R, Pp.t, X, P.R, P.t);
      }
      S.putX(i, 0, P);
      if (poses && act) {
        float* out = poses + (int64_t)i * 12 * B + e;
#pragma unroll
        for (int c = 0; c < 9; ++c) out[(int64_t)c * B] = P.R[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) out[(int64_t)(9 + c) * B] = P.t[c];
      }
    }
    __syncthreads();
  }
}

// Jacobians after fk_level: one (link, body) column per work item; columns
// of bodies off a link's support path are written as zeros. (Clearing the
// tile's rows first and writing only the support-path columns, as
// crba_level does for M, was measured slower here: the columns are cheap to
// write, and the clear adds L2 writes.)
template <class TP>
__device__ __forceinline__ void jac_columns(const TP& tp, int nv, const LinkList& links, const LaneState& S,
                                           float* __restrict__ J, int64_t B, int64_t e, bool act) {
  const int W = n_warps(), w = warp_id();
  const int n = tp.n();
  for (int item = w; item < links.n * n; item += W) {
    const int l = item / n, k = item % n;
    const BodyI bk = tp.I(k);
    const int nvk = nv_of(bk.type);
    if (nvk == 0 || !act) continue;
    const bool on_path = (tp.C(links.idx[l]).anc >> k) & 1ull;
    float* Jl = J + (int64_t)l * 6 * nv * B + e;
    const Xf P = S.X(k, 0);
    const f3 p = tvec(P);
    if (nvk == 1) {
      float col[6] = {0, 0, 0, 0, 0, 0};
      if (on_path) {
        const SV s = S_of(tp.C(k));
        const f3 wv = Rmul(P.R, s.w);
        const f3 v = Rmul(P.R, s.v) + cross(p, wv);
        col[0] = v.x; col[1] = v.y; col[2] = v.z;
        col[3] = wv.x; col[4] = wv.y; col[5] = wv.z;
      }
#pragma unroll
      for (int r = 0; r < 6; ++r) Jl[((int64_t)r * nv + bk.vi) * B] = col[r];
    } else {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        float col[6] = {0, 0, 0, 0, 0, 0};
        if (on_path) {
          const int a = j % 3;
          const f3 Re = f3{P.R[a], P.R[3 + a], P.R[6 + a]};
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

// FK, then the Jacobian columns of `links` when J is given.
template <class TP>
__device__ __forceinline__ void kin_level(const TP& tp, const Col& q, int nv, const LinkList& links,
                                          const LaneState& S, float* __restrict__ poses, float* __restrict__ J,
                                          int64_t B, int64_t e, bool act) {
  fk_level(tp, q, S, poses, B, e, act);
  if (J) jac_columns(tp, nv, links, S, J, B, e, act);
}

// ---- RNEA -----------------------------------------------------------------------
template <class TP>
__device__ __forceinline__ void rnea_level(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& qdd,
                                           const LaneState& S, float* __restrict__ tau, int64_t B, int64_t e,
                                           bool act) {
  const int W = n_warps(), w = warp_id();
  enum { X_ = 0, V_ = 12, A_ = 18, F_ = 24 };
  FST_UNROLL
  for (int l = 0; l < tp.depth(); ++l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyC& c = tp.C(i);
      const BodyI bi = tp.I(i);
      const Xf X = joint_X(c, bi, q);
      const SV vJ = S_times(c, bi, qd);
      const SV aJ = S_times(c, bi, qdd);
      SV vi, ai;
      if (bi.parent < 0) {
        vi = vJ;
        ai = X_motion(X, a0) + aJ;
      } else {
        vi = X_motion(X, S.sv(bi.parent, V_)) + vJ;
        ai = X_motion(X, S.sv(bi.parent, A_)) + aJ + crm(vi, vJ);
      }
      const In10 I = in_load(tp.theta(i));
      S.putX(i, X_, X);
      S.put(i, V_, vi);
      S.put(i, A_, ai);
      S.put(i, F_, in_mul(I, ai) + crf(vi, in_mul(I, vi)));
    }
    __syncthreads();
  }
  FST_UNROLL
  for (int l = tp.depth() - 1; l >= 0; --l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyI bi = tp.I(i);
      SV F = S.sv(i, F_);
      for (int ch = tp.child_begin(i); ch < tp.child_begin(i + 1); ++ch) F = F + S.sv(tp.child(ch), F_);
      if (act && tau) ST_store(tp.C(i), bi, F, tau, B, e);
      if (bi.parent >= 0) S.put(i, F_, XT_force(S.X(i, X_), F));
    }
    __syncthreads();
  }
}

// ---- CRBA -----------------------------------------------------------------------
// Zeros rows [0, rows) of a [rows][B] array for the tile's 32 environments
// e0 .. e0 + 31, shared among the tile's W warps (w = this warp). A full tile
// of a 16-byte aligned array with B a multiple of 4 is cleared with 16-byte
// stores (eight threads per row); otherwise with 4-byte stores, skipping
// environments past B.
__device__ __forceinline__ void m_clear_tile(float* __restrict__ M, int64_t rows, int64_t B, int64_t e0, int W,
                                             int w) {
  const int t = (threadIdx.x & 31) + (w << 5), nt = W << 5;
  if (e0 + kLaneEnvs <= B && (B & 3) == 0 && ((reinterpret_cast<unsigned long long>(M) & 15ull) == 0)) {
    const int part = t & 7;
    const int64_t step = (int64_t)(nt >> 3) * B;
    float4* p = reinterpret_cast<float4*>(M + (int64_t)(t >> 3) * B + e0 + 4 * part);
    for (int64_t r = t >> 3; r < rows; r += nt >> 3, p += step >> 2) *p = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int l = t & 31;
  if (e0 + l >= B) return;
  float* p = M + (int64_t)(t >> 5) * B + e0 + l;
  for (int64_t r = t >> 5; r < rows; r += W, p += (int64_t)W * B) *p = 0.f;
}

template <class TP>
__device__ __forceinline__ void crba_level(const TP& tp, const Col& q, int nv, const LaneState& S,
                                           float* __restrict__ M, int64_t B, int64_t e, bool act) {
  const int W = n_warps(), w = warp_id();
  enum { X_ = 0, IC_ = 12, CT_ = 22 };
  // Structural zeros: the tile clears its whole nv x nv block of M first,
  // and the column phase below overwrites the entries that are not zero.
  // The block barriers of the composite pass order the two sets of stores.
  // Nothing is read back, so DRAM sees each line once; the clear costs L2
  // writes, not a per-entry ancestry test.
  if (tp.depth() > 0) m_clear_tile(M, (int64_t)nv * nv, B, e - (threadIdx.x & 31), W, w);
  FST_UNROLL
  for (int l = tp.depth() - 1; l >= 0; --l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyI bi = tp.I(i);
      const Xf X = joint_X(tp.C(i), bi, q);
      In10 Ic = in_load(tp.theta(i));
      for (int ch = tp.child_begin(i); ch < tp.child_begin(i + 1); ++ch) in_add(Ic, S.in10(tp.child(ch), CT_));
      S.putX(i, X_, X);
      S.putin(i, IC_, Ic);
      if (bi.parent >= 0) S.putin(i, CT_, in_to_parent(X, Ic));
    }
    __syncthreads();
  }
  if (!act) return;
  float* Me = M + e;
  for (int i = w; i < tp.n(); i += W) {
    const BodyI bi = tp.I(i);
    if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
      const In10 Ic = S.in10(i, IC_);
      SV F = in_mul(Ic, S_of(tp.C(i)));
      Me[((int64_t)bi.vi * nv + bi.vi) * B] = dot(S_of(tp.C(i)), F);
      // up the support path, parent by parent (parents precede children)
      int kk = i;
      for (int j = bi.parent; j >= 0; j = tp.I(j).parent) {
        F = XT_force(S.X(kk, X_), F);
        kk = j;
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
      const In10 I = S.in10(i, IC_);
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
}

// ---- CRBA, lean shared memory ---------------------------------------------------
// Joint transform of body i with its coordinates read straight from global
// memory (rows of B; ec a valid environment index), for kernels that do not
// stage q in shared memory.
__device__ __forceinline__ Xf joint_X_rows(const BodyC& c, const BodyI& bi, const float* __restrict__ q, int64_t B,
                                           int64_t ec) {
  const int nqb = bi.type == FST_JOINT_FREE ? 7 : bi.type == FST_JOINT_FIXED ? 0 : 1;
  float qb[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) qb[k] = k < nqb ? __ldg(q + (int64_t)(bi.qi + k) * B + ec) : 0.f;
  BodyI b0 = bi;
  b0.qi = 0;
  return joint_X(c, b0, Col{qb, 1});
}

// The composite-rigid-body algorithm with less shared memory per tile (so
// that three tiles of a large tree fit on one SM): per body only X and
// F = I^c S stay (kCrbaLeanBodyFloats); a body's composite inertia moved to
// its parent lives in ring R, slot (level parity, position within the
// level), until the parent has added it; the root keeps its own I^c in its
// level-0 slot for a free base's 6 x 6 block. q is read from global memory,
// not staged. Same arithmetic, in the same order, as crba_level.
template <class TP>
__device__ __forceinline__ void crba_level_lean(const TP& tp, const float* __restrict__ q, int nv,
                                                const LaneState& S, const LaneState& R, int maxw,
                                                float* __restrict__ M, int64_t B, int64_t e, bool act) {
  const int W = n_warps(), w = warp_id();
  enum { X_ = 0, F_ = 12 };
  const int64_t ec = act ? e : B - 1;  // lanes past B compute on the last environment and store nothing
  if (tp.depth() > 0) m_clear_tile(M, (int64_t)nv * nv, B, e - (threadIdx.x & 31), W, w);
  FST_UNROLL
  for (int l = tp.depth() - 1; l >= 0; --l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyI bi = tp.I(i);
      const int slot = (l & 1) * maxw + (k - tp.level_begin(l));
      const int child_ring = ((l + 1) & 1) * maxw;
      const Xf X = joint_X_rows(tp.C(i), bi, q, B, ec);
      In10 Ic = in_load(tp.theta(i));
      for (int ch = tp.child_begin(i); ch < tp.child_begin(i + 1); ++ch)
        in_add(Ic, R.in10(child_ring + tp.C(tp.child(ch)).lpos, 0));
      S.putX(i, X_, X);
      if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) S.put(i, F_, in_mul(Ic, S_of(tp.C(i))));
      R.putin(slot, 0, bi.parent >= 0 ? in_to_parent(X, Ic) : Ic);
    }
    __syncthreads();
  }
  if (!act) return;
  float* Me = M + e;
  for (int i = w; i < tp.n(); i += W) {
    const BodyI bi = tp.I(i);
    if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
      SV F = S.sv(i, F_);
      Me[((int64_t)bi.vi * nv + bi.vi) * B] = dot(S_of(tp.C(i)), F);
      int kk = i;
      for (int j = bi.parent; j >= 0; j = tp.I(j).parent) {
        F = XT_force(S.X(kk, X_), F);
        kk = j;
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
      const In10 I = R.in10(tp.C(i).lpos, 0);  // the root's own slot (level 0, parity 0)
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
}

// ---- ABA ------------------------------------------------------------------------
template <class TP>
__device__ __forceinline__ void aba_level(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& tau,
                                          const LaneState& S, float* __restrict__ qdd, int64_t B, int64_t e,
                                          bool act) {
  const int W = n_warps(), w = warp_id();
  enum { X_ = 0, VA_ = 12, C_ = 18, IA_ = 24, PA_ = 45, U_ = 51, ID_ = 57, u_ = 58 };
  // 1. root to leaf: velocities, bias accelerations, rigid inertias
  FST_UNROLL
  for (int l = 0; l < tp.depth(); ++l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyC& c = tp.C(i);
      const BodyI bi = tp.I(i);
      const Xf X = joint_X(c, bi, q);
      const SV vJ = S_times(c, bi, qd);
      SV vi, ci;
      if (bi.parent < 0) {
        vi = vJ;
        ci = sv_zero();
      } else {
        vi = X_motion(X, S.sv(bi.parent, VA_)) + vJ;
        ci = crm(vi, vJ);
      }
      const In10 I = in_load(tp.theta(i));
      S.putX(i, X_, X);
      S.put(i, VA_, vi);
      S.put(i, C_, ci);
      S.putsym(i, IA_, sym6_from_in(I));
      S.put(i, PA_, crf(vi, in_mul(I, vi)));
    }
    __syncthreads();
  }
  // 2. leaf to root: articulated inertias; each body leaves X^T I^a X and
  //    X^T p^a for its parent in its own IA/PA slots
  FST_UNROLL
  for (int l = tp.depth() - 1; l >= 0; --l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyI bi = tp.I(i);
      Sym6 IA = S.sym(i, IA_);
      SV pA = S.sv(i, PA_);
      for (int ch = tp.child_begin(i); ch < tp.child_begin(i + 1); ++ch) {
        sym6_add(IA, S.sym(tp.child(ch), IA_));
        pA = pA + S.sv(tp.child(ch), PA_);
      }
      if (bi.type == FST_JOINT_FREE) {
        S.putsym(i, IA_, IA);
        S.put(i, PA_, pA);
        continue;
      }
      Sym6 Ia = IA;
      SV pa = pA;
      if (bi.type != FST_JOINT_FIXED) {
        const SV Sv = S_of(tp.C(i));
        const SV Ui = sym6_mul(IA, Sv);
        const float iD = 1.0f / dot(Sv, Ui);
        const float ui = tau[bi.vi] - dot(Sv, pA);
        S.put(i, U_, Ui);
        *S.at(i, ID_) = iD;
        *S.at(i, u_) = ui;
        if (bi.parent < 0) continue;
        sym6_rank1_sub(Ia, Ui, iD);
        pa = pa + sym6_mul(Ia, S.sv(i, C_)) + (ui * iD) * Ui;
      } else {
        if (bi.parent < 0) continue;
        pa = pa + sym6_mul(Ia, S.sv(i, C_));
      }
      const Xf X = S.X(i, X_);
      S.putsym(i, IA_, sym6_to_parent(X, Ia));
      S.put(i, PA_, XT_force(X, pa));
    }
    __syncthreads();
  }
  // 3. root to leaf: accelerations
  FST_UNROLL
  for (int l = 0; l < tp.depth(); ++l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyI bi = tp.I(i);
      const SV ap = bi.parent < 0 ? a0 : S.sv(bi.parent, VA_);
      SV ai = X_motion(S.X(i, X_), ap) + S.sv(i, C_);
      if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
        const float qi = (*S.at(i, u_) - dot(S.sv(i, U_), ai)) * *S.at(i, ID_);
        if (act) qdd[(int64_t)bi.vi * B + e] = qi;
        ai = ai + qi * S_of(tp.C(i));
      } else if (bi.type == FST_JOINT_FREE) {
        const SV tf = SV{f3{tau[bi.vi + 3], tau[bi.vi + 4], tau[bi.vi + 5]}, f3{tau[bi.vi], tau[bi.vi + 1], tau[bi.vi + 2]}};
        const SV anew = sym6_solve(S.sym(i, IA_), tf - S.sv(i, PA_));
        const SV x = anew - ai;
        if (act) {
          const float xo[6] = {x.v.x, x.v.y, x.v.z, x.w.x, x.w.y, x.w.z};
#pragma unroll
          for (int r = 0; r < 6; ++r) qdd[(int64_t)(bi.vi + r) * B + e] = xo[r];
        }
        ai = anew;
      }
      S.put(i, VA_, ai);
    }
    __syncthreads();
  }
}

// ---- ABA, lean shared memory ------------------------------------------------------
// The same three passes with less state per tile, so that a large tree's
// tiles fit two per SM: per body only VU (v in pass 1, U from pass 2, a in
// pass 3), c, invD and u stay (kAbaLeanBodyFloats); a body's contribution to
// its parent (X^T I^a X, X^T p^a) lives in ring R, slot (level parity,
// position within the level), only until the parent has read it
// (kAbaLeanRingFloats each, 2 x widest level slots); the rigid inertia and
// the bias force are formed in pass 2, and the joint transforms recomputed
// in passes 2 and 3 instead of stored. The root's I^A and p^A, which pass 3
// needs for a free base, stay in its level-0 ring slot.
template <class TP>
__device__ __forceinline__ void aba_level_lean(const TP& tp, SV a0, const Col& q, const Col& qd, const Col& tau,
                                               const LaneState& S, const LaneState& R, int maxw,
                                               float* __restrict__ qdd, int64_t B, int64_t e, bool act) {
  const int W = n_warps(), w = warp_id();
  enum { VU_ = 0, C_ = 6, ID_ = 12, u_ = 13 };  // per body
  enum { RI_ = 0, RP_ = 21 };                      // per ring slot
  // 1. root to leaf: velocities and bias accelerations
  FST_UNROLL
  for (int l = 0; l < tp.depth(); ++l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyC& c = tp.C(i);
      const BodyI bi = tp.I(i);
      const SV vJ = S_times(c, bi, qd);
      SV vi, ci;
      if (bi.parent < 0) {
        vi = vJ;
        ci = sv_zero();
      } else {
        vi = X_motion(joint_X(c, bi, q), S.sv(bi.parent, VU_)) + vJ;
        ci = crm(vi, vJ);
      }
      S.put(i, VU_, vi);
      S.put(i, C_, ci);
    }
    __syncthreads();
  }
  // 2. leaf to root: articulated inertias; a body of level l leaves its
  //    contribution in ring slot (l & 1) * maxw + its position in the level
  FST_UNROLL
  for (int l = tp.depth() - 1; l >= 0; --l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyI bi = tp.I(i);
      const int slot = (l & 1) * maxw + (k - tp.level_begin(l));
      const int child_ring = ((l + 1) & 1) * maxw;
      const In10 I = in_load(tp.theta(i));
      const SV vi = S.sv(i, VU_);
      Sym6 IA = sym6_from_in(I);
      SV pA = crf(vi, in_mul(I, vi));
      for (int ch = tp.child_begin(i); ch < tp.child_begin(i + 1); ++ch) {
        const int cs = child_ring + tp.C(tp.child(ch)).lpos;
        sym6_add(IA, R.sym(cs, RI_));
        pA = pA + R.sv(cs, RP_);
      }
      if (bi.type == FST_JOINT_FREE) {
        R.putsym(slot, RI_, IA);
        R.put(slot, RP_, pA);
        continue;
      }
      Sym6 Ia = IA;
      SV pa = pA;
      if (bi.type != FST_JOINT_FIXED) {
        const SV Sv = S_of(tp.C(i));
        const SV Ui = sym6_mul(IA, Sv);
        const float iD = 1.0f / dot(Sv, Ui);
        const float ui = tau[bi.vi] - dot(Sv, pA);
        S.put(i, VU_, Ui);
        *S.at(i, ID_) = iD;
        *S.at(i, u_) = ui;
        if (bi.parent < 0) continue;
        sym6_rank1_sub(Ia, Ui, iD);
        pa = pa + sym6_mul(Ia, S.sv(i, C_)) + (ui * iD) * Ui;
      } else {
        if (bi.parent < 0) continue;
        pa = pa + sym6_mul(Ia, S.sv(i, C_));
      }
      const Xf X = joint_X(tp.C(i), bi, q);
      R.putsym(slot, RI_, sym6_to_parent(X, Ia));
      R.put(slot, RP_, XT_force(X, pa));
    }
    __syncthreads();
  }
  // 3. root to leaf: accelerations (each body reads its U before it
  //    overwrites VU with its acceleration)
  FST_UNROLL
  for (int l = 0; l < tp.depth(); ++l) {
    FST_FOR_MY_BODIES(tp, l, k) {
      const int i = tp.level_body(k);
      const BodyI bi = tp.I(i);
      const SV ap = bi.parent < 0 ? a0 : S.sv(bi.parent, VU_);
      SV ai = X_motion(joint_X(tp.C(i), bi, q), ap) + S.sv(i, C_);
      if (bi.type == FST_JOINT_REVOLUTE || bi.type == FST_JOINT_PRISMATIC) {
        const float qi = (*S.at(i, u_) - dot(S.sv(i, VU_), ai)) * *S.at(i, ID_);
        if (act) qdd[(int64_t)bi.vi * B + e] = qi;
        ai = ai + qi * S_of(tp.C(i));
      } else if (bi.type == FST_JOINT_FREE) {
        const int slot = k - tp.level_begin(l);  // level 0: ring parity 0
        const SV tf = SV{f3{tau[bi.vi + 3], tau[bi.vi + 4], tau[bi.vi + 5]}, f3{tau[bi.vi], tau[bi.vi + 1], tau[bi.vi + 2]}};
        const SV anew = sym6_solve(R.sym(slot, RI_), tf - R.sv(slot, RP_));
        const SV x = anew - ai;
        if (act) {
          const float xo[6] = {x.v.x, x.v.y, x.v.z, x.w.x, x.w.y, x.w.z};
#pragma unroll
          for (int r = 0; r < 6; ++r) qdd[(int64_t)(bi.vi + r) * B + e] = xo[r];
        }
        ai = anew;
      }
      S.put(i, VU_, ai);
    }
    __syncthreads();
  }
}

}  // namespace fst
