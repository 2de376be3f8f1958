// Device-side spatial algebra for one environment per thread.
//
// Motion vectors are (w, v) and force vectors (n, f), angular first. A joint
// transform is kept as the child's pose in its parent, (R, t) with
// p_parent = R p_child + t, and applied directly; the 6x6 Plucker matrix
// X_up = [[R^T, 0], [-R^T [t]x, R^T]] is never formed (the paper stores
// X_up and X_up^T side by side as 6x6 tensors, Sec. 3.5; here both products
// are a handful of 3x3 operations on registers).
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif

#include "fst_layout.h"

namespace fst {

struct f3 {
  float x, y, z;
};

__device__ __forceinline__ f3 mk3(float x, float y, float z) { return f3{x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return f3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return f3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator-(f3 a) { return f3{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return f3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
  return f3{fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x)};
}

// R (row-major 9) times x, and R^T times x
__device__ __forceinline__ f3 Rmul(const float* R, f3 x) {
  return f3{fmaf(R[0], x.x, fmaf(R[1], x.y, R[2] * x.z)), fmaf(R[3], x.x, fmaf(R[4], x.y, R[5] * x.z)),
            fmaf(R[6], x.x, fmaf(R[7], x.y, R[8] * x.z))};
}
__device__ __forceinline__ f3 RTmul(const float* R, f3 x) {
  return f3{fmaf(R[0], x.x, fmaf(R[3], x.y, R[6] * x.z)), fmaf(R[1], x.x, fmaf(R[4], x.y, R[7] * x.z)),
            fmaf(R[2], x.x, fmaf(R[5], x.y, R[8] * x.z))};
}

struct Xf {
  float R[9];
  float t[3];
};
struct SV {
  f3 w, v;  // motion (w, v) or force (n, f)
};

__device__ __forceinline__ SV operator+(SV a, SV b) { return SV{a.w + b.w, a.v + b.v}; }
__device__ __forceinline__ SV operator-(SV a, SV b) { return SV{a.w - b.w, a.v - b.v}; }
__device__ __forceinline__ SV operator*(float s, SV a) { return SV{s * a.w, s * a.v}; }
__device__ __forceinline__ float dot(SV a, SV b) { return dot(a.w, b.w) + dot(a.v, b.v); }
__device__ __forceinline__ SV sv_zero() { return SV{f3{0, 0, 0}, f3{0, 0, 0}}; }
__device__ __forceinline__ f3 tvec(const Xf& X) { return f3{X.t[0], X.t[1], X.t[2]}; }

// motion, parent coordinates -> child coordinates (X_up m)
__device__ __forceinline__ SV X_motion(const Xf& X, SV m) {
  f3 t = tvec(X);
  return SV{RTmul(X.R, m.w), RTmul(X.R, m.v - cross(t, m.w))};
}
// motion, child coordinates -> parent coordinates (X_up^-1 m)
__device__ __forceinline__ SV Xinv_motion(const Xf& X, SV m) {
  f3 w = Rmul(X.R, m.w);
  return SV{w, Rmul(X.R, m.v) + cross(tvec(X), w)};
}
// force, child coordinates -> parent coordinates (X_up^T f)
__device__ __forceinline__ SV XT_force(const Xf& X, SV f) {
  f3 fl = Rmul(X.R, f.v);
  return SV{Rmul(X.R, f.w) + cross(tvec(X), fl), fl};
}
// motion cross product v x m (Featherstone crm)
__device__ __forceinline__ SV crm(SV v, SV m) { return SV{cross(v.w, m.w), cross(v.w, m.v) + cross(v.v, m.w)}; }
// force cross product v x* f (Featherstone crf)
__device__ __forceinline__ SV crf(SV v, SV f) { return SV{cross(v.w, f.w) + cross(v.v, f.v), cross(v.w, f.v)}; }

// Rigid-body inertia by its 10 linear parameters about the frame origin.
struct In10 {
  float m;
  f3 h;       // m * com
  float I[6]; // xx xy yy xz yz zz
};

__device__ __forceinline__ f3 sym_mul(const float* I, f3 w) {
  return f3{fmaf(I[0], w.x, fmaf(I[1], w.y, I[3] * w.z)), fmaf(I[1], w.x, fmaf(I[2], w.y, I[4] * w.z)),
            fmaf(I[3], w.x, fmaf(I[4], w.y, I[5] * w.z))};
}
// I * (w, v) = (I_o w + h x v, m v - h x w)
__device__ __forceinline__ SV in_mul(const In10& I, SV m) {
  return SV{sym_mul(I.I, m.w) + cross(I.h, m.v), I.m * m.v - cross(I.h, m.w)};
}
__device__ __forceinline__ In10 in_load(const float* th) {
  In10 I;
  I.m = th[0];
  I.h = f3{th[1], th[2], th[3]};
#pragma unroll
  for (int k = 0; k < 6; ++k) I.I[k] = th[4 + k];
  return I;
}
__device__ __forceinline__ void in_add(In10& a, const In10& b) {
  a.m += b.m;
  a.h = a.h + b.h;
#pragma unroll
  for (int k = 0; k < 6; ++k) a.I[k] += b.I[k];
}

// R S R^T for a symmetric S (6 entries), result symmetric (6 entries)
__device__ __forceinline__ void sym_rot(const float* R, const float* S, float* out) {
  // P = R S (3x3 full)
  float P[9];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    f3 row = sym_mul(S, f3{R[3 * r], R[3 * r + 1], R[3 * r + 2]});  // (S R_r^T) = (R_r S)^T since S sym
    P[3 * r] = row.x;
    P[3 * r + 1] = row.y;
    P[3 * r + 2] = row.z;
  }
  // out_ab = sum_k P_ak R_bk
  out[0] = fmaf(P[0], R[0], fmaf(P[1], R[1], P[2] * R[2]));
  out[1] = fmaf(P[0], R[3], fmaf(P[1], R[4], P[2] * R[5]));
  out[2] = fmaf(P[3], R[3], fmaf(P[4], R[4], P[5] * R[5]));
  out[3] = fmaf(P[0], R[6], fmaf(P[1], R[7], P[2] * R[8]));
  out[4] = fmaf(P[3], R[6], fmaf(P[4], R[7], P[5] * R[8]));
  out[5] = fmaf(P[6], R[6], fmaf(P[7], R[7], P[8] * R[8]));
}

// X^T I X for a rigid-body inertia given in child coordinates: the same body
// expressed about the parent origin in parent coordinates.
//   h' = R h + m t
//   I' = R I R^T + (2 y.t + m |t|^2) 1 - (y t^T + t y^T + m t t^T),  y = R h
__device__ __forceinline__ In10 in_to_parent(const Xf& X, const In10& I) {
  In10 o;
  o.m = I.m;
  f3 y = Rmul(X.R, I.h);
  f3 t = tvec(X);
  o.h = y + I.m * t;
  sym_rot(X.R, I.I, o.I);
  float d = fmaf(2.0f, dot(y, t), I.m * dot(t, t));
  f3 z = y + (0.5f * I.m) * t;  // y t^T + t y^T + m t t^T = z t^T + t z^T
  o.I[0] += d - 2.0f * z.x * t.x;
  o.I[1] -= fmaf(z.x, t.y, t.x * z.y);
  o.I[2] += d - 2.0f * z.y * t.y;
  o.I[3] -= fmaf(z.x, t.z, t.x * z.z);
  o.I[4] -= fmaf(z.y, t.z, t.y * z.z);
  o.I[5] += d - 2.0f * z.z * t.z;
  return o;
}

// General symmetric 6x6 spatial matrix [[A, Bk], [Bk^T, C]] (21 floats),
// used for articulated-body inertias, which are not rigid-body inertias.
struct Sym6 {
  float A[6];  // sym, xx xy yy xz yz zz
  float Bk[9]; // full, row-major
  float C[6];  // sym
};

__device__ __forceinline__ Sym6 sym6_from_in(const In10& I) {
  Sym6 s;
#pragma unroll
  for (int k = 0; k < 6; ++k) s.A[k] = I.I[k];
  // Bk = [h]x
  s.Bk[0] = 0.f;
  s.Bk[1] = -I.h.z;
  s.Bk[2] = I.h.y;
  s.Bk[3] = I.h.z;
  s.Bk[4] = 0.f;
  s.Bk[5] = -I.h.x;
  s.Bk[6] = -I.h.y;
  s.Bk[7] = I.h.x;
  s.Bk[8] = 0.f;
  s.C[0] = I.m;
  s.C[1] = 0.f;
  s.C[2] = I.m;
  s.C[3] = 0.f;
  s.C[4] = 0.f;
  s.C[5] = I.m;
  return s;
}

// (A w + Bk v, Bk^T w + C v)
__device__ __forceinline__ SV sym6_mul(const Sym6& s, SV m) {
  return SV{sym_mul(s.A, m.w) + Rmul(s.Bk, m.v), RTmul(s.Bk, m.w) + sym_mul(s.C, m.v)};
}

__device__ __forceinline__ void sym6_add(Sym6& a, const Sym6& b) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    a.A[k] += b.A[k];
    a.C[k] += b.C[k];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) a.Bk[k] += b.Bk[k];
}

// s -= U U^T * invD, with U = (Un, Uf) a force-space 6-vector
__device__ __forceinline__ void sym6_rank1_sub(Sym6& s, SV U, float invD) {
  f3 n = U.w, f = U.v;
  f3 ns = invD * n, fs = invD * f;
  s.A[0] -= ns.x * n.x;
  s.A[1] -= ns.x * n.y;
  s.A[2] -= ns.y * n.y;
  s.A[3] -= ns.x * n.z;
  s.A[4] -= ns.y * n.z;
  s.A[5] -= ns.z * n.z;
  s.C[0] -= fs.x * f.x;
  s.C[1] -= fs.x * f.y;
  s.C[2] -= fs.y * f.y;
  s.C[3] -= fs.x * f.z;
  s.C[4] -= fs.y * f.z;
  s.C[5] -= fs.z * f.z;
  s.Bk[0] -= ns.x * f.x;
  s.Bk[1] -= ns.x * f.y;
  s.Bk[2] -= ns.x * f.z;
  s.Bk[3] -= ns.y * f.x;
  s.Bk[4] -= ns.y * f.y;
  s.Bk[5] -= ns.y * f.z;
  s.Bk[6] -= ns.z * f.x;
  s.Bk[7] -= ns.z * f.y;
  s.Bk[8] -= ns.z * f.z;
}

// R M R^T for a full 3x3 M
__device__ __forceinline__ void full_rot(const float* R, const float* M, float* out) {
  float P[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) P[3 * r + c] = fmaf(R[3 * r], M[c], fmaf(R[3 * r + 1], M[3 + c], R[3 * r + 2] * M[6 + c]));
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * r + c] = fmaf(P[3 * r], R[3 * c], fmaf(P[3 * r + 1], R[3 * c + 1], P[3 * r + 2] * R[3 * c + 2]));
}

// X^T s X: a symmetric spatial matrix from child to parent coordinates.
// With A', Bk', C' the blocks rotated by R and T = [t]x:
//   C'' = C',  Bk'' = Bk' + T C',  A'' = A' - Y - Y^T,  Y = (Bk' + T C' / 2) T
__device__ __forceinline__ Sym6 sym6_to_parent(const Xf& X, const Sym6& s) {
  Sym6 o;
  sym_rot(X.R, s.A, o.A);
  sym_rot(X.R, s.C, o.C);
  float Bp[9];
  full_rot(X.R, s.Bk, Bp);
  const float tx = X.t[0], ty = X.t[1], tz = X.t[2];
  // W = T C' (C' symmetric: c00=C[0], c01=C[1], c11=C[2], c02=C[3], c12=C[4], c22=C[5])
  const float* C = o.C;
  float Cf[9] = {C[0], C[1], C[3], C[1], C[2], C[4], C[3], C[4], C[5]};
  float W[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    W[c] = fmaf(-tz, Cf[3 + c], ty * Cf[6 + c]);
    W[3 + c] = fmaf(tz, Cf[c], -tx * Cf[6 + c]);
    W[6 + c] = fmaf(-ty, Cf[c], tx * Cf[3 + c]);
  }
  float Z[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    o.Bk[k] = Bp[k] + W[k];
    Z[k] = fmaf(0.5f, W[k], Bp[k]);
  }
  // Y = Z T, T = [[0,-tz,ty],[tz,0,-tx],[-ty,tx,0]]
  float Y[9];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Y[3 * r + 0] = fmaf(Z[3 * r + 1], tz, -Z[3 * r + 2] * ty);
    Y[3 * r + 1] = fmaf(-Z[3 * r + 0], tz, Z[3 * r + 2] * tx);
    Y[3 * r + 2] = fmaf(Z[3 * r + 0], ty, -Z[3 * r + 1] * tx);
  }
  o.A[0] -= 2.0f * Y[0];
  o.A[1] -= Y[1] + Y[3];
  o.A[2] -= 2.0f * Y[4];
  o.A[3] -= Y[2] + Y[6];
  o.A[4] -= Y[5] + Y[7];
  o.A[5] -= 2.0f * Y[8];
  return o;
}

// ---------------------------------------------------------------------------
// model staging and joint transforms
// ---------------------------------------------------------------------------

// Loops over bodies: left rolled in the generic kernels (the topology is
// read at run time from shared memory), fully unrolled when a kernel is
// compiled for one fixed tree (then every body index is a compile-time
// constant and the per-body sweep state can live in registers).
#ifdef FST_FIXED_TOPOLOGY
#define FST_UNROLL _Pragma("unroll")
#else
#define FST_UNROLL _Pragma("unroll 1")
#endif

// Run-time topology: the model staged in shared memory. Any type with the
// same accessors (n, C, I, theta; depth and the level/child lists for the
// level-parallel kernels) can drive the operator templates.
struct SmemModel {
  const BodyC* c;
  const BodyI* i;
  int n_;
  const TopoLists* t = nullptr;
  int depth_ = 0;
  __device__ __forceinline__ int n() const { return n_; }
  __device__ __forceinline__ const BodyC& C(int k) const { return c[k]; }
  __device__ __forceinline__ BodyI I(int k) const { return i[k]; }
  // inertial parameters (the override, if any, was staged in place)
  __device__ __forceinline__ const float* theta(int k) const { return c[k].theta; }
  __device__ __forceinline__ int depth() const { return depth_; }
  __device__ __forceinline__ int level_begin(int l) const { return t->level_start[l]; }
  __device__ __forceinline__ int level_body(int k) const { return t->level_body[k]; }
  __device__ __forceinline__ int child_begin(int k) const { return t->child_start[k]; }
  __device__ __forceinline__ int child(int k) const { return t->child[k]; }
};

// Asynchronous global -> shared copies (no register staging, so a thread
// issues all of its loads before waiting on any of them): 4 bytes, and 16
// bytes with both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copies the model constants (and the inertia override, if any) to shared
// memory. Every thread of the block must call it (it synchronises). All
// copies are asynchronous, so the whole model arrives in one memory round
// trip whatever the block size (a load-then-store loop would wait for each
// of a thread's loads in turn). The wait also completes the calling thread's
// own earlier cp.async copies (its staged inputs). The BodyC and BodyI
// arrays are separate device allocations (256-byte aligned) of 256- and
// 16-byte records, so their 16-byte copies are aligned on both sides.
__device__ __forceinline__ SmemModel stage_model(const ModelView& mv, float4* smem) {
  BodyC* sc = reinterpret_cast<BodyC*>(smem);
  BodyI* si = reinterpret_cast<BodyI*>(sc + mv.n);
  TopoLists* st = reinterpret_cast<TopoLists*>(si + mv.n);
  const float4* src = reinterpret_cast<const float4*>(mv.c);
  float4* dst = reinterpret_cast<float4*>(sc);
  const int nc4 = mv.n * (int)(sizeof(BodyC) / sizeof(float4));
  static_assert(sizeof(BodyI) == 16, "BodyI is copied as one 16-byte record");
  // every thread of the block, whatever its shape
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  for (int k = tid; k < nc4; k += nt) cp_async16(dst + k, src + k);
  for (int k = tid; k < mv.n; k += nt) cp_async16(si + k, mv.i + k);
  const int* ts = reinterpret_cast<const int*>(mv.topo);
  int* td = reinterpret_cast<int*>(st);
  for (int k = tid; k < (int)(sizeof(TopoLists) / sizeof(int)); k += nt) cp_async4(td + k, ts + k);
  cp_async_wait_all();
  __syncthreads();
  if (mv.theta) {  // the override replaces the staged parameters, after they have landed
    for (int k = tid; k < mv.n * 10; k += nt) cp_async4(&sc[k / 10].theta[k % 10], mv.theta + k);
    cp_async_wait_all();
    __syncthreads();
  }
  return SmemModel{sc, si, mv.n, st, mv.depth};
}

__host__ __device__ inline size_t smem_bytes(int n) {
  return (size_t)n * (sizeof(BodyC) + sizeof(BodyI)) + (sizeof(TopoLists) + 15) / 16 * 16;
}

// Dynamic shared memory of a kernel: the model, then a float tile of
// `rows` staged input rows for each of the block's environments.
__host__ __device__ inline size_t smem_bytes(int n, int rows, int block) {
  return smem_bytes(n) + (size_t)rows * block * sizeof(float);
}

__device__ __forceinline__ float* smem_tile(float4* smem, int n) {
  return reinterpret_cast<float*>(reinterpret_cast<char*>(smem) + smem_bytes(n));
}

// Rotation matrix of the quaternion (x, y, z, w), normalised first.
__device__ __forceinline__ void quat_R(float x, float y, float z, float w, float* R) {
  float s = rsqrtf(fmaf(x, x, fmaf(y, y, fmaf(z, z, w * w))));
  x *= s;
  y *= s;
  z *= s;
  w *= s;
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// One environment's column of a staged [field][envs-per-block] tile in
// shared memory: element k is p[k * ld]. Consecutive threads hold
// consecutive environments, so a warp's accesses hit 32 distinct banks.
struct Col {
  const float* p;
  int ld;
  __device__ __forceinline__ float operator[](int k) const { return p[k * ld]; }
};


// ---- SM-pinned tile loops ---------------------------------------------------
// The straight-line specialised kernels run fast only while an SM keeps
// executing the same code: their instructions then stay in the SM's
// instruction caches from one step to the next. A pinned launch gives every
// SM one role (a table indexed by the SM id): a block serves the role of the
// SM it landed on, pulling tiles of environments from that role's counter,
// and leaves when they run out; blocks on SMs without a role leave at once.
// The block that finishes last then takes every tile still left in any slot
// (a role none of whose SMs received a block), so the launch always does all
// the work. No block ever waits for another.
__device__ __forceinline__ int sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return (int)r;
}

__device__ __forceinline__ int pinned_role(const PinArgs& p) {
  const int s = sm_id();
  return s < kPinTableSize ? p.table[s] : -1;
}

// body(slot, tile) for the tiles of `my_slot` (or none if my_slot < 0), then
// the clean-up described above; slot s has n_tiles[s] tiles. One call site of
// body, so its code is emitted once. Every thread of the block (of any
// shape) must call it.
template <class F>
__device__ __forceinline__ void pinned_tiles(const PinArgs& p, int my_slot, int n_slots, const int* n_tiles, F& body) {
  __shared__ int s_tile, s_last;
  const bool lead = (threadIdx.x | threadIdx.y | threadIdx.z) == 0;
  int slot = my_slot;
  bool cleanup = false;
  for (;;) {
    if (slot >= 0) {
      if (lead) s_tile = atomicAdd(&p.counters[slot], 1);
      __syncthreads();
      const int t = s_tile;
      __syncthreads();
      if (t < n_tiles[slot]) {
        body(slot, t);
        continue;
      }
    }
    if (!cleanup) {  // own tiles done: count this block out; the last one cleans up
      if (lead)
        s_last = atomicAdd(&p.counters[kPinRegion - 1], 1) == (int)(gridDim.x * gridDim.y * gridDim.z) - 1;
      __syncthreads();
      if (!s_last) return;
      cleanup = true;
      slot = 0;
      continue;
    }
    if (++slot >= n_slots) return;
  }
}

// The same with n_tiles tiles in every slot.
template <class F>
__device__ __forceinline__ void pinned_tiles(const PinArgs& p, int my_slot, int n_slots, int n_tiles, F& body) {
  const int t[4] = {n_tiles, n_tiles, n_tiles, n_tiles};
  pinned_tiles(p, my_slot, n_slots, t, body);
}

// Stages rows [0, rows) of a [rows][B] array for this thread's environment
// into tile[row * blockDim.x + threadIdx.x]. Only the calling thread reads
// its own column afterwards, so the thread's own wait is enough.
__device__ __forceinline__ Col stage_rows(float* tile, const float* __restrict__ src, int rows, int64_t B, int64_t e) {
  float* dst = tile + threadIdx.x;
  for (int k = 0; k < rows; ++k) cp_async4(dst + k * blockDim.x, src + (int64_t)k * B + e);
  return Col{dst, (int)blockDim.x};
}

// Pose of body i in its parent from q (paper Eq. 4-5 for revolute joints).
// sin q and 1 - cos q come from one sincos of q/2: sin q = 2 s c,
// 1 - cos q = 2 s^2, which keeps 1 - cos q accurate near q = 0.
__device__ __forceinline__ Xf joint_X(const BodyC& c, const BodyI& b, const Col& q) {
  Xf X;
  if (b.type == FST_JOINT_REVOLUTE) {
    const float qi = q[b.qi];
    float sh, ch;
    sincosf(0.5f * qi, &sh, &ch);
    const float s = 2.f * sh * ch;
    const float omc = 2.f * sh * sh;
#pragma unroll
    for (int k = 0; k < 9; ++k) X.R[k] = fmaf(omc, c.Bm[k], fmaf(s, c.A[k], c.R0[k]));
#pragma unroll
    for (int k = 0; k < 3; ++k) X.t[k] = fmaf(omc, c.b[k], fmaf(s, c.a[k], c.t0[k]));
  } else if (b.type == FST_JOINT_PRISMATIC) {
    const float qi = q[b.qi];
#pragma unroll
    for (int k = 0; k < 9; ++k) X.R[k] = c.R0[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) X.t[k] = fmaf(qi, c.a[k], c.t0[k]);
  } else if (b.type == FST_JOINT_FREE) {
    const float p[3] = {q[b.qi], q[b.qi + 1], q[b.qi + 2]};
    float Rq[9];
    quat_R(q[b.qi + 3], q[b.qi + 4], q[b.qi + 5], q[b.qi + 6], Rq);
    // T_joint * (Rq, p)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc)
        X.R[3 * r + cc] = fmaf(c.R0[3 * r], Rq[cc], fmaf(c.R0[3 * r + 1], Rq[3 + cc], c.R0[3 * r + 2] * Rq[6 + cc]));
      X.t[r] = fmaf(c.R0[3 * r], p[0], fmaf(c.R0[3 * r + 1], p[1], fmaf(c.R0[3 * r + 2], p[2], c.t0[r])));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) X.R[k] = c.R0[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) X.t[k] = c.t0[k];
  }
  return X;
}

__device__ __forceinline__ SV S_of(const BodyC& c) { return SV{f3{c.S[0], c.S[1], c.S[2]}, f3{c.S[3], c.S[4], c.S[5]}}; }

// S_i x_i for a joint-space column x; the free joint maps its velocity
// coordinates [v; w] to spatial (w, v).
__device__ __forceinline__ SV S_times(const BodyC& c, const BodyI& b, const Col& x) {
  if (b.type == FST_JOINT_REVOLUTE || b.type == FST_JOINT_PRISMATIC) return x[b.vi] * S_of(c);
  if (b.type == FST_JOINT_FREE)
    return SV{f3{x[b.vi + 3], x[b.vi + 4], x[b.vi + 5]}, f3{x[b.vi], x[b.vi + 1], x[b.vi + 2]}};
  return sv_zero();
}

// out_i = S_i^T f
__device__ __forceinline__ void ST_store(const BodyC& c, const BodyI& b, SV f, float* __restrict__ out, int64_t B,
                                         int64_t e) {
  if (b.type == FST_JOINT_REVOLUTE || b.type == FST_JOINT_PRISMATIC) {
    out[(int64_t)b.vi * B + e] = dot(S_of(c), f);
  } else if (b.type == FST_JOINT_FREE) {
    float* p = out + (int64_t)b.vi * B + e;
    p[0] = f.v.x;
    p[B] = f.v.y;
    p[2 * B] = f.v.z;
    p[3 * B] = f.w.x;
    p[4 * B] = f.w.y;
    p[5 * B] = f.w.z;
  }
}

__device__ __forceinline__ int nv_of(int type) {
  return type == FST_JOINT_FREE ? 6 : (type == FST_JOINT_FIXED ? 0 : 1);
}

}  // namespace fst
