// Device-safe layout shared by the host model builder, the kernels and the
// run-time specialised (NVRTC) kernels: no host-only headers here.
#pragma once

#ifdef __CUDACC_RTC__
typedef long long int64_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef unsigned long size_t;
#define FST_MAX_BODIES 64
#define FST_MAX_LINKS 16
enum { FST_JOINT_FIXED = 0, FST_JOINT_REVOLUTE = 1, FST_JOINT_PRISMATIC = 2, FST_JOINT_FREE = 3 };
#else
#include <cstdint>

#include "../../include/fst.h"
#endif

namespace fst {

// Per-body FP32 constants, 64 floats (256 B) so a body is 16 float4 loads.
// Revolute (paper Eq. 2-3, all in the parent frame):
//   R_pc = R0 + sin(q) A + (1 - cos q) Bm,  t_pc = t0 + sin(q) a + (1 - cos q) b
// Prismatic: R_pc = R0, t_pc = t0 + q a.   Fixed: R_pc = R0, t_pc = t0.
// Free (body 0 only): R0 = R of T_joint, t0 = t of T_joint; the joint's own
//   pose comes from q.
// S: motion subspace of a 1-DOF joint in body coordinates, [w; v].
// theta: 10 inertial parameters about the body origin [m, h(3), I(6)].
// anc: support-path bitmask (drives the zero blocks of J and M).
struct BodyC {
  float R0[9];
  float A[9];
  float Bm[9];
  float t0[3];
  float a[3];
  float b[3];
  float S[6];
  float theta[10];
  unsigned long long anc;  // bit j set: body j is on this body's support path (itself included)
  int32_t lpos;            // position of the body within its tree level (level_body order)
  float pad[9];
};
static_assert(sizeof(BodyC) == 256, "BodyC must stay 256 bytes");

struct BodyI {
  int32_t parent;
  int32_t type;
  int32_t qi;
  int32_t vi;
};

// Level and child lists of the tree (ints), used by the level-parallel
// kernels: bodies of level l (root = level 0) are
// level_body[level_start[l] .. level_start[l+1]), children of body i are
// child[child_start[i] .. child_start[i+1]). Laid out in one int array:
//   level_start (FST_MAX_BODIES + 1) | level_body (FST_MAX_BODIES) |
//   child_start (FST_MAX_BODIES + 1) | child (FST_MAX_BODIES)
struct TopoLists {
  int level_start[FST_MAX_BODIES + 1];
  int level_body[FST_MAX_BODIES];
  int child_start[FST_MAX_BODIES + 1];
  int child[FST_MAX_BODIES];
};

// Everything a kernel needs to find the model; passed by value.
struct ModelView {
  const BodyC* c;        // device, n entries
  const BodyI* i;        // device, n entries
  const TopoLists* topo; // device
  const float* theta;    // device [n][10] override, or nullptr
  int n, nq, nv, depth;
  float a0[3];           // linear part of the world's spatial acceleration: -gravity
};

struct LinkList {
  int n;
  int idx[FST_MAX_LINKS];
};

// Packed Jacobian layout of fst_eval: link l keeps only the columns of the
// DOFs on its support path, in DOF order, as a [6][cols[l]] block starting
// at row off[l] of a [rows][B] array.
struct PackedJ {
  int cols[FST_MAX_LINKS];
  int off[FST_MAX_LINKS];
};

// Floats of level-parallel state per body and environment (level.cuh):
// FK X 12; RNEA X 12 | v 6 | a 6 | f 6; CRBA X 12 | Ic 10 | contribution 10;
// ABA X 12 | va 6 | c 6 | IA 21 | pA 6 | U 6 | invD | u.
constexpr int kFkStateFloats = 12;
constexpr int kRneaStateFloats = 30;
constexpr int kCrbaStateFloats = 32;
constexpr int kAbaStateFloats = 59;
// The lean level-parallel ABA (FST_VARIANT_LEVEL_LEAN): per body VU 6 (v,
// then U, then a) | c 6 | invD | u; per level parity and position within the
// level, the contribution to the parent: X^T I^a X 21 | X^T p^a 6.
constexpr int kAbaLeanBodyFloats = 14;
constexpr int kAbaLeanRingFloats = 27;
// The lean level-parallel CRBA: per body X 12 | F = Ic S 6; per ring slot
// the composite-inertia contribution to the parent (10).
constexpr int kCrbaLeanBodyFloats = 18;
constexpr int kCrbaLeanRingFloats = 10;

// Operators of the fused evaluation kernel, in launch order (longest first,
// so the slowest role's blocks are dispatched first).
enum Role { ROLE_ABA = 0, ROLE_CRBA = 1, ROLE_RNEA = 2, ROLE_KIN = 3 };

// SM-pinned launches: the role each SM id serves (ROLE_*, -1 none), and the
// per-launch tile counters (slots 0..6, then the count of finished blocks).
// Two counter regions: one for the fused evaluation, one for ABA, so the two
// can run side by side.
constexpr int kPinTableSize = 256;
constexpr int kPinRegion = 8;
constexpr int kPinEvalRegion = 0;
constexpr int kPinAbaRegion = 1;
struct PinArgs {
  const int* table;  // [kPinTableSize]
  int* counters;     // [kPinRegion] of this launch
  // the fused pinned step (eval): per slot of EvalArgs::roles, the number of
  // tiles and the environments per tile (a multiple of 32; ABA's tiles are
  // 64 environments, two level-parallel tiles of 32)
  int tiles[4];
  int envs[4];
};

struct EvalArgs {
  const float* q;
  const float* qd;
  const float* qdd;
  const float* tau;
  float* poses;
  float* J;
  float* tau_out;
  float* M;
  float* qdd_out;
  LinkList links;
  int roles[4];
  int n_roles;
  int level_mask;  // bit r: role r runs level-parallel (32 environments per block)
  // RNEA role extras (EVAL_* bits in rnea_flags): the kinematics from the
  // RNEA sweep's own joint transforms, and the RNEA adjoint for tau_bar
  const float* tau_bar;
  float* qbar;
  float* qdbar;
  float* qddbar;
  int rnea_flags;
  int packed;   // M as its upper triangle and J as PackedJ (the KIN, RNEA and CRBA roles)
  PackedJ pj;
};

// rnea_flags of EvalArgs
enum {
  EVAL_KIN_IN_RNEA = 1,  // the RNEA role writes poses and J (no separate kinematics role)
  EVAL_RNEA_VJP = 2,     // the RNEA role runs the adjoint sweeps for tau_bar
  EVAL_TBAR_IS_TAU = 4   // ... with tau_bar = the tau it computed (tau_bar not read)
};

}  // namespace fst
