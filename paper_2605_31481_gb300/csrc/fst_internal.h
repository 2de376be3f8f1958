// Internal layout shared by the host model builder and the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fst.h"

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
  float pad[10];
};
static_assert(sizeof(BodyC) == 256, "BodyC must stay 256 bytes");

struct BodyI {
  int32_t parent;
  int32_t type;
  int32_t qi;
  int32_t vi;
};

// Everything a kernel needs to find the model; passed by value.
struct ModelView {
  const BodyC* c;        // device, n entries
  const BodyI* i;        // device, n entries
  const float* theta;    // device [n][10] override, or nullptr
  int n, nq, nv, depth;
  float a0[3];           // linear part of the world's spatial acceleration: -gravity
};

}  // namespace fst

struct fst_model {
  int n = 0, nq = 0, nv = 0, depth = 0;
  int device = -1;
  bool has_free = false;
  double gravity[3] = {0, 0, 0};
  std::vector<fst::BodyC> hc;
  std::vector<fst::BodyI> hi;
  std::vector<uint64_t> ancestors;   // bit j set: body j is on body i's support path (incl. i)
  std::vector<int> level;            // 1-based depth of each body
  fst::BodyC* dc = nullptr;
  fst::BodyI* di = nullptr;
};

namespace fst {
// Host-side helpers (model.cpp / api.cpp).
fst_status set_error(fst_status s, const std::string& msg);
fst_status build_model_host(const fst_body_desc* bodies, int32_t n, const double gravity[3],
                            fst_model* m);
inline ModelView view_of(const fst_model* m, const float* theta) {
  ModelView v;
  v.c = m->dc;
  v.i = m->di;
  v.theta = theta;
  v.n = m->n;
  v.nq = m->nq;
  v.nv = m->nv;
  v.depth = m->depth;
  for (int k = 0; k < 3; ++k) v.a0[k] = (float)(-m->gravity[k]);
  return v;
}
}  // namespace fst
