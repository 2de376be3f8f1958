// Internal layout shared by the host model builder and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fst.h"
#include "fst_layout.h"

namespace fst {
struct JitState;
}

struct fst_model {
  int n = 0, nq = 0, nv = 0, depth = 0;
  int max_width = 0;                 // bodies of the widest tree level
  int device = -1;
  bool has_free = false;
  double gravity[3] = {0, 0, 0};
  std::vector<fst::BodyC> hc;
  std::vector<fst::BodyI> hi;
  std::vector<uint64_t> ancestors;   // bit j set: body j is on body i's support path (incl. i)
  std::vector<int> level;            // 1-based depth of each body
  fst::BodyC* dc = nullptr;
  fst::BodyI* di = nullptr;
  fst::TopoLists ht{};               // level and child lists (host copy)
  fst::TopoLists* dt = nullptr;      // device copy
  int* dpin = nullptr;               // SM-pinned launches: role table, then the counter regions
  int pin_table[256] = {};           // host copy of the role table (FST_ROLE_*, -1 none)
  std::vector<int> sm_ids;           // the device's SM ids (probed when the role table is set)
  fst::JitState* jit = nullptr;      // run-time specialised kernels, if any
  int block[16] = {0};               // threads per block per kernel kind (0 = built-in heuristic)
  int variant[16] = {0};             // per kind: 0 auto, 1 generic, 2 specialised (see fst_model_set_launch)
};

namespace fst {
// Host-side helpers (model.cpp / api.cpp).
fst_status set_error(fst_status s, const std::string& msg);
// Checks shared by every compute entry point: a model, 0 <= B <= 2^31 - 1
// and the model's device current. FST_OK when the call may go on; *skip is
// set when B == 0 (nothing to launch).
fst_status check_call(const char* fn, const fst_model* m, int64_t B, bool* skip);
// Ids (%smid) of the current device's SMs, sorted (probe.cu; synchronous).
cudaError_t sm_ids(std::vector<int>& ids);
fst_status build_model_host(const fst_body_desc* bodies, int32_t n, const double gravity[3],
                            fst_model* m);
inline ModelView view_of(const fst_model* m, const float* theta) {
  ModelView v;
  v.c = m->dc;
  v.i = m->di;
  v.topo = m->dt;
  v.theta = theta;
  v.n = m->n;
  v.nq = m->nq;
  v.nv = m->nv;
  v.depth = m->depth;
  for (int k = 0; k < 3; ++k) v.a0[k] = (float)(-m->gravity[k]);
  return v;
}
}  // namespace fst
