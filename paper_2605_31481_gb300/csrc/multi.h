// Persistent multi-tree launch (multi.cu): per-call arguments.
#pragma once

#include "fst_internal.h"

namespace fst {

constexpr int kMaxMulti = FST_MAX_MULTI;

struct MultiIO {
  const float* q;
  const float* qd;
  const float* qdd;
  const float* tau;
  float* poses;
  float* tau_out;
  float* M;
  float* qdd_out;
  int64_t B;
};

// Work items: segment s covers items [seg_start[s], seg_start[s+1]), one
// tile of environments each, of operator seg_op[s] (a Role) on tree
// seg_model[s].
struct MultiArgs {
  ModelView mv[kMaxMulti];
  MultiIO io[kMaxMulti];
  int seg_start[4 * kMaxMulti + 1];
  unsigned char seg_model[4 * kMaxMulti];
  unsigned char seg_op[4 * kMaxMulti];
  int n_items;
  int max_rows;          // staged input rows of the widest item
  int maxw[kMaxMulti];   // level form: bodies of each tree's widest level (the lean ABA's ring)
  size_t model_bytes;    // shared memory reserved for the largest tree
  int* counter;          // device work counter (reset before each launch)
};

// Environments per item: `block` for the generic kernel (one environment per
// thread), 32 for the level-parallel one.
cudaError_t launch_multi(const MultiArgs& a, int max_n, int block, cudaStream_t s);
// The level-parallel form: items of 32 environments, the block's warps
// splitting each tree level; state_bytes of per-body state per block.
cudaError_t launch_multi_level(const MultiArgs& a, size_t state_bytes, int block, cudaStream_t s);

}  // namespace fst

struct fst_multi {
  std::vector<const fst_model*> models;
  int* counter = nullptr;
  int device = -1;
  int block = 64;
  int variant = FST_VARIANT_GENERIC;  // or FST_VARIANT_LEVEL
};
