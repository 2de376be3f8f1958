// C ABI of libfst.so: argument validation, device checks, launches.
#include <cuda_runtime.h>

#include <atomic>
#include <climits>
#include <cstring>
#include <initializer_list>
#include <new>
#include <sstream>
#include <string>
#include <utility>

#include "fst_internal.h"
#include "jit.h"
#include "launch.h"
#include "multi.h"

namespace fst {

namespace {
thread_local std::string g_last_error;
std::atomic<int> g_carveout{-1};
std::atomic<int> g_carveout_gen{0};
}  // namespace

int carveout_override() { return g_carveout.load(); }
int carveout_generation() { return g_carveout_gen.load(); }

fst_status set_error(fst_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

// Common checks of every compute call. Returns FST_OK when the call may
// launch; *skip is set when B == 0.
fst_status check_call(const char* fn, const fst_model* m, int64_t B, bool* skip) {
  *skip = false;
  if (!m) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null model");
  if (B < 0) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": B must be >= 0");
  if (B == 0) {
    *skip = true;
    return FST_OK;
  }
  // grids are sized B / (environments per block) and must stay within the
  // 2^31 - 1 limit of gridDim.x for every launch form (at least 4
  // environments per block)
  if (B > (int64_t)INT32_MAX)
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": B must be at most 2^31 - 1 per call");
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) {
    std::ostringstream os;
    os << fn << ": " << cudaGetErrorName(err) << ": " << cudaGetErrorString(err);
    return set_error(FST_ERR_CUDA, os.str());
  }
  if (dev != m->device) {
    std::ostringstream os;
    os << fn << ": current device " << dev << " is not the model's device " << m->device;
    return set_error(FST_ERR_INVALID_ARG, os.str());
  }
  return FST_OK;
}

namespace {

fst_status cuda_error(const char* where, cudaError_t err) {
  std::ostringstream os;
  os << where << ": " << cudaGetErrorName(err) << ": " << cudaGetErrorString(err);
  return set_error(FST_ERR_CUDA, os.str());
}

fst_status need(const char* fn, const void* p, const char* name) {
  if (p) return FST_OK;
  return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null " + name);
}

// Whether a call of this kind runs the specialised kernel: it must exist,
// and the kind must not be pinned to another variant.
bool use_jit(const fst_model* m, int kind) {
  const int v = m->variant[kind];
  return (v == FST_VARIANT_AUTO || v == FST_VARIANT_SPECIALIZED) && jit_has(m, kind);
}

// Whether a call of this kind runs the level-parallel kernel: selected, and
// its shared memory (which grows with the number of bodies) fits.
// Tiles of 32 environments per block of a level-parallel launch of this kind.
int level_tiles(const fst_model* m, int kind) { return m->variant[kind] == FST_VARIANT_LEVEL2 ? 2 : 1; }

bool use_level(const fst_model* m, int kind, int level_kind) {
  const int v = m->variant[kind];
  return (v == FST_VARIANT_LEVEL || v == FST_VARIANT_LEVEL2) &&
         level_smem_needed(view_of(m, nullptr), level_kind, level_tiles(m, kind)) <= kLevelSmemLimit;
}

// The path-parallel kernel slot a call of this kind runs (0: none): 1 for
// FST_VARIANT_PATH (a lane per path), 2 for FST_VARIANT_PATH_WARP (a warp
// per path).
int path_slot(const fst_model* m, int kind) {
  const int v = m->variant[kind];
  const int slot = v == FST_VARIANT_PATH ? 1 : v == FST_VARIANT_PATH_WARP ? 2 : 0;
  return slot && jit_has_slot(m, kind, slot) ? slot : 0;
}
bool use_path(const fst_model* m, int kind) { return path_slot(m, kind) != 0; }

// Launches a path-parallel kernel with `rows` staged input rows per
// environment and gy = blockIdx.y extent. A lane per path: G lanes per
// environment, so a block of T threads serves (T / 32) * (32 / G)
// environments. A warp per path: blocks of 32 environments and one warp per
// path, plus two merge buffers of 27 floats per warp and lane.
template <typename... A>
cudaError_t path_go(const fst_model* m, int kind, int64_t B, int rows, unsigned gy, cudaStream_t s, A... args) {
  void* argv[] = {(void*)&args...};
  const int slot = path_slot(m, kind);
  if (slot == 2) {
    const int np = jit_path_count(m);
    const size_t sh = ((size_t)rows * 32 + (size_t)2 * np * 27 * 32) * sizeof(float);
    return jit_launch_slot(m, kind, 2, dim3((unsigned)((B + 31) / 32), gy), 32 * np, sh, s, argv);
  }
  const int T = m->block[kind] ? m->block[kind] : 128;
  const int G = jit_path_lanes(m);
  const int EPB = (T / 32) * (32 / G);
  const dim3 grid((unsigned)((B + EPB - 1) / EPB), gy);
  return jit_launch_slot(m, kind, 1, grid, T, (size_t)rows * EPB * sizeof(float), s, argv);
}

// Threads per block of a level-parallel launch: a multiple of 32 (one warp
// per share of a level), 32 environments per block.
int level_block(const fst_model* m, int kind) {
  if (m->block[kind]) return m->block[kind];
  return m->variant[kind] == FST_VARIANT_LEVEL2 ? 256 : 128;
}

int block_of(const fst_model* m, int kind, int64_t B) { return m->block[kind] ? m->block[kind] : default_block(B); }

Launch launch_of(const fst_model* m, int kind, int64_t B, void* stream) {
  return Launch{block_of(m, kind, B), (cudaStream_t)stream};
}

// Zeroes the outputs of a call with nothing to compute (B = 0 or no degrees
// of freedom); null pointers and empty sizes are skipped.
cudaError_t zero_outputs(cudaStream_t s, std::initializer_list<std::pair<void*, size_t>> outs) {
  for (const auto& o : outs)
    if (o.first && o.second) {
      const cudaError_t err = cudaMemsetAsync(o.first, 0, o.second, s);
      if (err != cudaSuccess) return err;
    }
  return cudaSuccess;
}

fst_status finish(const char* fn, cudaError_t err) {
  if (err != cudaSuccess) return cuda_error(fn, err);
  return FST_OK;
}

// Launches a specialised kernel: one environment per thread, `rows` staged
// input rows per environment plus `P` floats per warp of reduction slots in
// shared memory; gy = blockIdx.y extent. *nblk receives the grid's x size.
template <typename... A>
cudaError_t jit_go_slot(const fst_model* m, int kind, int slot, int64_t B, int rows, int P, unsigned gy,
                        cudaStream_t s, unsigned* nblk, A... args) {
  int T = block_of(m, kind, B);
  auto smem = [&](int t) { return (size_t)rows * t * sizeof(float) + (size_t)(t / 32) * P * sizeof(float); };
  while (T > 32 && smem(T) > 96 * 1024) T /= 2;
  const dim3 grid(grid_for(B, T), gy);
  if (nblk) *nblk = grid.x;
  void* argv[] = {(void*)&args...};
  return jit_launch_slot(m, kind, slot, grid, T, smem(T), s, argv);
}

template <typename... A>
cudaError_t jit_go(const fst_model* m, int kind, int64_t B, int rows, int P, unsigned gy, cudaStream_t s,
                   unsigned* nblk, A... args) {
  return jit_go_slot(m, kind, 0, B, rows, P, gy, s, nblk, args...);
}

}  // namespace
}  // namespace fst

using namespace fst;

#define FST_CHECK(expr)                   \
  do {                                    \
    fst_status _s = (expr);               \
    if (_s != FST_OK) return _s;          \
  } while (0)

extern "C" {

const char* fst_last_error(void) { return g_last_error.c_str(); }

const char* fst_version(void) { return "fst 0.1 (sm_103a)"; }

fst_status fst_model_create(const fst_body_desc* bodies, int32_t n_bodies, const double gravity[3],
                            fst_model** out) {
  if (!out) return set_error(FST_ERR_INVALID_ARG, "fst_model_create: null out");
  *out = nullptr;
  fst_model* m = new (std::nothrow) fst_model();
  if (!m) return set_error(FST_ERR_NO_MEMORY, "fst_model_create: host allocation failed");
  fst_status s = build_model_host(bodies, n_bodies, gravity, m);
  if (s != FST_OK) {
    delete m;
    return s;
  }
  cudaError_t err = cudaGetDevice(&m->device);
  if (err == cudaSuccess) err = cudaMalloc((void**)&m->dc, sizeof(BodyC) * m->n);
  if (err == cudaSuccess) err = cudaMalloc((void**)&m->di, sizeof(BodyI) * m->n);
  if (err == cudaSuccess) err = cudaMemcpy(m->dc, m->hc.data(), sizeof(BodyC) * m->n, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(m->di, m->hi.data(), sizeof(BodyI) * m->n, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMalloc((void**)&m->dt, sizeof(TopoLists));
  if (err == cudaSuccess) err = cudaMemcpy(m->dt, &m->ht, sizeof(TopoLists), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMalloc((void**)&m->dpin, sizeof(int) * (kPinTableSize + 2 * kPinRegion));
  if (err == cudaSuccess) err = cudaMemset(m->dpin, 0xff, sizeof(int) * kPinTableSize);  // no roles: -1
  for (int i = 0; i < kPinTableSize; ++i) m->pin_table[i] = FST_ROLE_NONE;
  if (err != cudaSuccess) {
    fst_status st = (err == cudaErrorMemoryAllocation) ? set_error(FST_ERR_NO_MEMORY, "fst_model_create: cudaMalloc failed")
                                                       : cuda_error("fst_model_create", err);
    if (m->dc) cudaFree(m->dc);
    if (m->di) cudaFree(m->di);
    if (m->dt) cudaFree(m->dt);
    if (m->dpin) cudaFree(m->dpin);
    delete m;
    return st;
  }
  *out = m;
  return FST_OK;
}

fst_status fst_model_destroy(fst_model* m) {
  if (!m) return FST_OK;
  jit_release(m);
  if (m->dc) cudaFree(m->dc);
  if (m->di) cudaFree(m->di);
  if (m->dt) cudaFree(m->dt);
  if (m->dpin) cudaFree(m->dpin);
  delete m;
  return FST_OK;
}

fst_status fst_set_smem_carveout(int32_t percent) {
  if (percent < -1 || percent > 100)
    return set_error(FST_ERR_INVALID_ARG, "fst_set_smem_carveout: percent must be in [-1, 100]");
  g_carveout.store(percent);
  g_carveout_gen.fetch_add(1);
  return FST_OK;
}

fst_status fst_model_specialize(fst_model* m, uint32_t kinds) {
  if (!m) return set_error(FST_ERR_INVALID_ARG, "fst_model_specialize: null model");
  if (kinds == 0) kinds = FST_SPEC_ALL;
  if (kinds & ~(uint32_t)FST_SPEC_ALL) return set_error(FST_ERR_INVALID_ARG, "fst_model_specialize: unknown kind bits");
  return jit_specialize(m, kinds);
}

fst_status fst_model_set_launch(fst_model* m, uint32_t kinds, int32_t block, int32_t variant) {
  if (!m) return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: null model");
  if (block != 0 && block != 32 && block != 64 && block != 128 && block != 256)
    return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: block must be 0, 32, 64, 128 or 256");
  if (variant < FST_VARIANT_AUTO || variant > FST_VARIANT_LEVEL_LEAN)
    return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: unknown variant");
  if (variant == FST_VARIANT_LEVEL2 && block == 32)
    return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: the two-tile level variant needs block >= 64");
  // "all kinds" with the level or path variant means every kind that has one
  if (kinds == 0)
    kinds = (variant == FST_VARIANT_LEVEL || variant == FST_VARIANT_LEVEL2 || variant == FST_VARIANT_PATH ||
             variant == FST_VARIANT_PATH_WARP)
                ? (1u << (JK_EVAL + 1)) - 1u
                : variant == FST_VARIANT_PINNED ? (1u << JK_EVAL) | (1u << JK_ABA)
                : variant == FST_VARIANT_LEVEL_LEAN ? (1u << JK_ABA) | (1u << JK_CRBA)
                                                    : FST_SPEC_ALL;
  if (kinds & ~(uint32_t)FST_SPEC_ALL) return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: unknown kind bits");
  for (int k = 0; k < JK_COUNT; ++k) {
    if (((kinds >> k) & 1u) && variant == FST_VARIANT_MIXED && k != JK_EVAL)
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: the mixed variant is for eval only");
    if (((kinds >> k) & 1u) && variant == FST_VARIANT_SPECIALIZED && !jit_has(m, k))
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: a selected kind is not specialised yet");
    if (((kinds >> k) & 1u) && variant == FST_VARIANT_MIXED && !jit_has(m, JK_EVAL_MIXED))
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: a selected kind is not specialised yet");
    if (((kinds >> k) & 1u) && (variant == FST_VARIANT_PATH || variant == FST_VARIANT_PATH_WARP) &&
        !jit_has_slot(m, k, variant == FST_VARIANT_PATH ? 1 : 2))
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: no path-parallel kernel for a selected kind "
                                            "(specialise FK, Jacobian, RNEA, CRBA, ABA or eval first; trees with "
                                            "more than 8 leaves have none)");
    if (((kinds >> k) & 1u) && variant == FST_VARIANT_LEVEL_LEAN && k != JK_ABA && k != JK_CRBA)
      return set_error(FST_ERR_INVALID_ARG,
                       "fst_model_set_launch: the lean level-parallel variant is for CRBA and ABA only");
    if (((kinds >> k) & 1u) && variant == FST_VARIANT_PINNED && k != JK_EVAL && k != JK_ABA)
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: the pinned variant is for eval and ABA only");
    if (((kinds >> k) & 1u) && variant == FST_VARIANT_PINNED && k == JK_EVAL && !jit_has_slot(m, JK_EVAL, 3))
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: pinned eval needs the specialised eval kernel");
    if (((kinds >> k) & 1u) && variant == FST_VARIANT_PINNED && k == JK_EVAL &&
        (size_t)2 * (m->nq + 2 * m->nv + kAbaStateFloats * m->n) * 32 * sizeof(float) +
                (size_t)m->n * (sizeof(BodyC) + sizeof(BodyI)) + sizeof(TopoLists) + 16 >
            kLevelSmemLimit)
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: the tree is too large for the pinned step "
                                            "(two level-parallel ABA tiles do not fit in shared memory)");
    if (((kinds >> k) & 1u) && variant == FST_VARIANT_PINNED && k == JK_ABA &&
        level_smem_needed(view_of(m, nullptr), LEVEL_ABA) > kLevelSmemLimit)
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: the tree is too large for pinned ABA");
    if (((kinds >> k) & 1u) && (variant == FST_VARIANT_LEVEL || variant == FST_VARIANT_LEVEL2) && k > JK_EVAL)
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_launch: the level-parallel variant exists for FK, "
                                            "Jacobian, RNEA, CRBA, ABA and eval only");
  }
  for (int k = 0; k < JK_COUNT; ++k)
    if ((kinds >> k) & 1u) {
      m->block[k] = block;
      m->variant[k] = variant;
    }
  return FST_OK;
}

fst_status fst_model_set_sm_roles(fst_model* m, const int32_t* role_of_sm, int32_t n) {
  if (!m || (!role_of_sm && n)) return set_error(FST_ERR_INVALID_ARG, "fst_model_set_sm_roles: null argument");
  if (n < 0 || n > kPinTableSize)
    return set_error(FST_ERR_INVALID_ARG, "fst_model_set_sm_roles: n must be in [0, 256]");
  int table[kPinTableSize];
  for (int i = 0; i < kPinTableSize; ++i) {
    const int r = i < n ? role_of_sm[i] : FST_ROLE_NONE;
    if (r < FST_ROLE_NONE || r > FST_ROLE_KIN)
      return set_error(FST_ERR_INVALID_ARG, "fst_model_set_sm_roles: unknown role");
    table[i] = r;
  }
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess && dev != m->device)
    return set_error(FST_ERR_INVALID_ARG, "fst_model_set_sm_roles: the current device is not the model's device");
  if (err == cudaSuccess) err = cudaMemcpy(m->dpin, table, sizeof(table), cudaMemcpyHostToDevice);
  if (err == cudaSuccess)
    for (int i = 0; i < kPinTableSize; ++i) m->pin_table[i] = table[i];
  // the SM ids that exist, for the pinned step's tiles per role (once)
  if (err == cudaSuccess && m->sm_ids.empty()) err = sm_ids(m->sm_ids);
  return err == cudaSuccess ? FST_OK : cuda_error("fst_model_set_sm_roles", err);
}

fst_status fst_model_specialized(const fst_model* m, uint32_t* kinds) {
  if (!m || !kinds) return set_error(FST_ERR_INVALID_ARG, "fst_model_specialized: null argument");
  *kinds = jit_mask(m);
  return FST_OK;
}

fst_status fst_model_theta(const fst_model* m, float* theta) {
  if (!m || !theta) return set_error(FST_ERR_INVALID_ARG, "fst_model_theta: null argument");
  for (int i = 0; i < m->n; ++i)
    for (int k = 0; k < 10; ++k) theta[10 * i + k] = m->hc[i].theta[k];
  return FST_OK;
}

fst_status fst_model_info(const fst_model* m, int32_t* nq, int32_t* nv, int32_t* n_bodies, int32_t* depth) {
  if (!m) return set_error(FST_ERR_INVALID_ARG, "fst_model_info: null model");
  if (nq) *nq = m->nq;
  if (nv) *nv = m->nv;
  if (n_bodies) *n_bodies = m->n;
  if (depth) *depth = m->depth;
  return FST_OK;
}

fst_status fst_fk(const fst_model* m, int64_t B, const float* q, float* poses, void* stream) {
  static const char* fn = "fst_fk";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip) return FST_OK;
  if (m->nq) FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, poses, "poses"));
  const ModelView mv = view_of(m, nullptr);
  if (use_level(m, JK_FK, LEVEL_FK))
    return finish(fn, launch_fk_level(mv, B, q, poses, level_block(m, JK_FK), level_tiles(m, JK_FK),
                        (cudaStream_t)stream));
  if (use_path(m, JK_FK))
    return finish(fn, path_go(m, JK_FK, B, m->nq, 1, (cudaStream_t)stream, mv, B, q, poses));
  if (use_jit(m, JK_FK))
    return finish(fn, jit_go(m, JK_FK, B, m->nq, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q, poses));
  return finish(fn, launch_fk(mv, B, q, poses, launch_of(m, JK_FK, B, stream)));
}

fst_status fst_jacobian(const fst_model* m, int64_t B, const float* q, const int32_t* links, int32_t n_links,
                        float* J, void* stream) {
  static const char* fn = "fst_jacobian";
  if (!links && n_links) return set_error(FST_ERR_INVALID_ARG, "fst_jacobian: null links");
  if (n_links < 1 || n_links > FST_MAX_LINKS)
    return set_error(FST_ERR_INVALID_ARG, "fst_jacobian: n_links must be in [1, FST_MAX_LINKS]");
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  LinkList L{};
  L.n = n_links;
  for (int l = 0; l < n_links; ++l) {
    if (links[l] < 0 || links[l] >= m->n) return set_error(FST_ERR_INVALID_ARG, "fst_jacobian: link index out of range");
    L.idx[l] = links[l];
  }
  if (skip || m->nv == 0) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, J, "J"));
  const ModelView mv = view_of(m, nullptr);
  if (use_level(m, JK_JACOBIAN, LEVEL_JAC))
    return finish(fn, launch_jac_level(mv, B, q, L, J, level_block(m, JK_JACOBIAN), level_tiles(m, JK_JACOBIAN),
                        (cudaStream_t)stream));
  if (use_path(m, JK_JACOBIAN))
    return finish(fn, path_go(m, JK_JACOBIAN, B, m->nq, 1, (cudaStream_t)stream, mv, B, q, L, J));
  if (use_jit(m, JK_JACOBIAN))
    return finish(fn, jit_go(m, JK_JACOBIAN, B, m->nq, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q, L, J));
  return finish(fn, launch_jacobian(mv, B, q, L, J, launch_of(m, JK_JACOBIAN, B, stream)));
}

fst_status fst_rnea(const fst_model* m, int64_t B, const float* q, const float* qd, const float* qdd,
                    const float* theta, float* tau, void* stream) {
  static const char* fn = "fst_rnea";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip || m->nv == 0) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, qdd, "qdd"));
  FST_CHECK(need(fn, tau, "tau"));
  const ModelView mv = view_of(m, theta);
  if (use_level(m, JK_RNEA, LEVEL_RNEA))
    return finish(fn, launch_rnea_level(mv, B, q, qd, qdd, tau, level_block(m, JK_RNEA), level_tiles(m, JK_RNEA),
                        (cudaStream_t)stream));
  if (use_path(m, JK_RNEA))
    return finish(fn, path_go(m, JK_RNEA, B, m->nq + 2 * m->nv, 1, (cudaStream_t)stream, mv, B, q, qd, qdd, tau));
  if (use_jit(m, JK_RNEA))
    return finish(fn, jit_go(m, JK_RNEA, B, m->nq + 2 * m->nv, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q, qd,
                             qdd, tau));
  return finish(fn, launch_rnea(mv, B, q, qd, qdd, tau, launch_of(m, JK_RNEA, B, stream)));
}

fst_status fst_crba(const fst_model* m, int64_t B, const float* q, const float* theta, float* M, void* stream) {
  static const char* fn = "fst_crba";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip || m->nv == 0) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, M, "M"));
  const ModelView mv = view_of(m, theta);
  if (use_level(m, JK_CRBA, LEVEL_CRBA))
    return finish(fn, launch_crba_level(mv, B, q, M, level_block(m, JK_CRBA), level_tiles(m, JK_CRBA),
                        (cudaStream_t)stream));
  if (m->variant[JK_CRBA] == FST_VARIANT_LEVEL_LEAN && crba_lean_smem_needed(mv, m->max_width) <= kLevelSmemLimit)
    return finish(fn, launch_crba_level_lean(mv, B, q, M, level_block(m, JK_CRBA), m->max_width,
                                             (cudaStream_t)stream));
  if (use_path(m, JK_CRBA))
    return finish(fn, path_go(m, JK_CRBA, B, m->nq, 1, (cudaStream_t)stream, mv, B, q, M));
  if (use_jit(m, JK_CRBA))
    return finish(fn, jit_go(m, JK_CRBA, B, m->nq, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q, M));
  return finish(fn, launch_crba(mv, B, q, M, launch_of(m, JK_CRBA, B, stream)));
}

fst_status fst_aba(const fst_model* m, int64_t B, const float* q, const float* qd, const float* tau,
                   const float* theta, float* qdd, void* stream) {
  static const char* fn = "fst_aba";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip || m->nv == 0) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, tau, "tau"));
  FST_CHECK(need(fn, qdd, "qdd"));
  const ModelView mv = view_of(m, theta);
  if (use_level(m, JK_ABA, LEVEL_ABA))
    return finish(fn, launch_aba_level(mv, B, q, qd, tau, qdd, level_block(m, JK_ABA), level_tiles(m, JK_ABA),
                        (cudaStream_t)stream));
  if (m->variant[JK_ABA] == FST_VARIANT_LEVEL_LEAN && aba_lean_smem_needed(mv, m->max_width) <= kLevelSmemLimit)
    return finish(fn, launch_aba_level_lean(mv, B, q, qd, tau, qdd, level_block(m, JK_ABA), m->max_width,
                                            (cudaStream_t)stream));
  if (m->variant[JK_ABA] == FST_VARIANT_PINNED) {
    int* counters = m->dpin + kPinTableSize + kPinAbaRegion * kPinRegion;
    cudaError_t err = cudaMemsetAsync(counters, 0, sizeof(int) * kPinRegion, (cudaStream_t)stream);
    if (err == cudaSuccess)
      err = launch_aba_level_pinned(mv, B, q, qd, tau, qdd, m->block[JK_ABA] ? m->block[JK_ABA] : 256,
                                    PinArgs{m->dpin, counters}, (cudaStream_t)stream);
    return finish(fn, err);
  }
  if (use_path(m, JK_ABA))
    return finish(fn, path_go(m, JK_ABA, B, m->nq + 2 * m->nv, 1, (cudaStream_t)stream, mv, B, q, qd, tau, qdd));
  if (use_jit(m, JK_ABA))
    return finish(fn, jit_go(m, JK_ABA, B, m->nq + 2 * m->nv, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q, qd,
                             tau, qdd));
  return finish(fn, launch_aba(mv, B, q, qd, tau, qdd, launch_of(m, JK_ABA, B, stream)));
}

}  // extern "C"

namespace fst {
// Tiles of the SM-pinned fused step: per role slot, the number of tiles and
// the environments per tile. ABA runs two level-parallel tiles of 32 at a
// time (64 environments); the other roles take about as many tiles as they
// have SMs (pin_table), of a multiple of 32 and at most 256 environments.
// Returns the launch's dynamic shared memory: the larger of two ABA tiles
// and 256 environments' staged inputs, and at least 116 KB, so that no two
// blocks share an SM.
size_t pinned_step_plan(const fst_model* m, int64_t B, const EvalArgs& a, int sms, PinArgs& p) {
  const int rows = m->nq + 2 * m->nv;
  size_t sh = (size_t)rows * 256 * sizeof(float);
  for (int r = 0; r < a.n_roles; ++r) {
    const int role = a.roles[r];
    if (role == ROLE_ABA) {
      p.envs[r] = 64;
      p.tiles[r] = (int)((B + 63) / 64);
      const size_t aba = (size_t)2 * (rows + kAbaStateFloats * m->n) * 32 * sizeof(float);
      if (aba > sh) sh = aba;
      continue;
    }
    int n_sm = 0;
    if (m->sm_ids.empty()) {
      for (int s = 0; s < sms && s < kPinTableSize; ++s) n_sm += m->pin_table[s] == role;
    } else {
      for (int s : m->sm_ids) n_sm += s < kPinTableSize && m->pin_table[s] == role;
    }
    int64_t E = (B + (n_sm > 0 ? n_sm : 1) - 1) / (n_sm > 0 ? n_sm : 1);
    E = (E + 31) / 32 * 32;
    E = E < 32 ? 32 : (E > 256 ? 256 : E);
    p.envs[r] = (int)E;
    p.tiles[r] = (int)((B + E - 1) / E);
  }
  sh += (size_t)m->n * (sizeof(BodyC) + sizeof(BodyI)) + (sizeof(TopoLists) + 15) / 16 * 16;  // the staged model
  const size_t one_per_sm = 116 * 1024;
  return sh > one_per_sm ? sh : one_per_sm;
}

// Packed Jacobian layout: columns (support-path DOFs) of each link and the
// first row of its block.
void packed_cols(const fst_model* m, const LinkList& links, PackedJ& pj) {
  int off = 0;
  for (int l = 0; l < links.n; ++l) {
    int cols = 0;
    const uint64_t anc = m->ancestors[links.idx[l]];
    for (int k = 0; k < m->n; ++k)
      if ((anc >> k) & 1ull) {
        const int t = m->hi[k].type;
        cols += t == FST_JOINT_FREE ? 6 : (t == FST_JOINT_FIXED ? 0 : 1);
      }
    pj.cols[l] = cols;
    pj.off[l] = off;
    off += 6 * cols;
  }
}
}  // namespace fst

extern "C" {

fst_status fst_packed_layout(const fst_model* m, const int32_t* links, int32_t n_links, int32_t* cols, int32_t* j_rows,
                             int32_t* m_rows) {
  static const char* fn = "fst_packed_layout";
  if (!m) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null model");
  if (n_links < 0 || n_links > FST_MAX_LINKS || (n_links > 0 && !links))
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": need 0 <= n_links <= FST_MAX_LINKS links");
  LinkList L{};
  L.n = n_links;
  for (int l = 0; l < n_links; ++l) {
    if (links[l] < 0 || links[l] >= m->n) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": link out of range");
    L.idx[l] = links[l];
  }
  PackedJ pj{};
  packed_cols(m, L, pj);
  int rows = 0;
  for (int l = 0; l < n_links; ++l) {
    if (cols) cols[l] = pj.cols[l];
    rows += 6 * pj.cols[l];
  }
  if (j_rows) *j_rows = rows;
  if (m_rows) *m_rows = m->nv * (m->nv + 1) / 2;
  return FST_OK;
}

fst_status fst_eval(const fst_model* m, int64_t B, const fst_eval_io* io, const float* theta, void* stream) {
  static const char* fn = "fst_eval";
  if (!io) return set_error(FST_ERR_INVALID_ARG, "fst_eval: null io");
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  EvalArgs a{};
  a.q = io->q;
  a.qd = io->qd;
  a.qdd = io->qdd;
  a.tau = io->tau;
  a.poses = io->poses;
  a.J = io->J;
  a.tau_out = io->tau_out;
  a.M = io->M;
  a.qdd_out = io->qdd_out;
  if (io->J) {
    if (!io->links || io->n_links < 1 || io->n_links > FST_MAX_LINKS)
      return set_error(FST_ERR_INVALID_ARG, "fst_eval: J needs 1 <= n_links <= FST_MAX_LINKS links");
    a.links.n = io->n_links;
    for (int l = 0; l < io->n_links; ++l) {
      if (io->links[l] < 0 || io->links[l] >= m->n) return set_error(FST_ERR_INVALID_ARG, "fst_eval: link index out of range");
      a.links.idx[l] = io->links[l];
    }
  }
  if (io->flags & ~(FST_EVAL_ONE_SWEEP | FST_EVAL_PACKED))
    return set_error(FST_ERR_INVALID_ARG, "fst_eval: unknown flags");
  if (io->flags & FST_EVAL_PACKED) {
    a.packed = 1;
    packed_cols(m, a.links, a.pj);
  }
  const bool dyn = m->nv > 0;
  const bool vjp = dyn && (io->q_bar || io->qd_bar || io->qdd_bar);
  if (io->qdd_out && dyn) {
    FST_CHECK(need(fn, io->qd, "qd"));
    FST_CHECK(need(fn, io->tau, "tau"));
    a.roles[a.n_roles++] = ROLE_ABA;
  }
  if (io->M && dyn) a.roles[a.n_roles++] = ROLE_CRBA;
  const bool rnea = dyn && (io->tau_out || vjp);
  if (rnea) {
    FST_CHECK(need(fn, io->qd, "qd"));
    FST_CHECK(need(fn, io->qdd, "qdd"));
    if (vjp) {
      FST_CHECK(need(fn, io->tau_bar, "tau_bar"));
      a.tau_bar = io->tau_bar;
      a.qbar = m->nq ? io->q_bar : nullptr;
      a.qdbar = io->qd_bar;
      a.qddbar = io->qdd_bar;
      a.rnea_flags |= EVAL_RNEA_VJP;
      if (io->tau_bar == io->tau_out) a.rnea_flags |= EVAL_TBAR_IS_TAU;
    }
    a.roles[a.n_roles++] = ROLE_RNEA;
  }
  if (io->poses || (io->J && dyn)) {
    if (!io->poses) a.poses = nullptr;
    if (!dyn) a.J = nullptr;
    if (rnea && (io->flags & FST_EVAL_ONE_SWEEP))
      a.rnea_flags |= EVAL_KIN_IN_RNEA;
    else
      a.roles[a.n_roles++] = ROLE_KIN;
  }
  if (skip || a.n_roles == 0) return FST_OK;
  if (m->nq) FST_CHECK(need(fn, io->q, "q"));
  const ModelView mv = view_of(m, theta);
  if (a.rnea_flags || a.packed) {
    // the shared sweep and the packed layouts live in the one-environment-
    // per-thread fused kernels
    const int rows = m->nq + (vjp ? 3 : 2) * m->nv;
    if (jit_has_slot(m, JK_EVAL, JK_SLOT_EVAL_EXT) && m->variant[JK_EVAL] != FST_VARIANT_GENERIC)
      return finish(fn, jit_go_slot(m, JK_EVAL, JK_SLOT_EVAL_EXT, B, rows, 0, (unsigned)a.n_roles,
                                    (cudaStream_t)stream, nullptr, mv, B, a));
    return finish(fn, launch_eval(mv, B, a, launch_of(m, JK_EVAL, B, stream)));
  }
  if (use_level(m, JK_EVAL, LEVEL_EVAL))
    return finish(fn, launch_eval_level(mv, B, a, level_block(m, JK_EVAL), level_tiles(m, JK_EVAL),
                        (cudaStream_t)stream));
  if (m->variant[JK_EVAL] == FST_VARIANT_MIXED && jit_has(m, JK_EVAL_MIXED)) {
    // roles whose own operator is tuned level-parallel run that way here too
    const int T = block_of(m, JK_EVAL, B);
    const int rows = m->nq + 2 * m->nv;
    size_t sh = 0;
    int64_t gx = 0;
    for (int r = 0; r < a.n_roles; ++r) {
      const int role = a.roles[r];
      const int kind = role == ROLE_ABA ? JK_ABA : role == ROLE_CRBA ? JK_CRBA : role == ROLE_RNEA ? JK_RNEA
                                                                     : (a.J ? JK_JACOBIAN : JK_FK);
      // a level-parallel role of the mixed kernel runs on a model copy in
      // shared memory and keeps its per-body state after nq + 2 nv staged
      // rows whatever rows the role stages (the kernel's layout)
      const int F = role == ROLE_ABA ? kAbaStateFloats : role == ROLE_CRBA ? kCrbaStateFloats
                  : role == ROLE_RNEA ? kRneaStateFloats : kFkStateFloats;
      const size_t level_need = model_smem_bytes(m->n) + ((size_t)rows + (size_t)F * m->n) * 32 * sizeof(float);
      size_t need;
      int64_t blocks;
      // any level-parallel setting of the operator (one tile, two tiles or
      // lean state) makes its role level-parallel here, one tile per block
      const int kv = m->variant[kind];
      if ((kv == FST_VARIANT_LEVEL || kv == FST_VARIANT_LEVEL2 || kv == FST_VARIANT_LEVEL_LEAN) &&
          level_need <= kLevelSmemLimit) {
        a.level_mask |= 1 << role;
        need = level_need;
        blocks = (B + 31) / 32;
      } else {
        need = (size_t)rows * T * sizeof(float);
        blocks = (B + T - 1) / T;
      }
      if (need > sh) sh = need;
      if (blocks > gx) gx = blocks;
    }
    void* argv[] = {(void*)&mv, (void*)&B, (void*)&a};
    return finish(fn, jit_launch(m, JK_EVAL_MIXED, dim3((unsigned)gx, (unsigned)a.n_roles), T, sh,
                                 (cudaStream_t)stream, argv));
  }
  if (m->variant[JK_EVAL] == FST_VARIANT_PINNED && jit_has_slot(m, JK_EVAL, 3)) {
    int* counters = m->dpin + kPinTableSize + kPinEvalRegion * kPinRegion;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
    if (sms < 1) sms = 1;
    PinArgs p{m->dpin, counters, {0, 0, 0, 0}, {0, 0, 0, 0}};
    const size_t sh = pinned_step_plan(m, B, a, sms, p);
    if (sh > kLevelSmemLimit) return set_error(FST_ERR_INVALID_ARG, "fst_eval: the tree is too large for the pinned step");
    cudaError_t err = cudaMemsetAsync(counters, 0, sizeof(int) * kPinRegion, (cudaStream_t)stream);
    if (err == cudaSuccess) {
      void* argv[] = {(void*)&mv, (void*)&B, (void*)&a, (void*)&p};
      err = jit_launch_slot3(m, JK_EVAL, 3, dim3((unsigned)sms), dim3(32, 2, 4), sh, (cudaStream_t)stream, argv);
    }
    return finish(fn, err);
  }
  if (use_path(m, JK_EVAL))
    return finish(fn, path_go(m, JK_EVAL, B, m->nq + 2 * m->nv, (unsigned)a.n_roles, (cudaStream_t)stream, mv, B, a));
  if (use_jit(m, JK_EVAL))
    return finish(fn, jit_go(m, JK_EVAL, B, m->nq + 2 * m->nv, 0, (unsigned)a.n_roles, (cudaStream_t)stream, nullptr,
                             mv, B, a));
  return finish(fn, launch_eval(mv, B, a, launch_of(m, JK_EVAL, B, stream)));
}

fst_status fst_adjoint_scratch_bytes(const fst_model* m, int64_t B, size_t* bytes) {
  if (!m || !bytes || B < 0) return set_error(FST_ERR_INVALID_ARG, "fst_adjoint_scratch_bytes: bad argument");
  *bytes = vjp_scratch_floats(m->n, B) * sizeof(float);
  return FST_OK;
}

namespace {
fst_status need_scratch(const char* fn, const fst_model* m, int64_t B, const void* scratch, size_t bytes) {
  if (!scratch) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": theta_bar needs scratch");
  if (bytes < vjp_scratch_floats(m->n, B) * sizeof(float))
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": scratch smaller than fst_adjoint_scratch_bytes()");
  return FST_OK;
}
}  // namespace

fst_status fst_fk_vjp(const fst_model* m, int64_t B, const float* q, const float* poses_bar, float* q_bar,
                      void* stream) {
  static const char* fn = "fst_fk_vjp";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip || m->nq == 0 || !q_bar) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, poses_bar, "poses_bar"));
  const ModelView mv = view_of(m, nullptr);
  if (use_jit(m, JK_FK_VJP))
    return finish(fn, jit_go(m, JK_FK_VJP, B, m->nq + 12 * m->n, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q,
                             poses_bar, q_bar));
  return finish(fn, launch_fk_vjp(mv, B, q, poses_bar, q_bar, (cudaStream_t)stream));
}

fst_status fst_rnea_vjp(const fst_model* m, int64_t B, const float* q, const float* qd, const float* qdd,
                        const float* theta, const float* tau_bar, float* q_bar, float* qd_bar, float* qdd_bar,
                        float* theta_bar, void* scratch, size_t scratch_bytes, void* stream) {
  static const char* fn = "fst_rnea_vjp";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (theta_bar) FST_CHECK(need_scratch(fn, m, B, scratch, scratch_bytes));
  if (skip || m->nv == 0) {
    return finish(fn, zero_outputs((cudaStream_t)stream, {{theta_bar, sizeof(float) * m->n * 10}}));
  }
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, qdd, "qdd"));
  FST_CHECK(need(fn, tau_bar, "tau_bar"));
  const ModelView mv = view_of(m, theta);
  if (use_jit(m, JK_RNEA_VJP)) {
    unsigned nblk = 0;
    float* partial = theta_bar ? (float*)scratch : nullptr;
    const int P = theta_bar ? m->n * 10 : 0;
    cudaError_t err = jit_go(m, JK_RNEA_VJP, B, m->nq + 3 * m->nv, P, 1, (cudaStream_t)stream, &nblk, mv, B, q, qd,
                             qdd, tau_bar, q_bar, qd_bar, qdd_bar, partial);
    if (err == cudaSuccess && theta_bar) err = launch_partial_reduce(partial, (int)nblk, P, theta_bar, (cudaStream_t)stream);
    return finish(fn, err);
  }
  return finish(fn, launch_rnea_vjp(mv, B, q, qd, qdd, tau_bar, q_bar, qd_bar, qdd_bar, theta_bar,
                                    (float*)scratch, (cudaStream_t)stream));
}

fst_status fst_rnea_tape_bytes(const fst_model* m, int64_t B, size_t* bytes) {
  if (!m || !bytes) return set_error(FST_ERR_INVALID_ARG, "fst_rnea_tape_bytes: null argument");
  if (B < 0) return set_error(FST_ERR_INVALID_ARG, "fst_rnea_tape_bytes: B must be >= 0");
  *bytes = sizeof(float) * (size_t)kTapeFloatsPerBody * (size_t)m->n * (size_t)B;
  return FST_OK;
}

fst_status fst_rnea_store(const fst_model* m, int64_t B, const float* q, const float* qd, const float* qdd,
                          const float* theta, float* tau, float* tape, size_t tape_bytes, void* stream) {
  static const char* fn = "fst_rnea_store";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip) return FST_OK;
  FST_CHECK(need(fn, tape, "tape"));
  if (tape_bytes < sizeof(float) * (size_t)kTapeFloatsPerBody * (size_t)m->n * (size_t)B)
    return set_error(FST_ERR_INVALID_ARG, "fst_rnea_store: tape smaller than fst_rnea_tape_bytes()");
  FST_CHECK(need(fn, q, "q"));
  if (m->nv) {
    FST_CHECK(need(fn, qd, "qd"));
    FST_CHECK(need(fn, qdd, "qdd"));
  }
  const ModelView mv = view_of(m, theta);
  if (use_jit(m, JK_RNEA_STORE))
    return finish(fn, jit_go(m, JK_RNEA_STORE, B, m->nq + 2 * m->nv, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q,
                             qd, qdd, tau, tape));
  return finish(fn, launch_rnea_store(mv, B, q, qd, qdd, tau, tape, launch_of(m, JK_RNEA_STORE, B, stream)));
}

fst_status fst_rnea_vjp_stored(const fst_model* m, int64_t B, const float* q, const float* qd, const float* theta,
                               const float* tape, size_t tape_bytes, const float* tau_bar, float* q_bar,
                               float* qd_bar, float* qdd_bar, float* theta_bar, void* scratch, size_t scratch_bytes,
                               void* stream) {
  static const char* fn = "fst_rnea_vjp_stored";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (theta_bar) FST_CHECK(need_scratch(fn, m, B, scratch, scratch_bytes));
  if (skip || m->nv == 0) {
    return finish(fn, zero_outputs((cudaStream_t)stream, {{theta_bar, sizeof(float) * m->n * 10}}));
  }
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, tape, "tape"));
  FST_CHECK(need(fn, tau_bar, "tau_bar"));
  if (tape_bytes < sizeof(float) * (size_t)kTapeFloatsPerBody * (size_t)m->n * (size_t)B)
    return set_error(FST_ERR_INVALID_ARG, "fst_rnea_vjp_stored: tape smaller than fst_rnea_tape_bytes()");
  const ModelView mv = view_of(m, theta);
  if (use_jit(m, JK_RNEA_VJP_STORED)) {
    unsigned nblk = 0;
    float* partial = theta_bar ? (float*)scratch : nullptr;
    const int P = theta_bar ? m->n * 10 : 0;
    cudaError_t err = jit_go(m, JK_RNEA_VJP_STORED, B, m->nq + 2 * m->nv, P, 1, (cudaStream_t)stream, &nblk, mv, B, q,
                             qd, tape, tau_bar, q_bar, qd_bar, qdd_bar, partial);
    if (err == cudaSuccess && theta_bar) err = launch_partial_reduce(partial, (int)nblk, P, theta_bar, (cudaStream_t)stream);
    return finish(fn, err);
  }
  return finish(fn, launch_rnea_vjp_stored(mv, B, q, qd, tape, tau_bar, q_bar, qd_bar, qdd_bar, theta_bar,
                                           (float*)scratch, (cudaStream_t)stream));
}

fst_status fst_jacobian_vjp(const fst_model* m, int64_t B, const float* q, const int32_t* links, int32_t n_links,
                            const float* J_bar, float* q_bar, void* stream) {
  static const char* fn = "fst_jacobian_vjp";
  if (!links && n_links) return set_error(FST_ERR_INVALID_ARG, "fst_jacobian_vjp: null links");
  if (n_links < 1 || n_links > FST_MAX_LINKS)
    return set_error(FST_ERR_INVALID_ARG, "fst_jacobian_vjp: n_links must be in [1, FST_MAX_LINKS]");
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  LinkList L{};
  L.n = n_links;
  for (int l = 0; l < n_links; ++l) {
    if (links[l] < 0 || links[l] >= m->n)
      return set_error(FST_ERR_INVALID_ARG, "fst_jacobian_vjp: link index out of range");
    L.idx[l] = links[l];
  }
  if (skip) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, q_bar, "q_bar"));
  if (m->nv == 0) return finish(fn, cudaMemsetAsync(q_bar, 0, sizeof(float) * m->nq * (size_t)B, (cudaStream_t)stream));
  FST_CHECK(need(fn, J_bar, "J_bar"));
  return finish(fn, launch_jac_vjp(view_of(m, nullptr), B, q, L, J_bar, q_bar, (cudaStream_t)stream));
}

fst_status fst_crba_vjp(const fst_model* m, int64_t B, const float* q, const float* theta, const float* M_bar,
                        float* q_bar, float* theta_bar, void* scratch, size_t scratch_bytes, void* stream) {
  static const char* fn = "fst_crba_vjp";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (theta_bar) FST_CHECK(need_scratch(fn, m, B, scratch, scratch_bytes));
  if (skip || m->nv == 0) {
    return finish(fn, zero_outputs((cudaStream_t)stream, {{theta_bar, sizeof(float) * m->n * 10},
                                                          {q_bar, sizeof(float) * m->nq * (size_t)B}}));
  }
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, M_bar, "M_bar"));
  return finish(fn, launch_crba_vjp(view_of(m, theta), B, q, M_bar, q_bar, theta_bar, (float*)scratch,
                                    (cudaStream_t)stream));
}

fst_status fst_rnea_derivatives(const fst_model* m, int64_t B, const float* q, const float* qd, const float* qdd,
                                const float* theta, float* dtau_dq, float* dtau_dqd, void* stream) {
  static const char* fn = "fst_rnea_derivatives";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip || m->nv == 0 || (!dtau_dq && !dtau_dqd)) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, qdd, "qdd"));
  const ModelView mv = view_of(m, theta);
  if (use_jit(m, JK_RNEA_DERIVS))
    return finish(fn, jit_go(m, JK_RNEA_DERIVS, B, m->nq + 2 * m->nv, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q,
                             qd, qdd, dtau_dq, dtau_dqd));
  return finish(fn, launch_rnea_derivs(mv, B, q, qd, qdd, dtau_dq, dtau_dqd, launch_of(m, JK_RNEA_DERIVS, B, stream)));
}

fst_status fst_aba_derivatives(const fst_model* m, int64_t B, const float* q, const float* qd, const float* tau,
                               const float* theta, float* qdd, float* dqdd_dq, float* dqdd_dqd, float* Minv,
                               void* stream) {
  static const char* fn = "fst_aba_derivatives";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip || m->nv == 0) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, tau, "tau"));
  FST_CHECK(need(fn, Minv, "Minv"));
  const ModelView mv = view_of(m, theta);
  if (use_jit(m, JK_ABA_DERIVS))
    return finish(fn, jit_go(m, JK_ABA_DERIVS, B, m->nq + 3 * m->nv, 0, 1, (cudaStream_t)stream, nullptr, mv, B, q,
                             qd, tau, qdd, dqdd_dq, dqdd_dqd, Minv));
  return finish(fn, launch_aba_derivs(mv, B, q, qd, tau, qdd, dqdd_dq, dqdd_dqd, Minv,
                                      launch_of(m, JK_ABA_DERIVS, B, stream)));
}

fst_status fst_aba_vjp(const fst_model* m, int64_t B, const float* q, const float* qd, const float* qdd,
                       const float* theta, const float* qdd_bar, float* q_bar, float* qd_bar, float* tau_bar,
                       float* theta_bar, void* scratch, size_t scratch_bytes, void* stream) {
  static const char* fn = "fst_aba_vjp";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (theta_bar) FST_CHECK(need_scratch(fn, m, B, scratch, scratch_bytes));
  if (skip || m->nv == 0) {
    return finish(fn, zero_outputs((cudaStream_t)stream, {{theta_bar, sizeof(float) * m->n * 10}}));
  }
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, qdd, "qdd"));
  FST_CHECK(need(fn, qdd_bar, "qdd_bar"));
  const ModelView mv = view_of(m, theta);
  if (use_jit(m, JK_ABA_VJP)) {
    unsigned nblk = 0;
    float* partial = theta_bar ? (float*)scratch : nullptr;
    const int P = theta_bar ? m->n * 10 : 0;
    cudaError_t err = jit_go(m, JK_ABA_VJP, B, m->nq + 4 * m->nv, P, 1, (cudaStream_t)stream, &nblk, mv, B, q, qd,
                             qdd, qdd_bar, q_bar, qd_bar, tau_bar, partial);
    if (err == cudaSuccess && theta_bar) err = launch_partial_reduce(partial, (int)nblk, P, theta_bar, (cudaStream_t)stream);
    return finish(fn, err);
  }
  return finish(fn, launch_aba_vjp(mv, B, q, qd, qdd, qdd_bar, q_bar, qd_bar, tau_bar, theta_bar,
                                   (float*)scratch, (cudaStream_t)stream));
}

fst_status fst_rnea_loss_grad(const fst_model* m, int64_t B, const float* q, const float* qd, const float* qdd,
                              const float* theta, const float* tau_meas, float* loss_theta_bar, float* q_bar,
                              float* qd_bar, void* scratch, size_t scratch_bytes, void* stream) {
  static const char* fn = "fst_rnea_loss_grad";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  FST_CHECK(need(fn, loss_theta_bar, "loss_theta_bar"));
  FST_CHECK(need_scratch(fn, m, B, scratch, scratch_bytes));
  if (skip || m->nv == 0) {
    return finish(fn, zero_outputs((cudaStream_t)stream, {{loss_theta_bar, sizeof(float) * (m->n * 10 + 1)}}));
  }
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, qdd, "qdd"));
  FST_CHECK(need(fn, tau_meas, "tau_meas"));
  const ModelView mv = view_of(m, theta);
  if (use_jit(m, JK_LOSS_GRAD)) {
    unsigned nblk = 0;
    const int P = m->n * 10 + 1;
    cudaError_t err = jit_go(m, JK_LOSS_GRAD, B, m->nq + 3 * m->nv, P, 1, (cudaStream_t)stream, &nblk, mv, B, q, qd,
                             qdd, tau_meas, q_bar, qd_bar, (float*)scratch);
    if (err == cudaSuccess) err = launch_partial_reduce((float*)scratch, (int)nblk, P, loss_theta_bar, (cudaStream_t)stream);
    return finish(fn, err);
  }
  return finish(fn, launch_rnea_loss_grad(mv, B, q, qd, qdd, tau_meas, loss_theta_bar, q_bar, qd_bar,
                                          (float*)scratch, (cudaStream_t)stream));
}

fst_status fst_multi_create(const fst_model* const* models, int32_t n_models, fst_multi** out) {
  static const char* fn = "fst_multi_create";
  if (!out || !models) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null argument");
  *out = nullptr;
  if (n_models < 1 || n_models > FST_MAX_MULTI)
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": n_models must be in [1, FST_MAX_MULTI]");
  for (int k = 0; k < n_models; ++k) {
    if (!models[k]) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null model");
    if (models[k]->device != models[0]->device)
      return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": models live on different devices");
  }
  fst_multi* g = new (std::nothrow) fst_multi();
  if (!g) return set_error(FST_ERR_NO_MEMORY, std::string(fn) + ": host allocation failed");
  g->models.assign(models, models + n_models);
  g->device = models[0]->device;
  cudaError_t err = cudaMalloc((void**)&g->counter, sizeof(int));
  if (err != cudaSuccess) {
    delete g;
    return cuda_error(fn, err);
  }
  *out = g;
  return FST_OK;
}

fst_status fst_multi_destroy(fst_multi* g) {
  if (!g) return FST_OK;
  if (g->counter) cudaFree(g->counter);
  delete g;
  return FST_OK;
}

fst_status fst_multi_eval(fst_multi* g, const fst_multi_io* io, void* stream) {
  static const char* fn = "fst_multi_eval";
  if (!g || !io) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null argument");
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return cuda_error(fn, err);
  if (dev != g->device) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": not the group's device");
  const int n = (int)g->models.size();
  MultiArgs a{};
  a.counter = g->counter;
  int max_n = 1;
  for (int k = 0; k < n; ++k) {
    const fst_model* m = g->models[k];
    const fst_multi_io& x = io[k];
    if (x.B < 0 || x.B > (int64_t)INT32_MAX)
      return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": B must be in [0, 2^31 - 1]");
    if (x.B > 0 && m->nq && !x.q) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null q");
    if (x.B > 0 && x.tau_out && (!x.qd || !x.qdd)) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": RNEA needs qd and qdd");
    if (x.B > 0 && x.qdd_out && (!x.qd || !x.tau)) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": ABA needs qd and tau");
    a.mv[k] = view_of(m, nullptr);
    a.io[k] = MultiIO{x.q, x.qd, x.qdd, x.tau, x.poses, m->nv ? x.tau_out : nullptr, m->nv ? x.M : nullptr,
                      m->nv ? x.qdd_out : nullptr, x.B};
    if (m->n > max_n) max_n = m->n;
    a.maxw[k] = m->max_width;
    const int rows = m->nq + 2 * m->nv;
    if (rows > a.max_rows) a.max_rows = rows;
  }
  // heaviest first: ABA, CRBA, RNEA, FK; within one, trees with most bodies first
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && g->models[order[j]]->n > g->models[order[j - 1]]->n; --j) std::swap(order[j], order[j - 1]);
  const bool level = g->variant == FST_VARIANT_LEVEL;
  const int T = level ? 32 : g->block;  // environments per item
  size_t state_bytes = 0;               // level: per-body state of the largest (tree, operator) pair
  // every block of the persistent grid draws one item past the last, so the
  // int work counter reaches n_items + grid: keep ample headroom below 2^31
  const int64_t kMaxItems = (int64_t)INT32_MAX - (1 << 24);
  int seg = 0;
  int64_t items = 0;
  const int roles[4] = {ROLE_ABA, ROLE_CRBA, ROLE_RNEA, ROLE_KIN};
  for (int r : roles)
    for (int k : order) {
      const MultiIO& x = a.io[k];
      const void* outp = r == ROLE_ABA ? (const void*)x.qdd_out
                       : r == ROLE_CRBA ? (const void*)x.M
                       : r == ROLE_RNEA ? (const void*)x.tau_out : (const void*)x.poses;
      if (!outp || x.B == 0) continue;
      if (level) {
        const fst_model* m = g->models[k];
        const size_t floats = r == ROLE_ABA ? (size_t)kAbaLeanBodyFloats * m->n + 2 * kAbaLeanRingFloats * m->max_width
                              : (size_t)(r == ROLE_CRBA ? kCrbaStateFloats
                                         : r == ROLE_RNEA ? kRneaStateFloats : kFkStateFloats) * m->n;
        const size_t need = floats * 32 * sizeof(float);
        if (need > state_bytes) state_bytes = need;
      }
      a.seg_start[seg] = (int)items;  // within kMaxItems: checked below on every addition
      a.seg_model[seg] = (unsigned char)k;
      a.seg_op[seg] = (unsigned char)r;
      items += (x.B + T - 1) / T;
      if (items > kMaxItems)
        return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": too many work items (environments x operators)");
      ++seg;
    }
  a.seg_start[seg] = (int)items;
  a.n_items = (int)items;
  a.model_bytes = (size_t)max_n * (sizeof(BodyC) + sizeof(BodyI)) + (sizeof(TopoLists) + 15) / 16 * 16;
  a.model_bytes = (a.model_bytes + 15) / 16 * 16;
  if (items == 0) return FST_OK;
  if (level) {
    const size_t sh = a.model_bytes + (size_t)a.max_rows * 32 * sizeof(float) + state_bytes;
    if (sh > kLevelSmemLimit)
      return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": the level-parallel state of the largest tree "
                                                              "does not fit in shared memory");
    return finish(fn, launch_multi_level(a, state_bytes, g->block, (cudaStream_t)stream));
  }
  return finish(fn, launch_multi(a, max_n, T, (cudaStream_t)stream));
}

fst_status fst_multi_set_launch(fst_multi* g, int32_t block, int32_t variant) {
  static const char* fn = "fst_multi_set_launch";
  if (!g) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null group");
  if (variant != FST_VARIANT_GENERIC && variant != FST_VARIANT_LEVEL)
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": the variant must be FST_VARIANT_GENERIC or FST_VARIANT_LEVEL");
  if (block != 32 && block != 64 && block != 128 && block != 256)
    return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": block must be 32, 64, 128 or 256");
  g->block = block;
  g->variant = variant;
  return FST_OK;
}

}  // extern "C"
