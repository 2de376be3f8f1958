// C ABI of libfst.so: argument validation, device checks, launches.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <sstream>
#include <string>

#include "fst_internal.h"
#include "launch.h"

namespace fst {

namespace {
thread_local std::string g_last_error;
}

fst_status set_error(fst_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

namespace {

fst_status cuda_error(const char* where, cudaError_t err) {
  std::ostringstream os;
  os << where << ": " << cudaGetErrorName(err) << ": " << cudaGetErrorString(err);
  return set_error(FST_ERR_CUDA, os.str());
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
  if (B > (int64_t)1 << 40) return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": B too large");
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return cuda_error(fn, err);
  if (dev != m->device) {
    std::ostringstream os;
    os << fn << ": current device " << dev << " is not the model's device " << m->device;
    return set_error(FST_ERR_INVALID_ARG, os.str());
  }
  return FST_OK;
}

fst_status need(const char* fn, const void* p, const char* name) {
  if (p) return FST_OK;
  return set_error(FST_ERR_INVALID_ARG, std::string(fn) + ": null " + name);
}

Launch launch_of(int64_t B, void* stream) { return Launch{default_block(B), (cudaStream_t)stream}; }

fst_status finish(const char* fn, cudaError_t err) {
  if (err != cudaSuccess) return cuda_error(fn, err);
  return FST_OK;
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
  if (err != cudaSuccess) {
    fst_status st = (err == cudaErrorMemoryAllocation) ? set_error(FST_ERR_NO_MEMORY, "fst_model_create: cudaMalloc failed")
                                                       : cuda_error("fst_model_create", err);
    if (m->dc) cudaFree(m->dc);
    if (m->di) cudaFree(m->di);
    delete m;
    return st;
  }
  *out = m;
  return FST_OK;
}

fst_status fst_model_destroy(fst_model* m) {
  if (!m) return FST_OK;
  if (m->dc) cudaFree(m->dc);
  if (m->di) cudaFree(m->di);
  delete m;
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
  return finish(fn, launch_fk(view_of(m, nullptr), B, q, poses, launch_of(B, stream)));
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
  return finish(fn, launch_jacobian(view_of(m, nullptr), B, q, L, J, launch_of(B, stream)));
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
  return finish(fn, launch_rnea(view_of(m, theta), B, q, qd, qdd, tau, launch_of(B, stream)));
}

fst_status fst_crba(const fst_model* m, int64_t B, const float* q, const float* theta, float* M, void* stream) {
  static const char* fn = "fst_crba";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (skip || m->nv == 0) return FST_OK;
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, M, "M"));
  return finish(fn, launch_crba(view_of(m, theta), B, q, M, launch_of(B, stream)));
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
  return finish(fn, launch_aba(view_of(m, theta), B, q, qd, tau, qdd, launch_of(B, stream)));
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
  const bool dyn = m->nv > 0;
  if (io->qdd_out && dyn) {
    FST_CHECK(need(fn, io->qd, "qd"));
    FST_CHECK(need(fn, io->tau, "tau"));
    a.roles[a.n_roles++] = ROLE_ABA;
  }
  if (io->M && dyn) a.roles[a.n_roles++] = ROLE_CRBA;
  if (io->tau_out && dyn) {
    FST_CHECK(need(fn, io->qd, "qd"));
    FST_CHECK(need(fn, io->qdd, "qdd"));
    a.roles[a.n_roles++] = ROLE_RNEA;
  }
  if (io->poses || (io->J && dyn)) {
    if (!io->poses) a.poses = nullptr;
    if (!dyn) a.J = nullptr;
    a.roles[a.n_roles++] = ROLE_KIN;
  }
  if (skip || a.n_roles == 0) return FST_OK;
  if (m->nq) FST_CHECK(need(fn, io->q, "q"));
  return finish(fn, launch_eval(view_of(m, theta), B, a, launch_of(B, stream)));
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
  return finish(fn, launch_fk_vjp(view_of(m, nullptr), B, q, poses_bar, q_bar, (cudaStream_t)stream));
}

fst_status fst_rnea_vjp(const fst_model* m, int64_t B, const float* q, const float* qd, const float* qdd,
                        const float* theta, const float* tau_bar, float* q_bar, float* qd_bar, float* qdd_bar,
                        float* theta_bar, void* scratch, size_t scratch_bytes, void* stream) {
  static const char* fn = "fst_rnea_vjp";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (theta_bar) FST_CHECK(need_scratch(fn, m, B, scratch, scratch_bytes));
  if (skip || m->nv == 0) {
    if (theta_bar && m->n) cudaMemsetAsync(theta_bar, 0, sizeof(float) * m->n * 10, (cudaStream_t)stream);
    return FST_OK;
  }
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, qdd, "qdd"));
  FST_CHECK(need(fn, tau_bar, "tau_bar"));
  return finish(fn, launch_rnea_vjp(view_of(m, theta), B, q, qd, qdd, tau_bar, q_bar, qd_bar, qdd_bar, theta_bar,
                                    (float*)scratch, (cudaStream_t)stream));
}

fst_status fst_aba_vjp(const fst_model* m, int64_t B, const float* q, const float* qd, const float* qdd,
                       const float* theta, const float* qdd_bar, float* q_bar, float* qd_bar, float* tau_bar,
                       float* theta_bar, void* scratch, size_t scratch_bytes, void* stream) {
  static const char* fn = "fst_aba_vjp";
  bool skip;
  FST_CHECK(check_call(fn, m, B, &skip));
  if (theta_bar) FST_CHECK(need_scratch(fn, m, B, scratch, scratch_bytes));
  if (skip || m->nv == 0) {
    if (theta_bar && m->n) cudaMemsetAsync(theta_bar, 0, sizeof(float) * m->n * 10, (cudaStream_t)stream);
    return FST_OK;
  }
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, qdd, "qdd"));
  FST_CHECK(need(fn, qdd_bar, "qdd_bar"));
  return finish(fn, launch_aba_vjp(view_of(m, theta), B, q, qd, qdd, qdd_bar, q_bar, qd_bar, tau_bar, theta_bar,
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
    cudaMemsetAsync(loss_theta_bar, 0, sizeof(float) * (m->n * 10 + 1), (cudaStream_t)stream);
    return FST_OK;
  }
  FST_CHECK(need(fn, q, "q"));
  FST_CHECK(need(fn, qd, "qd"));
  FST_CHECK(need(fn, qdd, "qdd"));
  FST_CHECK(need(fn, tau_meas, "tau_meas"));
  return finish(fn, launch_rnea_loss_grad(view_of(m, theta), B, q, qd, qdd, tau_meas, loss_theta_bar, q_bar, qd_bar,
                                          (float*)scratch, (cudaStream_t)stream));
}

}  // extern "C"
