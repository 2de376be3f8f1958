// Adjoint kernels (bodies in adjoint.cuh) and the deterministic two-stage
// reduction of the inertial-parameter gradient.
//
// thetabar is a sum over all B environments. Each block first reduces its
// environments (warp shuffles, then one shared-memory slot per warp) into a
// per-block partial in the caller's scratch buffer; a second kernel adds the
// partials in block order. No floating-point atomics, so the result is
// bit-reproducible run to run.
#include "adjoint.cuh"
#include "launch.h"

namespace fst {
static_assert(kTapeFloats == kTapeFloatsPerBody, "tape layout");
namespace {

// shared memory: model | staged rows (rows x T floats) | per-warp theta slots
__host__ __device__ inline size_t vjp_smem(int n, int rows, int block, bool theta) {
  return smem_bytes(n, rows, block) + (theta ? (size_t)(block / 32) * n * 10 * sizeof(float) : 0);
}

// Stages rows of src for an active thread, zeros for a padding thread (so
// padding threads run the sweep on finite numbers and add nothing).
__device__ __forceinline__ Col stage_or_zero(float* tile, const float* __restrict__ src, int rows, int64_t B,
                                             int64_t e, bool act) {
  if (act) return stage_rows(tile, src, rows, B, e);
  float* dst = tile + threadIdx.x;
  for (int k = 0; k < rows; ++k) dst[k * blockDim.x] = 0.f;
  return Col{dst, (int)blockDim.x};
}

__device__ __forceinline__ float* theta_slots(float4* smem, int n, int rows) {
  return smem_tile(smem, n) + rows * blockDim.x;
}

__device__ __forceinline__ void zero_slots(float* slots, int count) {
  for (int k = threadIdx.x; k < count; k += blockDim.x) slots[k] = 0.f;
}

// Sums the per-warp slots into this block's partial (P = n*10 values, plus
// `extra` trailing values already summed into slot row 0 by lane 0s).
__device__ __forceinline__ void write_partial(const float* slots, int P, float* partial) {
  const int warps = blockDim.x / 32;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < warps; ++w) s += slots[w * P + p];
    partial[(int64_t)blockIdx.x * P + p] = s;
  }
}

template <int NB>
__global__ void __launch_bounds__(256) rnea_vjp_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                       const float* __restrict__ qd, const float* __restrict__ qdd,
                                                       const float* __restrict__ tbar, float* qbar, float* qdbar,
                                                       float* qddbar, float* partial) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  const int rows = mv.nq + 3 * mv.nv;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  const Col cq = stage_or_zero(tile, q, mv.nq, B, e, act);
  const Col cqd = stage_or_zero(tile + mv.nq * T, qd, mv.nv, B, e, act);
  const Col cqdd = stage_or_zero(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e, act);
  const Col ctb = stage_or_zero(tile + (mv.nq + 2 * mv.nv) * T, tbar, mv.nv, B, e, act);
  float* slots = partial ? theta_slots(smem, mv.n, rows) : nullptr;
  const int P = mv.n * 10;
  if (slots) zero_slots(slots, (T / 32) * P);
  const SmemModel sm = stage_model(mv, smem);
  cp_async_wait_all();
  VjpOut o{qbar, qdbar, qddbar, slots ? slots + (threadIdx.x / 32) * P : nullptr, 1.f, act};
  rnea_vjp_env<NB>(sm, world_accel(mv), cq, cqd, cqdd, ctb, o, B, e);
  if (partial) {
    __syncthreads();
    write_partial(slots, P, partial);
  }
}

// Store variant, forward: tau (optional) and the tape.
template <int NB>
__global__ void __launch_bounds__(256) rnea_store_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                         const float* __restrict__ qd, const float* __restrict__ qdd,
                                                         float* __restrict__ tau, float* __restrict__ tape) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  Col cq{}, cqd{}, cqdd{};
  if (act) {
    cq = stage_rows(tile, q, mv.nq, B, e);
    cqd = stage_rows(tile + mv.nq * T, qd, mv.nv, B, e);
    cqdd = stage_rows(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e);
  }
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  rnea_store_env<NB>(sm, world_accel(mv), cq, cqd, cqdd, tau, tape, B, e);
}

// Store variant, adjoint: the reverse sweeps read the tape (no forward sweep).
template <int NB>
__global__ void __launch_bounds__(256) rnea_vjp_stored_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                              const float* __restrict__ qd,
                                                              const float* __restrict__ tape,
                                                              const float* __restrict__ tbar, float* qbar,
                                                              float* qdbar, float* qddbar, float* partial) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  const int rows = mv.nq + 2 * mv.nv;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  const Col cq = stage_or_zero(tile, q, mv.nq, B, e, act);
  const Col cqd = stage_or_zero(tile + mv.nq * T, qd, mv.nv, B, e, act);
  const Col ctb = stage_or_zero(tile + (mv.nq + mv.nv) * T, tbar, mv.nv, B, e, act);
  float* slots = partial ? theta_slots(smem, mv.n, rows) : nullptr;
  const int P = mv.n * 10;
  if (slots) zero_slots(slots, (T / 32) * P);
  const SmemModel sm = stage_model(mv, smem);
  cp_async_wait_all();
  VjpOut o{qbar, qdbar, qddbar, slots ? slots + (threadIdx.x / 32) * P : nullptr, 1.f, act};
  rnea_vjp_stored_env<NB>(sm, world_accel(mv), cq, cqd, tape, ctb, o, B, e);
  if (partial) {
    __syncthreads();
    write_partial(slots, P, partial);
  }
}

// ABA adjoint: lambda = M^-1 qddbar by an ABA sweep (qd = 0, no gravity),
// then minus the RNEA adjoint at the forward solution qdd with taubar = lambda.
template <int NB>
__global__ void __launch_bounds__(256) aba_vjp_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                      const float* __restrict__ qd, const float* __restrict__ qdd,
                                                      const float* __restrict__ qddbar, float* qbar, float* qdbar,
                                                      float* taubar, float* partial) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  const int rows = mv.nq + 4 * mv.nv;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  const Col cq = stage_or_zero(tile, q, mv.nq, B, e, act);
  const Col cqd = stage_or_zero(tile + mv.nq * T, qd, mv.nv, B, e, act);
  const Col cqdd = stage_or_zero(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e, act);
  const Col cqb = stage_or_zero(tile + (mv.nq + 2 * mv.nv) * T, qddbar, mv.nv, B, e, act);
  float* lam = tile + (mv.nq + 3 * mv.nv) * T + threadIdx.x;
  float* slots = partial ? theta_slots(smem, mv.n, rows) : nullptr;
  const int P = mv.n * 10;
  if (slots) zero_slots(slots, (T / 32) * P);
  const SmemModel sm = stage_model(mv, smem);
  cp_async_wait_all();
  const SV zero = sv_zero();
  aba_env<NB>(sm, zero, cq, cqd, cqb, nullptr, B, e, /*qd_zero=*/true, lam, T);
  const Col clam{lam, T};
  if (taubar && act)
    for (int k = 0; k < mv.nv; ++k) taubar[(int64_t)k * B + e] = clam[k];
  VjpOut o{qbar, qdbar, nullptr, slots ? slots + (threadIdx.x / 32) * P : nullptr, -1.f, act};
  rnea_vjp_env<NB>(sm, world_accel(mv), cq, cqd, cqdd, clam, o, B, e);
  if (partial) {
    __syncthreads();
    write_partial(slots, P, partial);
  }
}

// System-identification loss and its gradient in one pass (paper Sec. 4.3):
// L = sum_env sum_i (RNEA(q, qd, qdd; theta)_i - tau_meas_i)^2. The forward
// state stays on chip between the forward sweep and the reverse sweeps.
// The block's share of L goes to partial[P] (after the P theta values).
template <int NB>
__global__ void __launch_bounds__(256) rnea_loss_grad_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                             const float* __restrict__ qd,
                                                             const float* __restrict__ qdd,
                                                             const float* __restrict__ tau_meas, float* qbar,
                                                             float* qdbar, float* partial) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  const int rows = mv.nq + 3 * mv.nv;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  const Col cq = stage_or_zero(tile, q, mv.nq, B, e, act);
  const Col cqd = stage_or_zero(tile + mv.nq * T, qd, mv.nv, B, e, act);
  const Col cqdd = stage_or_zero(tile + (mv.nq + mv.nv) * T, qdd, mv.nv, B, e, act);
  const Col ctm = stage_or_zero(tile + (mv.nq + 2 * mv.nv) * T, tau_meas, mv.nv, B, e, act);
  float* slots = theta_slots(smem, mv.n, rows);
  const int P = mv.n * 10 + 1;
  zero_slots(slots, (T / 32) * P);
  const SmemModel sm = stage_model(mv, smem);
  cp_async_wait_all();
  const SV a0 = world_accel(mv);
  Xf X[NB];
  SV v[NB], a[NB], F[NB];
  rnea_forward<NB>(sm, a0, cq, cqd, cqdd, X, v, a, F);
  rnea_backward<NB>(sm, X, F, nullptr, B, e);
  // residual r = tau - tau_meas, overwriting tau_meas's column with taubar = 2 r
  float* tb = tile + (mv.nq + 2 * mv.nv) * T + threadIdx.x;
  float loss = 0.f;
  FST_UNROLL
  for (int i = 0; i < sm.n(); ++i) {
    const BodyI bi = sm.I(i);
    const int nvi = nv_of(bi.type);
    if (nvi == 0) continue;
    float tau6[6];
    if (nvi == 1) {
      tau6[0] = dot(S_of(sm.C(i)), F[i]);
    } else {
      tau6[0] = F[i].v.x; tau6[1] = F[i].v.y; tau6[2] = F[i].v.z;
      tau6[3] = F[i].w.x; tau6[4] = F[i].w.y; tau6[5] = F[i].w.z;
    }
    for (int r = 0; r < nvi; ++r) {
      const float res = tau6[r] - tb[(bi.vi + r) * T];
      loss = fmaf(res, res, loss);
      tb[(bi.vi + r) * T] = 2.f * res;
    }
  }
  float* wslot = slots + (threadIdx.x / 32) * P;
  float lg = act ? loss : 0.f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, off);
  if ((threadIdx.x & 31) == 0) wslot[P - 1] += lg;
  VjpOut o{qbar, qdbar, nullptr, wslot, 1.f, act};
  rnea_vjp_reverse<NB>(sm, a0, cq, cqd, X, v, a, F, Col{tb, T}, o, B, e);
  __syncthreads();
  write_partial(slots, P, partial);
}

template <int NB>
__global__ void __launch_bounds__(256) fk_vjp_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                     const float* __restrict__ pbar, float* __restrict__ qbar) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  Col cq{}, cpb{};
  if (act) {
    cq = stage_rows(tile, q, mv.nq, B, e);
    cpb = stage_rows(tile + mv.nq * T, pbar, mv.n * 12, B, e);
  }
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  fk_vjp_env<NB>(sm, cq, cpb, qbar, B, e);
}

// Jacobian adjoint: Jbar [n_links][6][nv][B] -> q_bar.
template <int NB>
__global__ void __launch_bounds__(256) jac_vjp_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                      LinkList links, const float* __restrict__ Jbar,
                                                      float* __restrict__ qbar) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  Col cq{};
  if (act) cq = stage_rows(tile, q, mv.nq, B, e);
  const SmemModel sm = stage_model(mv, smem);
  if (!act) return;
  cp_async_wait_all();
  jac_vjp_env<NB>(sm, cq, mv.nv, links, Jbar, qbar, B, e);
}

// Mass-matrix adjoint. M e_k = RNEA(q, 0, e_k) without gravity, so for
// L = sum_rc Mbar_rc M_rc the cotangents are the sum over columns k of the
// RNEA adjoint at (q, qd = 0, qdd = e_k, no gravity) with taubar = Mbar[:, k];
// q_bar accumulates in place, thetabar in the per-warp slots.
template <int NB>
__global__ void __launch_bounds__(256) crba_vjp_kernel(ModelView mv, int64_t B, const float* __restrict__ q,
                                                       const float* __restrict__ Mbar, float* qbar, float* partial) {
  extern __shared__ float4 smem[];
  const int T = blockDim.x;
  const int rows = mv.nq + 3 * mv.nv;
  const int nv = mv.nv;
  float* tile = smem_tile(smem, mv.n);
  const int64_t e = (int64_t)blockIdx.x * T + threadIdx.x;
  const bool act = e < B;
  const Col cq = stage_or_zero(tile, q, mv.nq, B, e, act);
  float* zc = tile + mv.nq * T + threadIdx.x;  // qd = 0
  float* uc = zc + nv * T;                      // qdd = e_k
  float* tc = uc + nv * T;                      // taubar = Mbar[:, k]
  for (int k = 0; k < nv; ++k) {
    zc[k * T] = 0.f;
    uc[k * T] = 0.f;
  }
  float* slots = partial ? theta_slots(smem, mv.n, rows) : nullptr;
  const int P = mv.n * 10;
  if (slots) zero_slots(slots, (T / 32) * P);
  const SmemModel sm = stage_model(mv, smem);
  cp_async_wait_all();
  for (int k = 0; k < nv; ++k) {
    uc[k * T] = 1.f;
    if (k > 0) uc[(k - 1) * T] = 0.f;
    for (int i = 0; i < nv; ++i) tc[i * T] = act ? __ldg(Mbar + ((int64_t)i * nv + k) * B + e) : 0.f;
    VjpOut o{qbar, nullptr, nullptr, slots ? slots + (threadIdx.x / 32) * P : nullptr, 1.f, act, k > 0};
    rnea_vjp_env<NB>(sm, sv_zero(), cq, Col{zc, T}, Col{uc, T}, Col{tc, T}, o, B, e);
  }
  if (partial) {
    __syncthreads();
    write_partial(slots, P, partial);
  }
}

// out[p] = sum over blocks b (in order) of partial[b * P + p]
__global__ void partial_reduce_kernel(const float* __restrict__ partial, int nblk, int P, float* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * P + p];
  out[p] = s;
}

// Largest power-of-two block (<= the default, >= 32) whose shared memory
// stays under 96 KB, so big trees keep several blocks per SM.
int fit_block(int64_t B, int n, int rows, bool theta) {
  int T = default_block(B);
  while (T > 32 && vjp_smem(n, rows, T, theta) > 96 * 1024) T /= 2;
  return T;
}

cudaError_t reduce(const float* partial, int nblk, int P, float* out, cudaStream_t s) {
  partial_reduce_kernel<<<(P + 127) / 128, 128, 0, s>>>(partial, nblk, P, out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_partial_reduce(const float* partial, int nblk, int P, float* out, cudaStream_t s) {
  return reduce(partial, nblk, P, out, s);
}

size_t vjp_scratch_floats(int n, int64_t B) { return (size_t)((B + 31) / 32) * (n * 10 + 1); }

cudaError_t launch_rnea_vjp(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                            const float* tbar, float* qbar, float* qdbar, float* qddbar, float* thbar, float* scratch,
                            cudaStream_t s) {
  const int rows = mv.nq + 3 * mv.nv;
  const int T = fit_block(B, mv.n, rows, thbar != nullptr);
  const size_t sh = vjp_smem(mv.n, rows, T, thbar != nullptr);
  float* partial = thbar ? scratch : nullptr;
  FST_NB_DISPATCH(mv.n, prepare(rnea_vjp_kernel<NB>, sh);
                  rnea_vjp_kernel<NB><<<grid_for(B, T), T, sh, s>>>(mv, B, q, qd, qdd, tbar, qbar, qdbar, qddbar, partial));
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess && thbar) err = reduce(partial, (int)grid_for(B, T), mv.n * 10, thbar, s);
  return err;
}

cudaError_t launch_rnea_store(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                              float* tau, float* tape, const Launch& L) {
  const size_t sh = smem_bytes(mv.n, mv.nq + 2 * mv.nv, L.block);
  FST_NB_DISPATCH(mv.n, prepare(rnea_store_kernel<NB>, sh);
                  rnea_store_kernel<NB><<<grid_for(B, L.block), L.block, sh, L.stream>>>(mv, B, q, qd, qdd, tau, tape));
  return cudaGetLastError();
}

cudaError_t launch_rnea_vjp_stored(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* tape,
                                   const float* tbar, float* qbar, float* qdbar, float* qddbar, float* thbar,
                                   float* scratch, cudaStream_t s) {
  const int rows = mv.nq + 2 * mv.nv;
  const int T = fit_block(B, mv.n, rows, thbar != nullptr);
  const size_t sh = vjp_smem(mv.n, rows, T, thbar != nullptr);
  float* partial = thbar ? scratch : nullptr;
  FST_NB_DISPATCH(mv.n, prepare(rnea_vjp_stored_kernel<NB>, sh);
                  rnea_vjp_stored_kernel<NB><<<grid_for(B, T), T, sh, s>>>(mv, B, q, qd, tape, tbar, qbar, qdbar,
                                                                           qddbar, partial));
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess && thbar) err = reduce(partial, (int)grid_for(B, T), mv.n * 10, thbar, s);
  return err;
}

cudaError_t launch_aba_vjp(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                           const float* qddbar, float* qbar, float* qdbar, float* taubar, float* thbar, float* scratch,
                           cudaStream_t s) {
  const int rows = mv.nq + 4 * mv.nv;
  const int T = fit_block(B, mv.n, rows, thbar != nullptr);
  const size_t sh = vjp_smem(mv.n, rows, T, thbar != nullptr);
  float* partial = thbar ? scratch : nullptr;
  FST_NB_DISPATCH(mv.n, prepare(aba_vjp_kernel<NB>, sh);
                  aba_vjp_kernel<NB><<<grid_for(B, T), T, sh, s>>>(mv, B, q, qd, qdd, qddbar, qbar, qdbar, taubar, partial));
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess && thbar) err = reduce(partial, (int)grid_for(B, T), mv.n * 10, thbar, s);
  return err;
}

cudaError_t launch_rnea_loss_grad(const ModelView& mv, int64_t B, const float* q, const float* qd, const float* qdd,
                                  const float* tau_meas, float* loss_theta, float* qbar, float* qdbar, float* scratch,
                                  cudaStream_t s) {
  const int rows = mv.nq + 3 * mv.nv;
  int T = default_block(B);
  auto smem_of = [&](int t) { return smem_bytes(mv.n, rows, t) + (size_t)(t / 32) * (mv.n * 10 + 1) * sizeof(float); };
  while (T > 32 && smem_of(T) > 96 * 1024) T /= 2;
  const size_t sh = smem_of(T);
  FST_NB_DISPATCH(mv.n, prepare(rnea_loss_grad_kernel<NB>, sh);
                  rnea_loss_grad_kernel<NB><<<grid_for(B, T), T, sh, s>>>(mv, B, q, qd, qdd, tau_meas, qbar, qdbar, scratch));
  cudaError_t err = cudaGetLastError();
  // loss_theta: [n*10] theta gradient followed by the loss
  if (err == cudaSuccess) err = reduce(scratch, (int)grid_for(B, T), mv.n * 10 + 1, loss_theta, s);
  return err;
}

cudaError_t launch_jac_vjp(const ModelView& mv, int64_t B, const float* q, const LinkList& links, const float* Jbar,
                           float* qbar, cudaStream_t s) {
  const int T = fit_block(B, mv.n, mv.nq, false);
  const size_t sh = smem_bytes(mv.n, mv.nq, T);
  FST_NB_DISPATCH(mv.n, prepare(jac_vjp_kernel<NB>, sh);
                  jac_vjp_kernel<NB><<<grid_for(B, T), T, sh, s>>>(mv, B, q, links, Jbar, qbar));
  return cudaGetLastError();
}

cudaError_t launch_crba_vjp(const ModelView& mv, int64_t B, const float* q, const float* Mbar, float* qbar,
                            float* thbar, float* scratch, cudaStream_t s) {
  const int rows = mv.nq + 3 * mv.nv;
  const int T = fit_block(B, mv.n, rows, thbar != nullptr);
  const size_t sh = vjp_smem(mv.n, rows, T, thbar != nullptr);
  float* partial = thbar ? scratch : nullptr;
  FST_NB_DISPATCH(mv.n, prepare(crba_vjp_kernel<NB>, sh);
                  crba_vjp_kernel<NB><<<grid_for(B, T), T, sh, s>>>(mv, B, q, Mbar, qbar, partial));
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess && thbar) err = reduce(partial, (int)grid_for(B, T), mv.n * 10, thbar, s);
  return err;
}

cudaError_t launch_fk_vjp(const ModelView& mv, int64_t B, const float* q, const float* pbar, float* qbar,
                          cudaStream_t s) {
  const int rows = mv.nq + 12 * mv.n;
  const int T = fit_block(B, mv.n, rows, false);
  const size_t sh = smem_bytes(mv.n, rows, T);
  FST_NB_DISPATCH(mv.n, prepare(fk_vjp_kernel<NB>, sh);
                  fk_vjp_kernel<NB><<<grid_for(B, T), T, sh, s>>>(mv, B, q, pbar, qbar));
  return cudaGetLastError();
}

}  // namespace fst
