/*
 * fst.h - batched Featherstone rigid-body dynamics on GB300 (sm_103a).
 *
 * C ABI of libfst.so. One kinematic tree (the "model") is shared by B
 * independent environments; every operator evaluates all B environments in
 * one call. The operators are those of the paper "Batched Differentiable
 * Rigid Body Dynamics in PyTorch for GPU-Accelerated Robot Learning":
 * forward kinematics (Sec. 3.1 tier 3), the geometric Jacobian (Sec. 3.4,
 * Eq. 6), RNEA (Sec. 3.3, Eq. 7), CRBA and ABA (Sec. 3.5, Sec. 4.1), plus
 * hand-written adjoints of FK, the Jacobian, RNEA, CRBA and ABA (the paper
 * differentiates by autograd, Sec. 3.5 and Sec. 4.3), dense derivatives of
 * inverse and forward dynamics, and a persistent launch over several trees.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Arrays are FP32, caller-owned DEVICE memory on the model's device, in
 *   structure-of-arrays layout with the environment index fastest:
 *   element (field f, env e) lives at ptr[f * B + e]. So q is [nq][B],
 *   qd/qdd/tau are [nv][B].
 * - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are
 *   asynchronous on it; none allocates, frees or synchronises, so every
 *   compute call can be captured into a CUDA graph.
 * - B = 0 is valid and does nothing. B < 0, B > 2^31 - 1, null pointers
 *   with B > 0, or a call from a device other than the model's return
 *   FST_ERR_INVALID_ARG without launching anything.
 * - A failed kernel launch returns FST_ERR_CUDA. Nothing traps on the
 *   device. NaN/Inf inputs give NaN/Inf outputs for that environment only.
 * - On any status other than FST_OK, fst_last_error() gives a message
 *   (thread-local, valid until the next call on the same thread).
 *
 * Joint model (paper Sec. 3.2, first equation): the pose of body i in its
 * parent is T_joint[i] * J(q_i) * T_link[i], with J a rotation about `axis`
 * (revolute, 1 DOF), a translation along `axis` (prismatic, 1 DOF), the
 * identity (fixed, 0 DOF) or a free rigid motion (free, body 0 only,
 * q = [x y z qx qy qz qw], velocity = twist of the body frame in its own
 * coordinates, linear part first [v; w], 6 DOF; T_link must be identity).
 * q-index and v-index of each body are the running sums of its
 * predecessors' nq and nv, in body order.
 */
#ifndef FST_H
#define FST_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FST_API __attribute__((visibility("default")))
#else
#define FST_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FST_OK = 0,
  FST_ERR_INVALID_ARG = -1,  /* bad pointer, size, device or option */
  FST_ERR_TOPOLOGY = -2,     /* parent index not in [-1, i-1], misplaced free joint */
  FST_ERR_INERTIA = -3,      /* negative mass, non-PSD or non-finite inertia */
  FST_ERR_UNSUPPORTED = -4,  /* joint type or model size this build does not handle */
  FST_ERR_CUDA = -5,         /* a CUDA runtime call or kernel launch failed */
  FST_ERR_NO_MEMORY = -6,    /* device allocation at model creation failed */
  FST_ERR_DEVICE_CHECK = -7  /* reserved: no entry point returns it (every check runs on the host) */
} fst_status;

enum {
  FST_JOINT_FIXED = 0,
  FST_JOINT_REVOLUTE = 1,
  FST_JOINT_PRISMATIC = 2,
  FST_JOINT_FREE = 3
};

/* Largest model this build accepts (bodies). */
#define FST_MAX_BODIES 64
/* Largest number of end-effector links per Jacobian call. */
#define FST_MAX_LINKS 16

/* One row of the body table (host memory, FP64). Bodies are listed in
 * topological order: parent < own index, -1 = attached to the world. */
typedef struct fst_body_desc {
  int32_t parent;
  int32_t type;          /* FST_JOINT_* */
  double axis[3];        /* joint axis in the joint frame; normalised by create */
  double T_joint[12];    /* parent -> joint frame: R row-major (9), then t (3) */
  double T_link[12];     /* joint (moved) -> body frame; identity if unused */
  double mass;           /* kg */
  double com[3];         /* centre of mass in the body frame */
  double I_com[6];       /* rotational inertia about the COM, body frame: xx xy yy xz yz zz */
} fst_body_desc;

typedef struct fst_model fst_model;

/* Builds a model from the body table (host memory, not retained) and
 * uploads its constants to the CURRENT CUDA device: the Rodrigues constants
 * of paper Eq. 2-3 per joint, each body's motion subspace and its inertia as
 * the 10 linear parameters about the body origin. gravity[3] is the world
 * gravity vector (e.g. {0, 0, -9.81}). On success *out owns device memory;
 * release it with fst_model_destroy. Validation happens before any CUDA
 * call, so FST_ERR_TOPOLOGY / FST_ERR_INERTIA / FST_ERR_UNSUPPORTED /
 * FST_ERR_INVALID_ARG are returned on hosts without a GPU as well. */
FST_API fst_status fst_model_create(const fst_body_desc* bodies, int32_t n_bodies,
                            const double gravity[3], fst_model** out);

/* Frees the model's device memory (and its specialised kernels). NULL is
 * accepted. Model life cycle: no counterpart in the paper. */
FST_API fst_status fst_model_destroy(fst_model* model);

/* Sizes of a model: configuration dimension nq, velocity dimension nv,
 * number of bodies and tree depth (bodies on the longest root-leaf path:
 * the number of level steps of the level-parallel sweeps, Sec. 3.3).
 * Any output pointer may be NULL; a NULL model returns FST_ERR_INVALID_ARG. */
FST_API fst_status fst_model_info(const fst_model* model, int32_t* nq, int32_t* nv,
                          int32_t* n_bodies, int32_t* depth);

/* The model's own inertial parameters, theta layout of fst_rnea (about each
 * body origin), copied to HOST memory theta[n_b * 10] (FP32): the
 * parameters that the identification of Sec. 4.3 estimates (the paper
 * fixes no layout for them). Synchronous; FST_ERR_INVALID_ARG for NULL. */
FST_API fst_status fst_model_theta(const fst_model* model, float* theta);

/* Kernel kinds for fst_model_specialize (bit masks; 0 = all). */
#define FST_SPEC_FK (1u << 0)
#define FST_SPEC_JACOBIAN (1u << 1)
#define FST_SPEC_RNEA (1u << 2)
#define FST_SPEC_CRBA (1u << 3)
#define FST_SPEC_ABA (1u << 4)
#define FST_SPEC_EVAL (1u << 5)
#define FST_SPEC_FK_VJP (1u << 6)
#define FST_SPEC_RNEA_VJP (1u << 7)
#define FST_SPEC_ABA_VJP (1u << 8)
#define FST_SPEC_LOSS_GRAD (1u << 9)
#define FST_SPEC_EVAL_MIXED (1u << 10) /* the fused kernel of FST_VARIANT_MIXED */
#define FST_SPEC_RNEA_STORE (1u << 11)
#define FST_SPEC_RNEA_VJP_STORED (1u << 12)
#define FST_SPEC_RNEA_DERIVATIVES (1u << 13)
#define FST_SPEC_ABA_DERIVATIVES (1u << 14)
#define FST_SPEC_ALL 0x7fffu

/* Compiles kernels specialised for this model's tree (run-time compilation
 * with NVRTC for the current GPU). The paper folds the fixed joint offsets
 * into precomputed constants at build time (Sec. 3.2); this goes one step
 * further and bakes the whole tree into the kernel: the topology becomes a
 * compile-time constant, every body loop is unrolled and the sweep state
 * stays in registers. Afterwards, calls of the selected kinds on this model
 * run the specialised kernels (same results within FP32 rounding; the
 * inertial parameters, including a theta override, are still read at run
 * time). Synchronous: about a second per kind on first use; compiled code
 * is cached on disk ($FST_JIT_CACHE, default ~/.cache/fst_jit). Call it
 * before capturing a stream. Returns FST_ERR_UNSUPPORTED (and changes
 * nothing) when NVRTC or the CUDA driver entry points are unavailable; the
 * generic kernels keep serving every call. */
FST_API fst_status fst_model_specialize(fst_model* model, uint32_t kinds);

/* Launch configuration of the selected kinds (FST_SPEC_* mask, 0 = all) on
 * this model: threads per block (32, 64, 128 or 256; 0 = built-in heuristic)
 * and which kernel variant runs:
 *   AUTO        the specialised kernel when compiled, else the generic one;
 *   GENERIC     one environment per thread, tree from shared memory;
 *   SPECIALIZED one environment per thread, kernel compiled for this tree;
 *   LEVEL       level-parallel (paper Sec. 3.3 on warps): 32 environments per
 *               block, the block's block/32 warps split the bodies of each
 *               tree level, per-body state in shared memory; FK, Jacobian,
 *               RNEA, CRBA, ABA and eval only (a 0 mask then selects those
 *               six), and only while that state fits
 *               in shared memory (about 28 bodies for ABA); otherwise the
 *               generic kernel runs;
 *   MIXED, PATH, PATH_WARP, PINNED: see each below. A 0 mask with PATH or
 *               PATH_WARP selects the six kinds above; with PINNED, eval
 *               and ABA.
 * Results agree within FP32 rounding; only speed changes. SPECIALIZED for a
 * kind that fst_model_specialize has not compiled returns
 * FST_ERR_INVALID_ARG. The autotuner in the Python package measures the
 * candidates per kind and batch size and sets the fastest. */
#define FST_VARIANT_AUTO 0
#define FST_VARIANT_GENERIC 1
#define FST_VARIANT_SPECIALIZED 2
#define FST_VARIANT_LEVEL 3
/* eval only: the specialised fused kernel, with each role (ABA, CRBA, RNEA,
 * FK/Jacobian) level-parallel (one tile of 32 environments per block) where
 * that operator's own kind is set to LEVEL, LEVEL2 or LEVEL_LEAN and one
 * environment per thread otherwise. A level-parallel role runs on a
 * copy of the model staged in shared memory, as the operator's own
 * level-parallel kernel does (compact per-level loops rather than the
 * compiled-in tree unrolled into every warp's instructions). */
#define FST_VARIANT_MIXED 4
/* FK, Jacobian, RNEA, CRBA, ABA and eval of a specialised model: the
 * path-parallel mapping. Every root-to-leaf path of the tree gets its own
 * lane (G = the number of paths rounded up to a power of two, at most 8
 * lanes per environment, 32 / G environments per warp); a lane sweeps its
 * path with the sweep state in registers, bodies shared by several paths
 * are computed by each of them, and the leaf-to-root sums over a body's
 * children are warp shuffles. The serial chain per environment is the tree
 * depth instead of the body count. Needs fst_model_specialize of the kind;
 * trees with more than 8 leaves have no path-parallel kernels. */
#define FST_VARIANT_PATH 5
/* The same sweeps with a warp per path: blocks of 32 environments (one per
 * lane) and one warp per root-to-leaf path, each warp running code compiled
 * for its own path; the paths meet through shared memory, with one block
 * barrier per depth where paths join. The block size is fixed by the tree
 * (32 x number of paths); the block argument is ignored. */
#define FST_VARIANT_PATH_WARP 6
/* eval (specialised) and ABA (level-parallel): SM-pinned launches. Each SM
 * serves the role the table of fst_model_set_sm_roles gives it, so an SM
 * keeps running the same code from call to call (its instruction caches stay
 * warm). Blocks pull tiles of environments from per-call counters; blocks on
 * SMs without a matching role leave at once, and the block that finishes
 * last completes whatever is left, so results never depend on where the
 * hardware placed the blocks. For eval this is one launch of one block per
 * SM for every requested operator, ABA included (level-parallel, two tiles
 * of 32 environments at a time; the others one environment per thread, as
 * many tiles as the role has SMs); the block argument is ignored, and trees
 * whose two ABA tiles do not fit in shared memory are refused. Calls of one
 * model with this variant must not overlap in time, except one eval beside
 * one ABA (they count in separate regions). */
#define FST_VARIANT_PINNED 7
/* As LEVEL, with two tiles of 32 environments per block (block >= 64
 * threads, split evenly; the tiles' warps interleaved so that each tile's
 * busiest warp has an SM sub-partition of its own): half as many blocks,
 * each twice the shared memory. For trees whose per-tile state fits twice
 * in shared memory; otherwise the generic kernel runs. */
#define FST_VARIANT_LEVEL2 8
/* The level-parallel CRBA and ABA with less shared memory per tile, so that
 * more tiles of a large tree fit on one SM (FST_VARIANT_LEVEL_LEAN; CRBA and
 * ABA only; "all kinds" means those two). ABA: per body 14 floats per
 * environment (v, then U, then a; c; 1/D; u) instead of 59; each body's
 * contribution to its parent (X^T I^a X, X^T p^a: 27 floats) sits in a
 * ring of two levels' slots only until the parent reads it; the joint
 * transforms are recomputed in passes 2 and 3. CRBA: per body X and
 * F = I^c S (18 floats) instead of 32, the composite-inertia contributions
 * in the same kind of ring, q read from global memory instead of staged.
 * Same recursions (Sec. 3.3 level-parallel form); results agree with
 * FST_VARIANT_LEVEL within FP32 rounding. Where even the lean tile does not
 * fit in shared memory, the generic kernel runs. */
#define FST_VARIANT_LEVEL_LEAN 9
FST_API fst_status fst_model_set_launch(fst_model* model, uint32_t kinds, int32_t block, int32_t variant);

/* SM partitions (CUDA green contexts): disjoint sets of a device's SMs, each
 * with a stream whose kernels run only on its SMs, also when the launches
 * are captured into a CUDA graph from another stream that forks into them.
 * The operators of one step launched on separate partitions run side by
 * side without sharing an SM, so no SM refetches another operator's
 * instructions between launches (the level-parallel propagation of
 * Sec. 3.3 and the fused launch of the others, as concurrent branches).
 *
 * fst_sm_partition_create: device = CUDA ordinal; sm_counts = HOST array of
 * n (1 <= n <= FST_MAX_PARTITIONS) positive SM counts, each rounded up to
 * whole groups of 8 SMs; their sum must fit the device. *out receives the
 * handle (owned by the caller; release with fst_sm_partition_destroy, after
 * every launch and graph that uses its streams has finished).
 * FST_ERR_UNSUPPORTED when the driver has no green contexts,
 * FST_ERR_INVALID_ARG for bad counts or device, FST_ERR_CUDA when a green
 * context or stream cannot be created. Synchronous.
 * fst_sm_partition_info: partition k's stream (a CUstream / cudaStream_t,
 * owned by the partition) and its actual SM count; either output may be
 * NULL. */
#define FST_MAX_PARTITIONS 8
typedef struct fst_sm_partition fst_sm_partition;
FST_API fst_status fst_sm_partition_create(int32_t device, const int32_t* sm_counts, int32_t n,
                                           fst_sm_partition** out);
FST_API fst_status fst_sm_partition_info(const fst_sm_partition* p, int32_t k, void** stream, int32_t* sm_count);
FST_API fst_status fst_sm_partition_destroy(fst_sm_partition* p);

/* Roles of the SMs for FST_VARIANT_PINNED launches: role_of_sm[i] is the
 * role of SM id i (FST_ROLE_*, or FST_ROLE_NONE), for n <= 256 SM ids; ids
 * past n get FST_ROLE_NONE. The ids are the hardware's (fst_sm_ids lists
 * those that exist); the first call also probes them for the pinned step. The roles are the operator groups of fst_eval:
 * ABA, CRBA, RNEA and KIN (FK with the Jacobians). Synchronous (copies the
 * table to the model's device memory): call it before capturing a stream.
 * Until it is called every SM has no role, which is correct but slow (the
 * last block does all the work). */
#define FST_ROLE_NONE (-1)
#define FST_ROLE_ABA 0
#define FST_ROLE_CRBA 1
#define FST_ROLE_RNEA 2
#define FST_ROLE_KIN 3
FST_API fst_status fst_model_set_sm_roles(fst_model* model, const int32_t* role_of_sm, int32_t n);

/* Launch control (no counterpart in the paper). Shared-memory carveout (percent of the unified L1/shared storage given to
 * shared memory) requested for every kernel launched from now on; -1 (the
 * default) lets each kernel ask for what suits it alone. Kernels only share
 * an SM when they ask for the same carveout, so overlapping different
 * kernels on parallel streams (the step plan's concurrent modes) wants one
 * common value. Process-wide. */
FST_API fst_status fst_set_smem_carveout(int32_t percent);

/* Bit mask (FST_SPEC_*) of the specialised kinds currently in use for this
 * model, written to *kinds (host). A launch control with no counterpart in
 * the paper; FST_ERR_INVALID_ARG for NULL arguments. */
FST_API fst_status fst_model_specialized(const fst_model* model, uint32_t* kinds);

/* Forward kinematics (paper Sec. 3.1, tier 3; Eq. 4-5 for each joint).
 * q      [nq][B]        joint positions.
 * poses  [n_b][12][B]   world pose of every body: R row-major (9), then p (3). */
FST_API fst_status fst_fk(const fst_model* model, int64_t B, const float* q,
                  float* poses, void* stream);

/* Geometric Jacobians (paper Sec. 3.4, Eq. 6) of n_links bodies.
 * links   HOST array of n_links body indices (1 <= n_links <= FST_MAX_LINKS).
 * J       [n_links][6][nv][B]: world-frame twist at the world origin, rows
 *         [v; w] (linear first); column k is the twist produced by unit
 *         velocity of DOF k; DOFs not on the body's support path are 0. */
FST_API fst_status fst_jacobian(const fst_model* model, int64_t B, const float* q,
                        const int32_t* links, int32_t n_links, float* J,
                        void* stream);

/* Inverse dynamics by recursive Newton-Euler (paper Sec. 3.3, Eq. 7):
 * tau = M(q) qdd + C(q, qd) qd + g(q).
 * theta  [n_b][10] device, or NULL for the model's own inertias:
 *        per body [m, m*cx, m*cy, m*cz, Ixx, Ixy, Iyy, Ixz, Iyz, Izz] with
 *        the rotational inertia about the BODY-FRAME ORIGIN. Shared by all
 *        environments. */
FST_API fst_status fst_rnea(const fst_model* model, int64_t B, const float* q,
                    const float* qd, const float* qdd, const float* theta,
                    float* tau, void* stream);

/* Joint-space mass matrix by the composite-rigid-body algorithm (paper
 * Sec. 3.5). M [nv][nv][B], full symmetric (both triangles written). */
FST_API fst_status fst_crba(const fst_model* model, int64_t B, const float* q,
                    const float* theta, float* M, void* stream);

/* Forward dynamics by the articulated-body algorithm (paper Sec. 4.1, three
 * passes): qdd = M(q)^-1 (tau - C(q, qd) qd - g(q)). */
FST_API fst_status fst_aba(const fst_model* model, int64_t B, const float* q,
                   const float* qd, const float* tau, const float* theta,
                   float* qdd, void* stream);

/* fst_eval_io.flags */
#define FST_EVAL_ONE_SWEEP 1u  /* poses and J come from the RNEA sweep's own joint transforms */
#define FST_EVAL_PACKED 2u     /* M and J in the packed layouts of fst_packed_layout */

/* Inputs and outputs of fst_eval. Inputs: q always; qd and qdd when tau_out
 * or an RNEA cotangent is requested; qd and tau when qdd_out is requested.
 * Outputs: any subset, NULL = not computed. links/n_links (HOST array) are
 * used when J is set. Zero-initialise the struct: fields added later are
 * then off. */
typedef struct fst_eval_io {
  const float* q;        /* [nq][B] */
  const float* qd;       /* [nv][B] */
  const float* qdd;      /* [nv][B] */
  const float* tau;      /* [nv][B] */
  float* poses;          /* [n_b][12][B]        as fst_fk */
  float* J;              /* [n_links][6][nv][B] as fst_jacobian */
  const int32_t* links;
  int32_t n_links;
  float* tau_out;        /* [nv][B]             as fst_rnea (inputs q, qd, qdd) */
  float* M;              /* [nv][nv][B]         as fst_crba */
  float* qdd_out;        /* [nv][B]             as fst_aba (inputs q, qd, tau) */
  /* The RNEA adjoint in the same pass (as fst_rnea_vjp without theta_bar):
   * set any of q_bar / qd_bar / qdd_bar to request it; tau_bar [nv][B] is
   * then its cotangent, or the computed tau itself when tau_bar == tau_out
   * (e.g. for the loss |tau|^2 / 2). */
  const float* tau_bar;
  float* q_bar;          /* [nq][B] */
  float* qd_bar;         /* [nv][B] */
  float* qdd_bar;        /* [nv][B] */
  uint32_t flags;        /* FST_EVAL_* */
} fst_eval_io;

/* Sizes of the packed outputs of fst_eval (FST_EVAL_PACKED), which drop
 * what the full layouts repeat or know to be zero, so that less has to be
 * copied off the device:
 *  - M: its upper triangle, row by row: element (r, c), r <= c, is row
 *    r*nv - r*(r-1)/2 + (c - r) of an [nv*(nv+1)/2][B] array;
 *  - J: for each link l, only the columns of the DOFs on its support path
 *    (the joints between it and the root; every other column is zero), in
 *    DOF order, as a [6][cols[l]] block; the blocks follow each other in
 *    link order in one [j_rows][B] array, j_rows = 6 * sum of cols.
 * Host only (no device work). cols (n_links entries), j_rows and m_rows may
 * be NULL. The paper has no counterpart: it returns dense tensors. */
FST_API fst_status fst_packed_layout(const fst_model* model, const int32_t* links, int32_t n_links,
                                     int32_t* cols, int32_t* j_rows, int32_t* m_rows);

/* Every requested operator of one batch in ONE launch. The paper computes
 * only the kinematic tiers a query needs (Sec. 3.1); here the operators
 * whose outputs are NULL are skipped and the others run side by side on the
 * GPU, one group of thread blocks per operator. Results are bit-identical
 * to the per-operator calls. theta as in fst_rnea.
 * With an RNEA cotangent requested, the RNEA operator's blocks run its
 * forward sweep once and feed tau and the adjoint's reverse sweeps from it
 * (the controller step of the paper's RL experiment, Sec. 4.4: FK,
 * Jacobians and inverse dynamics, here with RNEA's gradient). With
 * FST_EVAL_ONE_SWEEP and the RNEA operator requested, poses and J are also
 * computed by those blocks from the same joint transforms (paper Eq. 4-5
 * evaluated once per joint) instead of by blocks of their own. Both run the
 * one-environment-per-thread fused kernel: the one specialised for the tree
 * when it is compiled (FST_SPEC_EVAL) and the eval kind is not set to
 * FST_VARIANT_GENERIC, else the generic one. FST_EVAL_PACKED writes M and J
 * in the layouts of fst_packed_layout (M then has nv*(nv+1)/2 rows), on the
 * same kernels; values are bit-identical to the full layouts' entries. */
FST_API fst_status fst_eval(const fst_model* model, int64_t B, const fst_eval_io* io,
                            const float* theta, void* stream);

/* ---------------------------------------------------------------------------
 * Adjoints (vector-Jacobian products). The paper obtains gradients with
 * autograd (Sec. 3.5) and identifies link masses through the RNEA gradient
 * (Sec. 4.3); these entry points compute the same products with hand-written
 * reverse sweeps. Any output pointer may be NULL (that cotangent is not
 * computed). theta_bar is [n_b][10] in the theta layout of fst_rnea, summed
 * over all B environments and OVERWRITTEN (not accumulated); it is reduced
 * deterministically (no floating-point atomics), so repeated calls give
 * bit-identical results. Computing theta_bar needs caller-allocated device
 * scratch of fst_adjoint_scratch_bytes() bytes; scratch may be NULL when
 * theta_bar is NULL. Too small a scratch returns FST_ERR_INVALID_ARG.
 * The free joint's q_bar is the gradient with respect to the 7 raw
 * coordinates [x y z qx qy qz qw] (through the quaternion normalisation).
 * ------------------------------------------------------------------------- */

/* Device scratch bytes the adjoints need for theta_bar over B environments
 * (the per-block partial sums of the deterministic reduction), written to
 * *bytes (host). Workspace sizing for the gradients of Sec. 4.3. */
FST_API fst_status fst_adjoint_scratch_bytes(const fst_model* model, int64_t B, size_t* bytes);

/* FK (Sec. 3.1, Eq. 4-5): q_bar [nq][B] = (d poses / d q)^T poses_bar,
 * poses_bar [n_b][12][B] in the layout of fst_fk. */
FST_API fst_status fst_fk_vjp(const fst_model* model, int64_t B, const float* q,
                              const float* poses_bar, float* q_bar, void* stream);

/* RNEA (Sec. 3.3; its theta-gradient drives the identification of
 * Sec. 4.3): cotangents of tau = RNEA(q, qd, qdd; theta) for tau_bar
 * [nv][B]: q_bar [nq][B], qd_bar [nv][B], qdd_bar [nv][B] (= M tau_bar),
 * theta_bar. */
FST_API fst_status fst_rnea_vjp(const fst_model* model, int64_t B, const float* q,
                                const float* qd, const float* qdd, const float* theta,
                                const float* tau_bar, float* q_bar, float* qd_bar,
                                float* qdd_bar, float* theta_bar, void* scratch,
                                size_t scratch_bytes, void* stream);

/* Jacobian (Sec. 3.4, Eq. 6): q_bar [nq][B] = sum (d J / d q)^T J_bar for J_bar
 * [n_links][6][nv][B] in the layout of fst_jacobian (the same links).
 * q_bar is required. */
FST_API fst_status fst_jacobian_vjp(const fst_model* model, int64_t B, const float* q,
                                    const int32_t* links, int32_t n_links, const float* J_bar,
                                    float* q_bar, void* stream);

/* Mass matrix (the CRBA of Sec. 3.5): cotangents of M = CRBA(q; theta) for M_bar [nv][nv][B]:
 * q_bar [nq][B] (may be NULL) and theta_bar (may be NULL; needs scratch as
 * for fst_rnea_vjp). Uses M e_k = RNEA(q, 0, e_k) without gravity: the sum
 * over columns k of RNEA adjoints with tau_bar = M_bar[:, k]. */
FST_API fst_status fst_crba_vjp(const fst_model* model, int64_t B, const float* q, const float* theta,
                                const float* M_bar, float* q_bar, float* theta_bar, void* scratch,
                                size_t scratch_bytes, void* stream);

/* Store variant of the RNEA adjoint. The paper differentiates through an
 * autograd tape that keeps every intermediate (Sec. 3.5); fst_rnea_vjp
 * instead recomputes the forward sweep inside the adjoint kernel. These
 * three calls keep the choice open: fst_rnea_store runs RNEA (tau optional,
 * may be NULL) and writes the forward state the reverse sweeps read, per
 * body and environment 30 floats: the joint transform (R row-major 9, t 3),
 * the spatial velocity and acceleration ([w; v] each) and the accumulated
 * force ([n; f]), as tape [n_b][30][B] in caller-owned device memory of
 * fst_rnea_tape_bytes() bytes (tape_bytes smaller returns
 * FST_ERR_INVALID_ARG). fst_rnea_vjp_stored then gives the same cotangents
 * as fst_rnea_vjp (within FP32 rounding)
 * without the forward sweep, reading q (free-joint quaternion only), qd and
 * the tape; theta must be the one the tape was written with. The tape costs
 * 120 n_b bytes per environment of HBM traffic each way; recomputation costs
 * the forward sweep's arithmetic. */
FST_API fst_status fst_rnea_tape_bytes(const fst_model* model, int64_t B, size_t* bytes);
FST_API fst_status fst_rnea_store(const fst_model* model, int64_t B, const float* q,
                                  const float* qd, const float* qdd, const float* theta,
                                  float* tau, float* tape, size_t tape_bytes, void* stream);
FST_API fst_status fst_rnea_vjp_stored(const fst_model* model, int64_t B, const float* q,
                                       const float* qd, const float* theta, const float* tape,
                                       size_t tape_bytes, const float* tau_bar, float* q_bar,
                                       float* qd_bar, float* qdd_bar, float* theta_bar,
                                       void* scratch, size_t scratch_bytes, void* stream);

/* ABA (forward dynamics, Sec. 4.1): cotangents of qdd = ABA(q, qd, tau; theta) for qdd_bar [nv][B].
 * qdd [nv][B] must be the forward result for the same inputs. Uses
 * tau_bar = M^-1 qdd_bar and {q_bar, qd_bar, theta_bar} = -RNEA-VJP at qdd. */
FST_API fst_status fst_aba_vjp(const fst_model* model, int64_t B, const float* q,
                               const float* qd, const float* qdd, const float* theta,
                               const float* qdd_bar, float* q_bar, float* qd_bar,
                               float* tau_bar, float* theta_bar, void* scratch,
                               size_t scratch_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Dense derivatives of the dynamics (the analytical derivatives the paper
 * names as the step after its autograd gradients, Sec. 3.5). Matrices are
 * [nv][nv][B] device arrays, element (row r, column c) of environment e at
 * (r * nv + c) * B + e; row = output component, column = direction.
 * Derivatives with respect to q are taken along the configuration's tangent
 * space (nv directions): a revolute or prismatic coordinate directly; a free
 * joint's 6 directions displace its moving frame by [dp; dw] expressed in
 * that frame (position += R dp, R := R exp(dw)), in the order of its
 * velocity [v; w]. Computed by forward-mode sweeps through RNEA, one per
 * degree of freedom.
 * ------------------------------------------------------------------------- */

/* d tau / d q and d tau / d qd of tau = RNEA(q, qd, qdd; theta) (the
 * analytical derivatives of the section above); either output may be NULL
 * (not computed). d tau / d qdd is M (fst_crba). */
FST_API fst_status fst_rnea_derivatives(const fst_model* model, int64_t B, const float* q,
                                        const float* qd, const float* qdd, const float* theta,
                                        float* dtau_dq, float* dtau_dqd, void* stream);

/* Derivatives of qdd = ABA(q, qd, tau; theta): d qdd / d q, d qdd / d qd
 * (either may be NULL) and Minv = d qdd / d tau = M^-1 (required: it also
 * serves as the per-environment Cholesky workspace). qdd [nv][B] optionally
 * receives the forward-dynamics result itself. An environment whose M is
 * not positive definite (for example a massless body on a moving joint)
 * gets non-finite values. */
FST_API fst_status fst_aba_derivatives(const fst_model* model, int64_t B, const float* q,
                                       const float* qd, const float* tau, const float* theta,
                                       float* qdd, float* dqdd_dq, float* dqdd_dqd, float* Minv,
                                       void* stream);

/* System-identification loss L = sum_env sum_i (tau_i - tau_meas_i)^2,
 * tau = RNEA(q, qd, qdd; theta) (paper Sec. 4.3), and its gradient, in one
 * pass that keeps the forward state on chip. loss_theta_bar [n_b*10 + 1]
 * (device) receives dL/dtheta followed by L. q_bar / qd_bar [.][B] optional.
 * scratch is required. */
FST_API fst_status fst_rnea_loss_grad(const fst_model* model, int64_t B, const float* q,
                                      const float* qd, const float* qdd, const float* theta,
                                      const float* tau_meas, float* loss_theta_bar,
                                      float* q_bar, float* qd_bar, void* scratch,
                                      size_t scratch_bytes, void* stream);

/* fst_rnea_vjp for callers that cannot allocate device memory (the paper
 * has no counterpart; this is a deployment convenience). Some callers cannot
 * call cudaMalloc or hand over a scratch buffer: code whose device memory is
 * owned by a pool or arena, real-time loops where an allocation and its
 * implicit synchronisation are not allowed, plugins that only see their
 * input and output tensors. This variant takes the scratch for theta_bar's
 * partial sums from a 4 MiB array that the library keeps in device memory
 * (held by every GPU that loads the library until the process exits) and
 * allocates nothing. Inputs and outputs are as fst_rnea_vjp and are still
 * the caller's.
 * Limits: theta_bar needs ceil(B/32) * (10 n_b + 1) <= 1,048,576 floats
 * (about B = 300,000 for 11 bodies); a larger B with theta_bar set returns
 * FST_ERR_INVALID_ARG before any launch. All calls share the array: calls
 * whose kernels overlap on the GPU (unordered streams) race and give wrong
 * theta_bar; sequential calls are fine and need no clearing. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress with
 * that device current) and caches it; make that first call before any
 * stream capture. The cached address lives as long as the device's primary
 * context: do not call this entry point after a cudaDeviceReset. Argument
 * checks are those of every entry point (B <= 2^31 - 1, the model's device
 * current, non-null inputs), and the call then runs exactly what
 * fst_rnea_vjp runs for this model (its specialised kernel, if compiled). */
FST_API fst_status fst_rnea_vjp_noalloc(const fst_model* model, int64_t B, const float* q,
                                        const float* qd, const float* qdd, const float* theta,
                                        const float* tau_bar, float* q_bar, float* qd_bar,
                                        float* qdd_bar, float* theta_bar, void* stream);

/* ---------------------------------------------------------------------------
 * Mixed batches of several trees in ONE persistent launch. Not in the paper,
 * which evaluates one robot at a time; a mixed batch would otherwise need one
 * launch per tree and operator, each too small to fill the GPU.
 * ------------------------------------------------------------------------- */
#define FST_MAX_MULTI 16

typedef struct fst_multi fst_multi;

/* Per-tree inputs and outputs (device arrays as for the single-tree calls).
 * A NULL output skips that operator for that tree; inputs as fst_eval. */
typedef struct fst_multi_io {
  int64_t B;
  const float* q;
  const float* qd;
  const float* qdd;
  const float* tau;
  float* poses;    /* FK   [n_b][12][B] */
  float* tau_out;  /* RNEA [nv][B] */
  float* M;        /* CRBA [nv][nv][B] */
  float* qdd_out;  /* ABA  [nv][B] */
} fst_multi_io;

/* Groups 1..FST_MAX_MULTI models (same device; they must outlive the group)
 * and allocates its 4-byte device work counter; the handle is owned by the
 * caller and released with fst_multi_destroy (NULL accepted). A batching
 * form with no counterpart in the paper (which batches one tree at a time).
 * FST_ERR_INVALID_ARG for a bad count, a NULL model or models on different
 * devices, FST_ERR_CUDA when the counter cannot be allocated. */
FST_API fst_status fst_multi_create(const fst_model* const* models, int32_t n_models, fst_multi** out);
FST_API fst_status fst_multi_destroy(fst_multi* multi);

/* Evaluates the requested operators (FK Sec. 3.1, RNEA Sec. 3.3, CRBA
 * Sec. 3.5, ABA Sec. 4.1) of every tree in one persistent launch
 * (plus a 4-byte memset that resets the work counter; both are ordered on
 * `stream` and can be captured into a CUDA graph). io has n_models entries,
 * in the order given to fst_multi_create. Overlapping calls on the same
 * group (unordered streams) race on its counter; create one group per
 * stream for that. Results are bit-identical to the per-tree generic calls
 * (with the default launch form; see fst_multi_set_launch). */
FST_API fst_status fst_multi_eval(fst_multi* multi, const fst_multi_io* io, void* stream);

/* Launch form of a group's fst_multi_eval (not in the paper; a tuning knob).
 * FST_VARIANT_GENERIC (the default, block 64): one environment per thread,
 * items of `block` environments. FST_VARIANT_LEVEL: the level-parallel
 * bodies of paper Sec. 3.3, items of 32 environments with the block's
 * block/32 warps splitting each tree level, ABA in its lean form (results
 * then bit-identical to the per-tree calls at that block with
 * FST_VARIANT_LEVEL, and FST_VARIANT_LEVEL_LEAN for ABA); a group whose largest
 * tree's state does not fit in shared memory then returns
 * FST_ERR_INVALID_ARG from fst_multi_eval. block: 32, 64, 128 or 256. */
FST_API fst_status fst_multi_set_launch(fst_multi* multi, int32_t block, int32_t variant);

/* ---------------------------------------------------------------------------
 * Measurement. The paper reports speed against other libraries (Sec. 4.2);
 * this library reports it as a fraction of the GPU's own ceilings, and
 * this probe measures the arithmetic one.
 * ------------------------------------------------------------------------- */

/* Measurement (no counterpart in the paper). Launches an FP32 fused multiply-add throughput probe on `stream`:
 * (SMs x blocks_per_sm) blocks of 256 threads, each thread running 16
 * independent FMA chains for `iters` iterations, and writes one float per
 * thread to out (device memory of at least SMs x blocks_per_sm x 256 floats,
 * so the work cannot be optimised away). *flops (host) receives the flops
 * the launch executes (2 per FMA). Time the launch with CUDA events and
 * divide. blocks_per_sm in [1, 64], iters >= 1; FST_ERR_INVALID_ARG
 * otherwise or when out is too small. */
FST_API fst_status fst_fp32_probe(int32_t blocks_per_sm, int32_t iters, float* out, size_t out_bytes,
                                  double* flops, void* stream);

/* Launch placement (no counterpart in the paper). The ids (PTX %smid) of the current device's SMs, sorted ascending, for
 * building the role table of fst_model_set_sm_roles: a GPU may number its
 * SMs with gaps, so they need not be 0 .. SMs - 1. Writes up to `capacity`
 * ids and sets *n to their number. Synchronous (launches a probe kernel of
 * one block per SM three times and reads the ids back). */
FST_API fst_status fst_sm_ids(int32_t* ids, int32_t capacity, int32_t* n);

/* Output placement (no counterpart in the paper). *ok = 1 when the current device can address `ptr` with that same
 * pointer: device memory of the current device, managed memory, or pinned
 * host memory mapped into the device's address space (cudaHostAlloc'd
 * memory under unified addressing). Any output array of the compute calls
 * may be such pinned host memory: the kernels then write their results
 * straight to the host (on Grace-Blackwell over the coherent NVLink-C2C
 * link), with no separate copy. *ok = 0 for anything else, including
 * ordinary pageable host memory, which must never be passed. */
FST_API fst_status fst_device_can_access(const void* ptr, int32_t* ok);

/* Message for the last non-OK status on this thread ("" if none); the
 * string is owned by the library and valid until the next non-OK status on
 * this thread.
 * Error reporting: no counterpart in the paper. */
FST_API const char* fst_last_error(void);

/* Library version string (static storage, owned by the library). */
FST_API const char* fst_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FST_H */
