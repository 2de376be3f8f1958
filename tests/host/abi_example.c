/* A plain-C caller of libfst.so: a planar two-link arm, B environments, FK,
 * inverse dynamics and the mass matrix on the GPU, every status checked.
 * tests/test_abi_host.py compiles and links it as ISO C11 with warnings as
 * errors and runs it; without a GPU, model creation reports FST_ERR_CUDA. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include "fst.h"

#define CHECK(call)                                                          \
  do {                                                                       \
    fst_status s_ = (call);                                                  \
    if (s_ != FST_OK) {                                                      \
      fprintf(stderr, "%s failed (%d): %s\n", #call, (int)s_, fst_last_error()); \
      return 1;                                                              \
    }                                                                        \
  } while (0)

static void identity(double T[12]) {
  memset(T, 0, 12 * sizeof(double));
  T[0] = T[4] = T[8] = 1.0;
}

int main(void) {
  enum { B = 1024, NB = 2 };
  fst_body_desc bodies[NB];
  const double gravity[3] = {0.0, -9.81, 0.0};
  int i;
  memset(bodies, 0, sizeof(bodies));
  for (i = 0; i < NB; ++i) {
    bodies[i].parent = i - 1;
    bodies[i].type = FST_JOINT_REVOLUTE;
    bodies[i].axis[2] = 1.0;                  /* about z */
    identity(bodies[i].T_joint);
    identity(bodies[i].T_link);
    bodies[i].mass = 1.0;
    bodies[i].com[0] = 0.25;                  /* half way along the link */
    bodies[i].I_com[0] = bodies[i].I_com[2] = bodies[i].I_com[5] = 0.01;
  }
  bodies[1].T_joint[9] = 0.5;                 /* second joint at the end of the first link */

  fst_model* model = NULL;
  CHECK(fst_model_create(bodies, NB, gravity, &model));
  int32_t nq = 0, nv = 0, nb = 0, depth = 0;
  CHECK(fst_model_info(model, &nq, &nv, &nb, &depth));

  float *q = NULL, *qd = NULL, *qdd = NULL, *tau = NULL, *poses = NULL, *M = NULL;
  if (cudaMalloc((void**)&q, sizeof(float) * nq * B) != cudaSuccess ||
      cudaMalloc((void**)&qd, sizeof(float) * nv * B) != cudaSuccess ||
      cudaMalloc((void**)&qdd, sizeof(float) * nv * B) != cudaSuccess ||
      cudaMalloc((void**)&tau, sizeof(float) * nv * B) != cudaSuccess ||
      cudaMalloc((void**)&poses, sizeof(float) * nb * 12 * B) != cudaSuccess ||
      cudaMalloc((void**)&M, sizeof(float) * nv * nv * B) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  cudaMemset(q, 0, sizeof(float) * nq * B);   /* arm stretched along x */
  cudaMemset(qd, 0, sizeof(float) * nv * B);
  cudaMemset(qdd, 0, sizeof(float) * nv * B);

  /* arrays are [field][B]: element (field f, environment e) at f * B + e */
  CHECK(fst_fk(model, B, q, poses, NULL));
  CHECK(fst_rnea(model, B, q, qd, qdd, NULL, tau, NULL));   /* gravity torques */
  CHECK(fst_crba(model, B, q, NULL, M, NULL));
  float tau0[2];
  cudaMemcpy(&tau0[0], tau, sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(&tau0[1], tau + B, sizeof(float), cudaMemcpyDeviceToHost);
  /* horizontal arm: tau1 = g (m1 c1 + m2 (l1 + c2)), tau2 = g m2 c2 */
  printf("tau = (%.4f, %.4f), expected (%.4f, %.4f)\n", tau0[0], tau0[1], 9.81 * (0.25 + 0.75), 9.81 * 0.25);

  cudaFree(q);
  cudaFree(qd);
  cudaFree(qdd);
  cudaFree(tau);
  cudaFree(poses);
  cudaFree(M);
  CHECK(fst_model_destroy(model));
  return 0;
}
