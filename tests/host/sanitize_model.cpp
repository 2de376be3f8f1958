// Host-only checks of the model builder (its per-joint constants against the
// plain product of the joint poses) and of the path tables of the
// specialised kernels, compiled with -fsanitize=address,undefined by
// tests/test_host_sanitize.py. Exits non-zero (with a message) on the first
// violated property; a sanitizer report also fails the run.
//
// The translation unit includes jit.cpp to reach its internal helpers
// (path_tables, make_source); nothing here calls NVRTC, the driver or a GPU.
#include "jit.cpp"

#include <array>
#include <cmath>
#include <cstdio>
#include <random>

namespace fst {
// stand-ins for the symbols the library defines elsewhere
fst_status set_error(fst_status s, const std::string&) { return s; }
int carveout_override() { return -1; }
int carveout_generation() { return 0; }
extern const int kJitHeaderCount = 0;
extern const char* const kJitHeaderNames[] = {nullptr};
extern const char* const kJitHeaderSources[] = {nullptr};
}  // namespace fst

namespace {

int fail(const char* what, int seed) {
  std::fprintf(stderr, "FAILED: %s (seed %d)\n", what, seed);
  return 1;
}

void identity12(double* T) {
  for (int k = 0; k < 12; ++k) T[k] = (k == 0 || k == 4 || k == 8) ? 1.0 : 0.0;
}

// A random valid table: parents before children, every joint type, a free
// root now and then, random unit axes, offsets and inertias.
std::vector<fst_body_desc> random_tree(std::mt19937& rng, int n, bool free_root) {
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::vector<fst_body_desc> b(n);
  for (int i = 0; i < n; ++i) {
    fst_body_desc& d = b[i];
    std::memset(&d, 0, sizeof(d));
    d.parent = i == 0 ? -1 : (int)(rng() % (unsigned)i);
    if (i > 0 && rng() % 7 == 0) d.parent = -1;  // a forest now and then
    const unsigned r = rng() % 10;
    d.type = (i == 0 && free_root) ? FST_JOINT_FREE : (r < 6 ? FST_JOINT_REVOLUTE : r < 8 ? FST_JOINT_PRISMATIC : FST_JOINT_FIXED);
    double a[3] = {U(rng), U(rng), U(rng)};
    const double na = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) + 1e-3;
    for (int k = 0; k < 3; ++k) d.axis[k] = a[k] / na;
    identity12(d.T_joint);
    identity12(d.T_link);
    for (int k = 9; k < 12; ++k) d.T_joint[k] = 0.3 * U(rng);
    d.mass = 0.5 + 2.0 * (U(rng) + 1.0);
    for (int k = 0; k < 3; ++k) d.com[k] = 0.1 * U(rng);
    const double l[3] = {0.05 + 0.01 * U(rng), 0.05 + 0.01 * U(rng), 0.05 + 0.01 * U(rng)};
    d.I_com[0] = l[0];
    d.I_com[2] = l[1];
    d.I_com[5] = l[2];
  }
  return b;
}

// Invariants of the root-to-leaf path tables.
int check_paths(const fst_model& m, const fst::PathTables& P, int seed) {
  const fst::TopoLists& T = m.ht;
  int leaves = 0;
  for (int i = 0; i < m.n; ++i) leaves += T.child_start[i] == T.child_start[i + 1];
  if (leaves > 8) return P.G == 0 ? 0 : fail("more than 8 leaves must give no path tables", seed);
  if (P.np != leaves || P.G < P.np || P.G > 8 || (P.G & (P.G - 1))) return fail("lane count", seed);
  const int D = m.depth;
  std::vector<int> seen(m.n, 0);
  for (int g = 0; g < P.G; ++g) {
    for (int t = 0; t < D; ++t) {
      const int b = P.path[(size_t)g * D + t];
      if (g >= P.np) {
        if (b != -1) return fail("padding lanes hold no bodies", seed);
        continue;
      }
      if (b < 0) {
        if (t + 1 < D && P.path[(size_t)g * D + t + 1] >= 0) return fail("a path has a gap", seed);
        continue;
      }
      ++seen[b];
      const int parent = m.hi[b].parent;
      if (t == 0 && parent != -1) return fail("a path starts at a root", seed);
      if (t > 0 && P.path[(size_t)g * D + t - 1] != parent) return fail("consecutive path bodies are parent and child", seed);
      const bool last = t + 1 == D || P.path[(size_t)g * D + t + 1] < 0;
      if (last && T.child_start[b] != T.child_start[b + 1]) return fail("a path ends at a leaf", seed);
      const int lo = P.seg[(size_t)g * D + t] & 0xff, hi = P.seg[(size_t)g * D + t] >> 8;
      if (!(lo <= g && g < hi && hi <= P.np)) return fail("segment holds its lane", seed);
      for (int k = 0; k < P.G; ++k)
        if ((P.path[(size_t)k * D + t] == b) != (k >= lo && k < hi)) return fail("segment is exactly the lanes sharing the body", seed);
      if (((P.lead[g] >> t) & 1u) != (unsigned)(lo == g)) return fail("leader is the segment's first lane", seed);
      if (P.owner[b] != lo || P.depth_of[b] != t) return fail("owner and depth of a body", seed);
    }
  }
  for (int b = 0; b < m.n; ++b)
    if (seen[b] == 0) return fail("every body lies on a path", seed);
  for (int b = 0; b < m.n; ++b)
    if (T.child_start[b + 1] - T.child_start[b] > 1 && !P.red[P.depth_of[b]])
      return fail("a depth with a branching body is marked for merging", seed);
  return 0;
}

// Rotation of a unit quaternion (w, x, y, z), in row-major order.
void quat_R(double w, double x, double y, double z, double* R) {
  const double n = std::sqrt(w * w + x * x + y * y + z * z);
  w /= n, x /= n, y /= n, z /= n;
  const double r[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                       2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                       2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
  std::memcpy(R, r, sizeof(r));
}

void random_pose(std::mt19937& rng, double* T) {
  std::normal_distribution<double> N(0.0, 1.0);
  quat_R(N(rng), N(rng), N(rng), N(rng), T);
  for (int k = 9; k < 12; ++k) T[k] = 0.3 * N(rng);
}

// C = A B for 3x4 poses (R row-major, then t).
void pose_mul(const double* A, const double* B, double* C) {
  double out[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      out[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
    out[9 + r] = A[3 * r] * B[9] + A[3 * r + 1] * B[10] + A[3 * r + 2] * B[11] + A[9 + r];
  }
  std::memcpy(C, out, sizeof(out));
}

// Parent-to-child pose T_joint * J(q) * T_link as a plain product, with the
// joint motion J(q) a rotation by q about the axis (built from the
// quaternion (cos q/2, sin q/2 axis)) or a translation by q along it.
void product_pose(const fst_body_desc& d, double q, double* T) {
  double J[12] = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0};
  const double na = std::sqrt(d.axis[0] * d.axis[0] + d.axis[1] * d.axis[1] + d.axis[2] * d.axis[2]);
  const double u[3] = {d.axis[0] / na, d.axis[1] / na, d.axis[2] / na};
  if (d.type == FST_JOINT_REVOLUTE)
    quat_R(std::cos(0.5 * q), std::sin(0.5 * q) * u[0], std::sin(0.5 * q) * u[1], std::sin(0.5 * q) * u[2], J);
  if (d.type == FST_JOINT_PRISMATIC)
    for (int k = 0; k < 3; ++k) J[9 + k] = q * u[k];
  pose_mul(d.T_joint, J, T);
  pose_mul(T, d.T_link, T);
}

// The model builder's per-joint constants (paper Sec. 3.2, Eq. 2-5), FP32,
// against the plain product of the joint's poses: the pose at random q, and
// the motion subspace against central differences of the pose (the child
// frame's twist in its own coordinates, [w; v]).
int check_joint_constants(int seed) {
  std::mt19937 rng(1000 + seed);
  std::normal_distribution<double> N(0.0, 1.0);
  const int n = 6;
  auto b = random_tree(rng, n, false);
  for (int i = 0; i < n; ++i) {
    random_pose(rng, b[i].T_joint);
    random_pose(rng, b[i].T_link);
  }
  fst_model m;
  if (fst::build_model_host(b.data(), n, std::array<double, 3>{0, 0, -9.81}.data(), &m) != FST_OK)
    return fail("a table with rotated joint and link frames is accepted", seed);
  for (int i = 0; i < n; ++i) {
    const fst_body_desc& d = b[i];
    const fst::BodyC& c = m.hc[i];
    for (int trial = 0; trial < 8; ++trial) {
      const double q = d.type == FST_JOINT_FIXED ? 0.0 : 3.0 * N(rng);
      double T[12], G[12];
      product_pose(d, q, T);
      const double s = std::sin(q), omc = 1.0 - std::cos(q);
      for (int k = 0; k < 9; ++k)
        G[k] = d.type == FST_JOINT_REVOLUTE ? c.R0[k] + s * c.A[k] + omc * c.Bm[k] : c.R0[k];
      for (int k = 0; k < 3; ++k)
        G[9 + k] = d.type == FST_JOINT_REVOLUTE   ? c.t0[k] + s * c.a[k] + omc * c.b[k]
                   : d.type == FST_JOINT_PRISMATIC ? c.t0[k] + q * c.a[k]
                                                   : c.t0[k];
      for (int k = 0; k < 12; ++k)
        if (std::fabs(G[k] - T[k]) > 2e-6 * (1.0 + std::fabs(q))) return fail("joint constants reproduce the pose product", seed);
      if (d.type == FST_JOINT_FIXED) continue;
      const double h = 1e-6;
      double Tp[12], Tm[12];
      product_pose(d, q + h, Tp);
      product_pose(d, q - h, Tm);
      double dR[9], dt[3];
      for (int k = 0; k < 9; ++k) dR[k] = (Tp[k] - Tm[k]) / (2 * h);
      for (int k = 0; k < 3; ++k) dt[k] = (Tp[9 + k] - Tm[9 + k]) / (2 * h);
      double W[9];  // R^T dR, skew
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) W[3 * r + cc] = T[r] * dR[cc] + T[3 + r] * dR[3 + cc] + T[6 + r] * dR[6 + cc];
      const double S[6] = {W[7], W[2], W[3],
                           T[0] * dt[0] + T[3] * dt[1] + T[6] * dt[2],
                           T[1] * dt[0] + T[4] * dt[1] + T[7] * dt[2],
                           T[2] * dt[0] + T[5] * dt[1] + T[8] * dt[2]};
      for (int k = 0; k < 6; ++k)
        if (std::fabs(S[k] - c.S[k]) > 2e-6) return fail("motion subspace is the child frame's twist", seed);
    }
  }
  return 0;
}

}  // namespace

int main() {
  const double g[3] = {0.0, 0.0, -9.81};
  int checked = 0;
  for (int seed = 0; seed < 400; ++seed) {
    std::mt19937 rng(seed);
    const int n = 1 + (int)(rng() % 64);
    auto b = random_tree(rng, n, seed % 5 == 0);
    fst_model m;
    if (fst::build_model_host(b.data(), n, g, &m) != FST_OK) return fail("a valid random table is accepted", seed);
    const fst::PathTables P = fst::path_tables(&m);
    if (check_paths(m, P, seed)) return 1;
    if (seed % 20 == 0)
      for (int k = 0; k < fst::JK_COUNT; ++k)
        if (fst::make_source(&m, k).find("jit_kernels.cuh") == std::string::npos) return fail("source generation", seed);
    ++checked;
  }
  for (int seed = 0; seed < 50; ++seed)
    if (check_joint_constants(seed)) return 1;
  // malformed tables are refused with an error status, never a crash
  std::mt19937 rng(1234);
  for (int c = 0; c < 8; ++c) {
    auto b = random_tree(rng, 6, false);
    switch (c) {
      case 0: b[3].parent = 3; break;
      case 1: b[2].parent = 5; break;
      case 2: b[4].type = 17; break;
      case 3: b[2].type = FST_JOINT_FREE; break;
      case 4: b[1].mass = std::nan(""); break;
      case 5: b[1].I_com[1] = 5.0; break;
      case 6: b[1].axis[0] = b[1].axis[1] = b[1].axis[2] = 0.0; b[1].type = FST_JOINT_REVOLUTE; break;
      case 7: b[0].parent = -7; break;
    }
    fst_model m;
    if (fst::build_model_host(b.data(), 6, g, &m) == FST_OK) return fail("a malformed table is refused", c);
  }
  fst_model m;
  if (fst::build_model_host(nullptr, 3, g, &m) == FST_OK) return fail("null table", 0);
  std::printf("ok %d random trees\n", checked);
  return 0;
}
