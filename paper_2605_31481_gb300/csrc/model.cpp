// Host model builder: validates the body table and precomputes, in FP64,
// every per-joint constant the kernels read (rounded to FP32 at the end).
//
// The revolute constants are the paper's matmul-free joint transform
// (Sec. 3.2, Eq. 2-3): with K = [axis]x, R_pre/t_pre from T_joint and
// R_post/t_post from T_link,
//   R0 = R_pre R_post,  A = R_pre K R_post,  Bm = R_pre K^2 R_post,
//   t0 = R_pre t_post + t_pre,  a = R_pre K t_post,  b = R_pre K^2 t_post,
// so that at run time R_pc = R0 + sin q A + (1 - cos q) Bm (Eq. 4) and
// t_pc = t0 + sin q a + (1 - cos q) b (Eq. 5) need no matrix product.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <sstream>

#include "fst_internal.h"

namespace fst {
namespace {

struct M3 {
  double m[9];
};
struct V3 {
  double v[3];
};

M3 mul(const M3& A, const M3& B) {
  M3 C;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A.m[3 * r + k] * B.m[3 * k + c];
      C.m[3 * r + c] = s;
    }
  return C;
}
V3 mulv(const M3& A, const V3& x) {
  V3 y;
  for (int r = 0; r < 3; ++r) y.v[r] = A.m[3 * r] * x.v[0] + A.m[3 * r + 1] * x.v[1] + A.m[3 * r + 2] * x.v[2];
  return y;
}
V3 mulTv(const M3& A, const V3& x) {
  V3 y;
  for (int r = 0; r < 3; ++r) y.v[r] = A.m[r] * x.v[0] + A.m[3 + r] * x.v[1] + A.m[6 + r] * x.v[2];
  return y;
}
V3 cross(const V3& a, const V3& b) {
  return V3{{a.v[1] * b.v[2] - a.v[2] * b.v[1], a.v[2] * b.v[0] - a.v[0] * b.v[2],
             a.v[0] * b.v[1] - a.v[1] * b.v[0]}};
}
M3 skew(const V3& a) { return M3{{0, -a.v[2], a.v[1], a.v[2], 0, -a.v[0], -a.v[1], a.v[0], 0}}; }

bool finite_all(const double* p, int n) {
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

bool is_rotation(const double* R) {
  M3 A;
  std::memcpy(A.m, R, sizeof(A.m));
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A.m[3 * r + k] * A.m[3 * c + k];
      if (std::fabs(s - (r == c ? 1.0 : 0.0)) > 1e-6) return false;
    }
  double det = A.m[0] * (A.m[4] * A.m[8] - A.m[5] * A.m[7]) - A.m[1] * (A.m[3] * A.m[8] - A.m[5] * A.m[6]) +
               A.m[2] * (A.m[3] * A.m[7] - A.m[4] * A.m[6]);
  return det > 0;
}

bool is_identity12(const double* T) {
  static const double I[12] = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0};
  for (int k = 0; k < 12; ++k)
    if (std::fabs(T[k] - I[k]) > 1e-12) return false;
  return true;
}

// Symmetric 3x3 from (xx xy yy xz yz zz) is positive semi-definite iff all
// principal minors are >= 0 (checked with a small relative slack).
bool psd_sym(const double* s) {
  double xx = s[0], xy = s[1], yy = s[2], xz = s[3], yz = s[4], zz = s[5];
  double scale = std::fabs(xx) + std::fabs(yy) + std::fabs(zz) + 1e-300;
  double eps = 1e-12 * scale;
  if (xx < -eps || yy < -eps || zz < -eps) return false;
  if (xx * yy - xy * xy < -eps * scale) return false;
  if (xx * zz - xz * xz < -eps * scale) return false;
  if (yy * zz - yz * yz < -eps * scale) return false;
  double det = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
  return det >= -eps * scale * scale;
}

void put(float* dst, const double* src, int n) {
  for (int k = 0; k < n; ++k) dst[k] = (float)src[k];
}

}  // namespace

fst_status build_model_host(const fst_body_desc* bodies, int32_t n, const double gravity[3], fst_model* m) {
  if (!bodies || !gravity) return set_error(FST_ERR_INVALID_ARG, "fst_model_create: null bodies or gravity");
  if (n < 1) return set_error(FST_ERR_INVALID_ARG, "fst_model_create: n_bodies must be >= 1");
  if (n > FST_MAX_BODIES) {
    std::ostringstream os;
    os << "fst_model_create: " << n << " bodies exceeds FST_MAX_BODIES=" << FST_MAX_BODIES;
    return set_error(FST_ERR_UNSUPPORTED, os.str());
  }
  if (!finite_all(gravity, 3)) return set_error(FST_ERR_INVALID_ARG, "fst_model_create: gravity not finite");

  m->n = n;
  m->hc.assign(n, BodyC{});
  m->hi.assign(n, BodyI{});
  m->ancestors.assign(n, 0);
  m->level.assign(n, 0);
  for (int k = 0; k < 3; ++k) m->gravity[k] = gravity[k];
  int nq = 0, nv = 0, depth = 0;
  for (int i = 0; i < n; ++i) {
    const fst_body_desc& d = bodies[i];
    std::ostringstream where;
    where << "fst_model_create: body " << i << ": ";
    if (d.parent < -1 || d.parent >= i)
      return set_error(FST_ERR_TOPOLOGY, where.str() + "parent must be in [-1, i-1] (topological order)");
    if (d.type < FST_JOINT_FIXED || d.type > FST_JOINT_FREE)
      return set_error(FST_ERR_UNSUPPORTED, where.str() + "unknown joint type");
    if (d.type == FST_JOINT_FREE && (i != 0 || d.parent != -1))
      return set_error(FST_ERR_TOPOLOGY, where.str() + "a free joint is only allowed on body 0 with parent -1");
    if (!finite_all(d.axis, 3) || !finite_all(d.T_joint, 12) || !finite_all(d.T_link, 12))
      return set_error(FST_ERR_INVALID_ARG, where.str() + "non-finite axis or transform");
    if (!is_rotation(d.T_joint) || !is_rotation(d.T_link))
      return set_error(FST_ERR_INVALID_ARG, where.str() + "T_joint/T_link rotation is not orthonormal");
    if (d.type == FST_JOINT_FREE && !is_identity12(d.T_link))
      return set_error(FST_ERR_UNSUPPORTED, where.str() + "a free joint needs T_link = identity");
    if (!std::isfinite(d.mass) || d.mass < 0 || !finite_all(d.com, 3) || !finite_all(d.I_com, 6) ||
        !psd_sym(d.I_com))
      return set_error(FST_ERR_INERTIA, where.str() + "mass must be >= 0 and I_com finite and positive semi-definite");

    BodyI& bi = m->hi[i];
    bi.parent = d.parent;
    bi.type = d.type;
    bi.qi = nq;
    bi.vi = nv;
    nq += (d.type == FST_JOINT_FREE) ? 7 : (d.type == FST_JOINT_FIXED ? 0 : 1);
    nv += (d.type == FST_JOINT_FREE) ? 6 : (d.type == FST_JOINT_FIXED ? 0 : 1);
    m->level[i] = d.parent < 0 ? 1 : m->level[d.parent] + 1;
    if (m->level[i] > depth) depth = m->level[i];
    m->ancestors[i] = (d.parent < 0 ? 0ull : m->ancestors[d.parent]) | (1ull << i);
    if (d.type == FST_JOINT_FREE) m->has_free = true;
    m->hc[i].anc = m->ancestors[i];

    M3 Rpre, Rpost;
    std::memcpy(Rpre.m, d.T_joint, sizeof(Rpre.m));
    std::memcpy(Rpost.m, d.T_link, sizeof(Rpost.m));
    V3 tpre{{d.T_joint[9], d.T_joint[10], d.T_joint[11]}};
    V3 tpost{{d.T_link[9], d.T_link[10], d.T_link[11]}};
    V3 ax{{d.axis[0], d.axis[1], d.axis[2]}};
    if (d.type == FST_JOINT_REVOLUTE || d.type == FST_JOINT_PRISMATIC) {
      double nrm = std::sqrt(ax.v[0] * ax.v[0] + ax.v[1] * ax.v[1] + ax.v[2] * ax.v[2]);
      if (!(nrm > 1e-12)) return set_error(FST_ERR_INVALID_ARG, where.str() + "joint axis has zero length");
      for (int k = 0; k < 3; ++k) ax.v[k] /= nrm;
    }
    BodyC& c = m->hc[i];
    M3 R0 = mul(Rpre, Rpost);
    V3 Rt = mulv(Rpre, tpost);
    V3 t0{{Rt.v[0] + tpre.v[0], Rt.v[1] + tpre.v[1], Rt.v[2] + tpre.v[2]}};
    if (d.type == FST_JOINT_FREE) {
      put(c.R0, Rpre.m, 9);
      put(c.t0, tpre.v, 3);
    } else {
      put(c.R0, R0.m, 9);
      put(c.t0, t0.v, 3);
    }
    if (d.type == FST_JOINT_REVOLUTE) {
      M3 K = skew(ax);
      M3 K2 = mul(K, K);
      M3 A = mul(mul(Rpre, K), Rpost);
      M3 Bm = mul(mul(Rpre, K2), Rpost);
      V3 a = mulv(Rpre, mulv(K, tpost));
      V3 b = mulv(Rpre, mulv(K2, tpost));
      put(c.A, A.m, 9);
      put(c.Bm, Bm.m, 9);
      put(c.a, a.v, 3);
      put(c.b, b.v, 3);
      // motion subspace in body coordinates: w = R_post^T axis, passing
      // through the joint origin, which sits at -R_post^T t_post in the body
      V3 w = mulTv(Rpost, ax);
      V3 o = mulTv(Rpost, tpost);
      for (int k = 0; k < 3; ++k) o.v[k] = -o.v[k];
      V3 v = cross(o, w);
      double S[6] = {w.v[0], w.v[1], w.v[2], v.v[0], v.v[1], v.v[2]};
      put(c.S, S, 6);
    } else if (d.type == FST_JOINT_PRISMATIC) {
      V3 a = mulv(Rpre, ax);
      put(c.a, a.v, 3);
      V3 w = mulTv(Rpost, ax);
      double S[6] = {0, 0, 0, w.v[0], w.v[1], w.v[2]};
      put(c.S, S, 6);
    }
    // inertia about the body origin: I_o = I_c + m (|c|^2 1 - c c^T)
    double mass = d.mass;
    const double* cm = d.com;
    double cc = cm[0] * cm[0] + cm[1] * cm[1] + cm[2] * cm[2];
    double th[10];
    th[0] = mass;
    th[1] = mass * cm[0];
    th[2] = mass * cm[1];
    th[3] = mass * cm[2];
    th[4] = d.I_com[0] + mass * (cc - cm[0] * cm[0]);
    th[5] = d.I_com[1] - mass * cm[0] * cm[1];
    th[6] = d.I_com[2] + mass * (cc - cm[1] * cm[1]);
    th[7] = d.I_com[3] - mass * cm[0] * cm[2];
    th[8] = d.I_com[4] - mass * cm[1] * cm[2];
    th[9] = d.I_com[5] + mass * (cc - cm[2] * cm[2]);
    put(c.theta, th, 10);
  }
  m->nq = nq;
  m->nv = nv;
  m->depth = depth;
  // level lists (stable: bodies of a level in body order) and child lists
  TopoLists& T = m->ht;
  int k = 0;
  m->max_width = 0;
  for (int l = 0; l < depth; ++l) {
    T.level_start[l] = k;
    for (int i = 0; i < n; ++i)
      if (m->level[i] == l + 1) {
        m->hc[i].lpos = k - T.level_start[l];
        T.level_body[k++] = i;
      }
    m->max_width = std::max(m->max_width, k - T.level_start[l]);
  }
  T.level_start[depth] = k;
  k = 0;
  for (int i = 0; i < n; ++i) {
    T.child_start[i] = k;
    for (int j = i + 1; j < n; ++j)
      if (bodies[j].parent == i) T.child[k++] = j;
  }
  T.child_start[n] = k;
  return FST_OK;
}

}  // namespace fst
