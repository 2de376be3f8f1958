// Writes the run-time generated source of every specialised kernel kind for
// a few fixed trees, as the library generates them (make_source), into the
// directory given as argv[1], one file per tree and kind:
// <dir>/<tree>_<kind>.cu. tests/test_jit_compile_host.py compiles each with
// NVRTC for sm_103a on the CPU, so a device-code error in the kernels that
// are only compiled at run time shows before any GPU run. Host only: nothing
// here calls NVRTC, the driver or a GPU.
#include "jit.cpp"

#include <cstdio>
#include <fstream>

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

fst_body_desc body(int parent, int type, double ax, double ay, double az, double ox, double oy, double oz) {
  fst_body_desc d;
  std::memset(&d, 0, sizeof(d));
  d.parent = parent;
  d.type = type;
  d.axis[0] = ax;
  d.axis[1] = ay;
  d.axis[2] = az;
  for (int k = 0; k < 12; ++k) d.T_joint[k] = d.T_link[k] = (k == 0 || k == 4 || k == 8) ? 1.0 : 0.0;
  d.T_joint[9] = ox;
  d.T_joint[10] = oy;
  d.T_joint[11] = oz;
  d.mass = 1.5;
  d.com[2] = 0.05;
  d.I_com[0] = 0.02;
  d.I_com[2] = 0.03;
  d.I_com[5] = 0.04;
  return d;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const std::string dir = argv[1];
  const double g[3] = {0.0, 0.0, -9.81};
  const int R = FST_JOINT_REVOLUTE, P = FST_JOINT_PRISMATIC, F = FST_JOINT_FIXED;
  std::vector<std::pair<std::string, std::vector<fst_body_desc>>> trees;
  // a 3-joint spine with two 2-joint legs off each end (depth 5, 4 leaves)
  std::vector<fst_body_desc> quad = {body(-1, R, 0, 0, 1, 0, 0, 0.5), body(0, R, 0, 1, 0, 0.2, 0, 0),
                                     body(1, R, 1, 0, 0, 0.2, 0, 0)};
  for (int side = 0; side < 2; ++side)
    for (int end = 0; end < 2; ++end) {
      const int hip = (int)quad.size();
      quad.push_back(body(end ? 2 : 0, R, 0, 1, 0, 0.1, side ? 0.1 : -0.1, 0));
      quad.push_back(body(hip, R, 0, 1, 0, 0, 0, -0.2));
    }
  trees.emplace_back("quadruped", quad);
  // a floating base with a revolute arm, a prismatic stage and a fixed frame
  trees.emplace_back("floating", std::vector<fst_body_desc>{
                                     body(-1, FST_JOINT_FREE, 0, 0, 1, 0, 0, 0), body(0, R, 0, 0, 1, 0.1, 0, 0),
                                     body(1, P, 1, 0, 0, 0.2, 0, 0), body(2, F, 0, 0, 1, 0, 0, 0.1),
                                     body(0, R, 1, 0, 0, -0.1, 0, 0), body(4, R, 0, 1, 0, 0, 0, -0.2)});
  int written = 0;
  for (auto& t : trees) {
    fst_model m;
    if (fst::build_model_host(t.second.data(), (int)t.second.size(), g, &m) != FST_OK) {
      std::fprintf(stderr, "FAILED: tree %s is refused\n", t.first.c_str());
      return 1;
    }
    for (int k = 0; k < fst::JK_COUNT; ++k) {
      std::ofstream f(dir + "/" + t.first + "_" + fst::kKindName[k] + ".cu");
      f << fst::make_source(&m, k);
      ++written;
    }
  }
  std::printf("ok %d\n", written);
  return 0;
}
