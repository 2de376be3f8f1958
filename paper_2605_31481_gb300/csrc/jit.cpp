// Run-time specialisation of the kernels for one model (fst_model_specialize).
//
// For each kernel kind the generator writes a small CUDA source: the model's
// constants as initialised device arrays (floats printed as exact hex
// literals), the body count as a compile-time constant, and an include of
// jit_kernels.cuh. NVRTC compiles it for the current GPU; the cubin is loaded
// through the driver API and cached on disk (keyed by a hash of the source
// and the compiler options), so a second process loads it without
// compiling. NVRTC is opened with dlopen and the driver functions come from
// cudaGetDriverEntryPointByVersion, so libfst.so itself links neither: on a
// host without them specialisation reports FST_ERR_UNSUPPORTED and the
// generic kernels keep serving every call.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <sys/stat.h>
#include <thread>
#include <vector>

#include "fst_internal.h"
#include "jit.h"
#include "launch.h"

namespace fst {

// Embedded copies of the device headers (generated into _build at build time).
extern const int kJitHeaderCount;
extern const char* const kJitHeaderNames[];
extern const char* const kJitHeaderSources[];

namespace {

const char* const kKindName[JK_COUNT] = {"fst_jit_fk",      "fst_jit_jacobian", "fst_jit_rnea",     "fst_jit_crba",
                                         "fst_jit_aba",     "fst_jit_eval",     "fst_jit_fk_vjp",   "fst_jit_rnea_vjp",
                                         "fst_jit_aba_vjp", "fst_jit_loss_grad", "fst_jit_eval_mixed", "fst_jit_rnea_store",
                                         "fst_jit_rnea_vjp_stored", "fst_jit_rnea_derivs", "fst_jit_aba_derivs"};
const char* const kKindMacro[JK_COUNT] = {"FST_JIT_FK",      "FST_JIT_JACOBIAN", "FST_JIT_RNEA",     "FST_JIT_CRBA",
                                          "FST_JIT_ABA",     "FST_JIT_EVAL",     "FST_JIT_FK_VJP",   "FST_JIT_RNEA_VJP",
                                          "FST_JIT_ABA_VJP", "FST_JIT_LOSS_GRAD", "FST_JIT_EVAL_MIXED", "FST_JIT_RNEA_STORE",
                                          "FST_JIT_RNEA_VJP_STORED", "FST_JIT_RNEA_DERIVS", "FST_JIT_ABA_DERIVS"};

// ---- NVRTC, opened at run time ---------------------------------------------
struct Nvrtc {
  bool ok = false;
  std::string why;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*) = nullptr;
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*) = nullptr;
  nvrtcResult (*log_size)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*log)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*cubin)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*destroy)(nvrtcProgram*) = nullptr;
  nvrtcResult (*version)(int*, int*) = nullptr;
};

template <typename F>
bool sym(void* h, const char* name, F& out) {
  out = reinterpret_cast<F>(dlsym(h, name));
  return out != nullptr;
}

const Nvrtc& nvrtc() {
  static Nvrtc N;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void* h = nullptr;
    for (const char* nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
      N.why = "libnvrtc.so could not be opened";
      return;
    }
    N.ok = sym(h, "nvrtcCreateProgram", N.create) && sym(h, "nvrtcCompileProgram", N.compile) &&
           sym(h, "nvrtcGetProgramLogSize", N.log_size) && sym(h, "nvrtcGetProgramLog", N.log) &&
           sym(h, "nvrtcGetCUBINSize", N.cubin_size) && sym(h, "nvrtcGetCUBIN", N.cubin) &&
           sym(h, "nvrtcDestroyProgram", N.destroy) && sym(h, "nvrtcVersion", N.version);
    if (!N.ok) N.why = "libnvrtc.so lacks an expected symbol";
  });
  return N;
}

// ---- driver API through the runtime's entry-point query -------------------
struct Driver {
  bool ok = false;
  CUresult (*load)(CUmodule*, const void*) = nullptr;
  CUresult (*get)(CUfunction*, CUmodule, const char*) = nullptr;
  CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                     void**, void**) = nullptr;
  CUresult (*set_attr)(CUfunction, CUfunction_attribute, int) = nullptr;
  CUresult (*unload)(CUmodule) = nullptr;
};

template <typename F>
bool entry(const char* name, F& out) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p)
    return false;
  out = reinterpret_cast<F>(p);
  return true;
}

const Driver& driver() {
  static Driver D;
  static std::once_flag once;
  std::call_once(once, [] {
    D.ok = entry("cuModuleLoadData", D.load) && entry("cuModuleGetFunction", D.get) &&
           entry("cuLaunchKernel", D.launch) && entry("cuFuncSetAttribute", D.set_attr) &&
           entry("cuModuleUnload", D.unload);
  });
  return D;
}

// ---- source generation ------------------------------------------------------
void put_floats(std::ostringstream& os, const float* p, int n) {
  os << "{";
  char buf[64];
  for (int k = 0; k < n; ++k) {
    std::snprintf(buf, sizeof(buf), "%af", (double)p[k]);
    os << (k ? "," : "") << buf;
  }
  os << "}";
}

// Root-to-leaf paths of the tree in depth-first order (so the paths through
// any body are adjacent), for the path-parallel kernels. Returns the lane
// count G (the number of paths rounded up to a power of two), or 0 when the
// tree has more than 8 leaves.
struct PathTables {
  int G = 0;
  int np = 0;              // number of paths
  std::vector<int> path;   // [G][depth], -1 past a path's end
  std::vector<int> seg;    // [G][depth], lo | hi << 8
  std::vector<unsigned> lead;  // [G], bit t: first lane holding that body
  std::vector<int> red;    // [depth]
  std::vector<int> owner;  // [n]
  std::vector<int> depth_of;  // [n]
};

PathTables path_tables(const fst_model* m) {
  PathTables P;
  const TopoLists& T = m->ht;
  const int D = m->depth;
  std::vector<std::vector<int>> paths;
  std::vector<int> cur;
  // iterative depth-first walk from every root, children in list order
  std::vector<std::pair<int, int>> stack;  // (body, next child position)
  for (int r = 0; r < m->n; ++r) {
    if (m->hi[r].parent >= 0) continue;
    stack.push_back({r, T.child_start[r]});
    cur.push_back(r);
    while (!stack.empty()) {
      auto& top = stack.back();
      const int b = top.first;
      if (T.child_start[b] == T.child_start[b + 1] && top.second == T.child_start[b]) {
        paths.push_back(cur);
        top.second = -1;  // mark done
      }
      if (top.second >= 0 && top.second < T.child_start[b + 1]) {
        const int c = T.child[top.second++];
        stack.push_back({c, T.child_start[c]});
        cur.push_back(c);
        continue;
      }
      stack.pop_back();
      cur.pop_back();
    }
  }
  const int n_paths = (int)paths.size();
  if (n_paths == 0 || n_paths > 8) return P;
  int G = 1;
  while (G < n_paths) G *= 2;
  P.G = G;
  P.np = n_paths;
  P.path.assign((size_t)G * D, -1);
  for (int g = 0; g < n_paths; ++g)
    for (int t = 0; t < (int)paths[g].size(); ++t) P.path[(size_t)g * D + t] = paths[g][t];
  P.seg.assign((size_t)G * D, 0);
  P.lead.assign(G, 0u);
  P.red.assign(D, 0);
  P.owner.assign(m->n, 0);
  P.depth_of.assign(m->n, 0);
  for (int g = 0; g < G; ++g)
    for (int t = 0; t < D; ++t) {
      const int b = P.path[(size_t)g * D + t];
      int lo = g, hi = g + 1;
      if (b >= 0) {
        while (lo > 0 && P.path[(size_t)(lo - 1) * D + t] == b) --lo;
        while (hi < G && P.path[(size_t)hi * D + t] == b) ++hi;
        if (lo == g) {
          P.lead[g] |= 1u << t;
          P.owner[b] = g;
          P.depth_of[b] = t;
        }
      }
      P.seg[(size_t)g * D + t] = lo | (hi << 8);
    }
  for (int b = 0; b < m->n; ++b) {
    const int nc = T.child_start[b + 1] - T.child_start[b];
    if (nc > 1) P.red[P.depth_of[b]] = 1;
  }
  return P;
}

std::string make_source(const fst_model* m, int kind) {
  std::ostringstream os;
  os << "#define FST_FIXED_TOPOLOGY 1\n#define FST_N " << m->n << "\n#define " << kKindMacro[kind] << " 1\n"
     << "#define FST_JIT_NAME " << kKindName[kind] << "\n#define FST_JIT_PATH_NAME " << kKindName[kind] << "_path\n"
     << "#define FST_JIT_WARP_NAME " << kKindName[kind] << "_pathw\n"
     << "#define FST_JIT_PIN_NAME " << kKindName[kind] << "_pin\n"
     << "#define FST_JIT_EXT_NAME " << kKindName[kind] << "_ext\n"
     << "#include \"fst_layout.h\"\nnamespace fst {\nstatic __device__ const BodyC kC[" << m->n << "] = {\n";
  for (int i = 0; i < m->n; ++i) {
    const BodyC& c = m->hc[i];
    os << (i ? ",\n" : "") << "{";
    put_floats(os, c.R0, 9);
    os << ",";
    put_floats(os, c.A, 9);
    os << ",";
    put_floats(os, c.Bm, 9);
    os << ",";
    put_floats(os, c.t0, 3);
    os << ",";
    put_floats(os, c.a, 3);
    os << ",";
    put_floats(os, c.b, 3);
    os << ",";
    put_floats(os, c.S, 6);
    os << ",";
    put_floats(os, c.theta, 10);
    os << "," << c.anc << "ull," << c.lpos << ",{0}}";
  }
  os << "};\nstatic __device__ const BodyI kI[" << m->n << "] = {";
  for (int i = 0; i < m->n; ++i) {
    const BodyI& b = m->hi[i];
    os << (i ? "," : "") << "{" << b.parent << "," << b.type << "," << b.qi << "," << b.vi << "}";
  }
  os << "};\n";
  const TopoLists& T = m->ht;
  auto ints = [&](const char* name, const int* v, int n) {
    os << "static __device__ const int " << name << "[" << (n > 0 ? n : 1) << "] = {";
    for (int k = 0; k < n; ++k) os << (k ? "," : "") << v[k];
    if (n == 0) os << "0";
    os << "};\n";
  };
  ints("kLevelStart", T.level_start, m->depth + 1);
  ints("kLevelBody", T.level_body, m->n);
  ints("kChildStart", T.child_start, m->n + 1);
  ints("kChild", T.child, T.child_start[m->n]);
  const PathTables P = path_tables(m);
  if (P.G > 0) {
    ints("kPath", P.path.data(), (int)P.path.size());
    ints("kSeg", P.seg.data(), (int)P.seg.size());
    os << "static __device__ const unsigned kLead[" << P.G << "] = {";
    for (int g = 0; g < P.G; ++g) os << (g ? "," : "") << P.lead[g] << "u";
    os << "};\n";
    ints("kRed", P.red.data(), (int)P.red.size());
    ints("kOwner", P.owner.data(), m->n);
    ints("kDepthOf", P.depth_of.data(), m->n);
  }
  os << "}  // namespace fst\n#define FST_DEPTH " << m->depth << "\n#define FST_PATH_NP " << P.np
     << "\n#define FST_PATH_G " << P.G
     << "\n#include \"jit_kernels.cuh\"\n";
  return os.str();
}

uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ull) {
  for (unsigned char ch : s) {
    h ^= ch;
    h *= 1099511628211ull;
  }
  return h;
}

std::string cache_dir() {
  if (const char* d = std::getenv("FST_JIT_CACHE")) return d;
  if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/fst_jit";
  return "";
}

bool read_file(const std::string& path, std::vector<char>& out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  out.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
  return !out.empty();
}

void write_file_atomic(const std::string& dir, const std::string& path, const std::vector<char>& data) {
  if (dir.empty()) return;
  std::string cur;
  for (size_t i = 0; i <= dir.size(); ++i) {  // mkdir -p
    if (i == dir.size() || dir[i] == '/') {
      if (!cur.empty()) mkdir(cur.c_str(), 0755);
    }
    if (i < dir.size()) cur += dir[i];
  }
  const std::string tmp = path + ".tmp" + std::to_string((unsigned long)std::hash<std::thread::id>()(std::this_thread::get_id()));
  std::ofstream f(tmp, std::ios::binary);
  if (!f) return;
  f.write(data.data(), (std::streamsize)data.size());
  f.close();
  std::rename(tmp.c_str(), path.c_str());
}

struct CompileJob {
  int kind;
  std::string src;
  std::vector<char> cubin;
  std::string error;
};

void compile_one(CompileJob& job, const std::string& arch_opt) {
  const Nvrtc& N = nvrtc();
  int maj = 0, min = 0;
  N.version(&maj, &min);
  // FST_JIT_MAXRREG=<n> caps the registers per thread of the specialised
  // kernels (more resident warps per SM, at the risk of spills)
  std::string maxrreg;
  if (const char* r = std::getenv("FST_JIT_MAXRREG")) maxrreg = std::string("--maxrregcount=") + r;
  const char* opts[] = {arch_opt.c_str(), "-std=c++17", "--device-as-default-execution-space", maxrreg.c_str()};
  const int nopt = maxrreg.empty() ? 3 : 4;
  std::string key = job.src + arch_opt + maxrreg + std::to_string(maj) + "." + std::to_string(min);
  for (int h = 0; h < kJitHeaderCount; ++h) key += kJitHeaderSources[h];
  char name[32];
  std::snprintf(name, sizeof(name), "%016llx", (unsigned long long)fnv1a(key));
  // FST_JIT_DUMP=<dir> writes each generated source (the tree's constants and
  // the kernel selection; it includes the library's device headers) as
  // <dir>/<kernel>_<hash>.cu, for offline compilation reports
  if (const char* d = std::getenv("FST_JIT_DUMP")) {
    const std::string dump = std::string(d) + "/" + kKindName[job.kind] + "_" + name + ".cu";
    std::ofstream f(dump);
    f << job.src;
  }
  const std::string dir = cache_dir();
  const std::string path = dir.empty() ? "" : dir + "/" + name + ".cubin";
  if (!path.empty() && read_file(path, job.cubin)) return;
  nvrtcProgram prog;
  if (N.create(&prog, job.src.c_str(), "fst_jit.cu", kJitHeaderCount, kJitHeaderSources, kJitHeaderNames) !=
      NVRTC_SUCCESS) {
    job.error = "nvrtcCreateProgram failed";
    return;
  }
  const nvrtcResult rc = N.compile(prog, nopt, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t n = 0;
    N.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) N.log(prog, &log[0]);
    job.error = "NVRTC compilation failed: " + log.substr(0, 2000);
    N.destroy(&prog);
    return;
  }
  size_t n = 0;
  N.cubin_size(prog, &n);
  job.cubin.resize(n);
  N.cubin(prog, job.cubin.data());
  N.destroy(&prog);
  if (!path.empty()) write_file_atomic(dir, path, job.cubin);
}

}  // namespace

// Per kind, up to five kernels of one module: the one-environment-per-thread
// kernel (slot 0), for trees with at most 8 leaves the path-parallel kernels
// with a lane per path (slot 1) or a warp per path (slot 2), and for eval the
// SM-pinned kernel (slot 3) and the extended fused kernel (slot 4).
struct JitState {
  CUmodule mod[JK_COUNT] = {};
  CUfunction fn[JK_SLOTS][JK_COUNT] = {};
  int smem_limit[JK_SLOTS][JK_COUNT] = {};
  int carveout_set[JK_SLOTS][JK_COUNT] = {};
  int path_G = 0, path_np = 0;
};

fst_status jit_specialize(fst_model* m, unsigned mask) {
  const Nvrtc& N = nvrtc();
  if (!N.ok) return set_error(FST_ERR_UNSUPPORTED, "fst_model_specialize: " + N.why);
  const Driver& D = driver();
  if (!D.ok) return set_error(FST_ERR_UNSUPPORTED, "fst_model_specialize: driver entry points unavailable");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
    return set_error(FST_ERR_INVALID_ARG, "fst_model_specialize: the current device is not the model's device");
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  char arch[32];
  std::snprintf(arch, sizeof(arch), "-arch=sm_%d%d%s", major, minor, major >= 9 ? "a" : "");
  if (!m->jit) m->jit = new JitState();
  std::vector<CompileJob> jobs;
  for (int k = 0; k < JK_COUNT; ++k)
    if (((mask >> k) & 1u) && !m->jit->fn[0][k]) jobs.push_back(CompileJob{k, make_source(m, k), {}, {}});
  std::vector<std::thread> threads;
  for (auto& j : jobs) threads.emplace_back([&j, &arch] { compile_one(j, arch); });
  for (auto& t : threads) t.join();
  cudaFree(nullptr);  // make sure the device's primary context is current
  for (auto& j : jobs) {
    if (!j.error.empty()) return set_error(FST_ERR_UNSUPPORTED, std::string("fst_model_specialize: ") + j.error);
    CUmodule mod;
    if (D.load(&mod, j.cubin.data()) != CUDA_SUCCESS)
      return set_error(FST_ERR_CUDA, "fst_model_specialize: cuModuleLoadData failed");
    CUfunction fn;
    if (D.get(&fn, mod, kKindName[j.kind]) != CUDA_SUCCESS) {
      D.unload(mod);
      return set_error(FST_ERR_CUDA, "fst_model_specialize: kernel not found in the compiled module");
    }
    m->jit->mod[j.kind] = mod;
    m->jit->fn[0][j.kind] = fn;
    const char* suffix[JK_SLOTS] = {"", "_path", "_pathw", "_pin", "_ext"};
    for (int v = 1; v < JK_SLOTS; ++v) {
      CUfunction fp;
      const std::string pname = std::string(kKindName[j.kind]) + suffix[v];
      if (D.get(&fp, mod, pname.c_str()) == CUDA_SUCCESS) m->jit->fn[v][j.kind] = fp;
    }
  }
  const PathTables P = path_tables(m);
  m->jit->path_G = P.G;
  m->jit->path_np = P.np;
  return FST_OK;
}

void jit_release(fst_model* m) {
  if (!m->jit) return;
  const Driver& D = driver();
  for (int k = 0; k < JK_COUNT; ++k)
    if (m->jit->mod[k] && D.ok) D.unload(m->jit->mod[k]);
  delete m->jit;
  m->jit = nullptr;
}

unsigned jit_mask(const fst_model* m) {
  unsigned mask = 0;
  if (m->jit)
    for (int k = 0; k < JK_COUNT; ++k)
      if (m->jit->fn[0][k]) mask |= 1u << k;
  return mask;
}

bool jit_has(const fst_model* m, int kind) { return m->jit && m->jit->fn[0][kind]; }

bool jit_has_slot(const fst_model* m, int kind, int slot) { return m->jit && m->jit->fn[slot][kind]; }

int jit_path_lanes(const fst_model* m) { return m->jit ? m->jit->path_G : 0; }

int jit_path_count(const fst_model* m) { return m->jit ? m->jit->path_np : 0; }

cudaError_t jit_launch_slot(const fst_model* m, int kind, int slot, dim3 grid, int block, size_t smem,
                            cudaStream_t s, void** args) {
  return jit_launch_slot3(m, kind, slot, grid, dim3((unsigned)block), smem, s, args);
}

cudaError_t jit_launch_slot3(const fst_model* m, int kind, int slot, dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, void** args) {
  const Driver& D = driver();
  JitState* J = m->jit;
  CUfunction f = J->fn[slot][kind];
  if (smem > 48 * 1024 && (int)smem > J->smem_limit[slot][kind]) {
    if (D.set_attr(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    J->smem_limit[slot][kind] = (int)smem;
  }
  const int gen = carveout_generation() + 1;
  if (J->carveout_set[slot][kind] != gen) {
    int pct = -1;  // the driver's default preference (CU_SHAREDMEM_CARVEOUT_DEFAULT)
    if (const char* env = std::getenv("FST_SMEM_CARVEOUT")) pct = std::atoi(env);
    if (carveout_override() >= 0) pct = carveout_override();
    pct = pct < -1 ? -1 : (pct > 100 ? 100 : pct);
    if (pct >= 0 || J->carveout_set[slot][kind] != 0)
      D.set_attr(f, CU_FUNC_ATTRIBUTE_PREFERRED_SHARED_MEMORY_CARVEOUT, pct);
    J->carveout_set[slot][kind] = gen;
  }
  const CUresult r = D.launch(f, grid.x, grid.y, grid.z, block.x, block.y, block.z, (unsigned)smem, (CUstream)s, args,
                              nullptr);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

cudaError_t jit_launch(const fst_model* m, int kind, dim3 grid, int block, size_t smem, cudaStream_t s, void** args) {
  return jit_launch_slot(m, kind, 0, grid, block, smem, s, args);
}

}  // namespace fst
