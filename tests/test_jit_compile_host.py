"""The kernels specialised at run time (NVRTC) compile for sm_103a, on the
CPU: the host generator writes the source of every kernel kind for two trees
(a branched fixed-base tree with path-parallel tables, a floating base with
prismatic and fixed joints), exactly as the library generates it, and NVRTC
compiles each with the options the library uses. A device-code error in
these kernels would otherwise show only on a GPU, at fst_model_specialize."""
import concurrent.futures
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_31481_gb300", "csrc")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
OPTS = ["-arch=sm_103a", "-std=c++17", "--device-as-default-execution-space"]


@pytest.fixture(scope="module")
def sources(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(os.path.join(CUDA, "include")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("jit")
    exe = d / "jit_sources"
    cmd = ["g++", "-std=c++17", "-O1", f"-I{CUDA}/include", f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}",
           os.path.join(ROOT, "tests", "host", "jit_sources.cpp"), os.path.join(CSRC, "model.cpp"),
           "-o", str(exe), f"-L{CUDA}/lib64", "-lcudart", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = d / "src"
    out.mkdir()
    r = subprocess.run([str(exe), str(out)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.stdout + r.stderr)[-2000:]
    return sorted(out.glob("*.cu"))


def test_every_kind_is_generated(sources):
    names = {p.name for p in sources}
    assert len(names) == 30
    assert "quadruped_fst_jit_eval_mixed.cu" in names and "floating_fst_jit_aba_derivs.cu" in names


def test_specialised_kernels_compile_with_nvrtc(sources):
    nvrtc = pytest.importorskip("cuda.bindings.nvrtc")
    opts = [o.encode() for o in OPTS + [f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}"]]

    def compile_one(p):
        err, prog = nvrtc.nvrtcCreateProgram(p.read_bytes(), b"fst_jit.cu", 0, [], [])
        if err != nvrtc.nvrtcResult.NVRTC_SUCCESS:
            return f"{p.name}: nvrtcCreateProgram {err}"
        msg = None
        if nvrtc.nvrtcCompileProgram(prog, len(opts), opts)[0] != nvrtc.nvrtcResult.NVRTC_SUCCESS:
            _, n = nvrtc.nvrtcGetProgramLogSize(prog)
            log = b" " * n
            nvrtc.nvrtcGetProgramLog(prog, log)
            msg = f"{p.name}: {log.decode(errors='replace')[-1500:]}"
        nvrtc.nvrtcDestroyProgram(prog)
        return msg

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        failed = [m for m in ex.map(compile_one, sources) if m]
    assert not failed, "\n".join(failed)
