"""The host-side model builder and the path tables of the specialised
kernels under AddressSanitizer and UndefinedBehaviorSanitizer (CPU only):
random valid trees build and give consistent root-to-leaf path tables, the
per-joint constants (Sec. 3.2, Eq. 2-5) reproduce the plain product of the
joint's poses and its motion subspace is the child frame's twist, and
malformed tables are refused with an error status."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_31481_gb300", "csrc")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_model_builder_and_path_tables_under_sanitizers(tmp_path):
    if shutil.which("g++") is None or not os.path.isdir(os.path.join(CUDA, "include")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "sanitize_model"
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           f"-I{CUDA}/include", f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}",
           os.path.join(ROOT, "tests", "host", "sanitize_model.cpp"), os.path.join(CSRC, "model.cpp"),
           "-o", str(exe), f"-L{CUDA}/lib64", "-lcudart", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, (r.stdout + r.stderr)[-3000:]
    assert r.stdout.startswith("ok")
