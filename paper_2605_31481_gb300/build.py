"""Builds libfst.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel; an object is rebuilt only when
its source, one of the shared headers or the flags changed. Usage:

    python -m paper_2605_31481_gb300.build [--verbose-ptxas] [--force]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfst.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-Xcompiler", "-Wall"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfst.so")


# Device headers embedded into the library for run-time specialisation
# (NVRTC compiles them again for one fixed tree; see csrc/jit.cpp).
JIT_HEADERS = ["fst_layout.h", "fst_device.cuh", "ops.cuh", "adjoint.cuh", "derivs.cuh", "level.cuh", "pathpar.cuh", "jit_kernels.cuh"]
EMBED = "jit_embed.cpp"


def _gen_embed() -> str:
    parts = ["// generated by build.py: device headers for run-time specialisation", "namespace fst {",
             f"extern const int kJitHeaderCount = {len(JIT_HEADERS)};",
             "extern const char* const kJitHeaderNames[] = {" + ", ".join(f'"{h}"' for h in JIT_HEADERS) + "};",
             "extern const char* const kJitHeaderSources[] = {"]
    for h in JIT_HEADERS:
        with open(os.path.join(CSRC, h)) as fh:
            text = fh.read()
        if ")fst_embed\"" in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        parts.append('R"fst_embed(' + text + ')fst_embed",')
    parts += ["};", "}  // namespace fst", ""]
    src = "\n".join(parts)
    path = os.path.join(BUILD, EMBED)
    if not os.path.exists(path) or open(path).read() != src:
        with open(path, "w") as fh:
            fh.write(src)
    return path


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    return h.hexdigest()


def _compile(nvcc, src, flags, hdr, force):
    path = os.path.join(BUILD if src == EMBED else CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    stamp = obj + ".stamp"
    with open(path, "rb") as fh:
        key = hashlib.sha256(fh.read() + hdr.encode() + " ".join(flags).encode()).hexdigest()
    if not force and os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == key:
        return src, None, False
    cmd = [nvcc, *ARCH, *flags, "-I", INCLUDE, "-I", CSRC, "-c", path, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc, *flags, "-I", INCLUDE, "-I", CSRC, "-x", "c++", "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    with open(stamp, "w") as fh:
        fh.write(key)
    return src, (r.stdout + r.stderr).strip(), True


def build(verbose_ptxas: bool = False, force: bool = False, quiet: bool = False) -> str:
    nvcc = nvcc_path()
    os.makedirs(BUILD, exist_ok=True)
    flags = list(NVCC_FLAGS)
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]
    hdr = _headers_digest()
    _gen_embed()
    srcs = _sources() + [EMBED]
    changed = False
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        for src, log, did in ex.map(lambda s: _compile(nvcc, s, flags, hdr, force), srcs):
            changed |= did
            if log and (verbose_ptxas or not quiet):
                print(f"[{src}]\n{log}", file=sys.stderr)
    if changed or force or not os.path.exists(LIB):
        objs = [os.path.join(BUILD, s + ".o") for s in srcs]
        tmp = LIB + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--verbose-ptxas", action="store_true")
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    print(build(verbose_ptxas=a.verbose_ptxas, force=a.force))


if __name__ == "__main__":
    main()
