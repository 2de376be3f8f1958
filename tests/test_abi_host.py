"""Host-only checks of the C ABI: the library loads, exports every entry
point include/fst.h declares, and rejects bad body tables with the right
status before touching CUDA. No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_31481_gb300 import _ffi
from paper_2605_31481_gb300 import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_names():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"FST_API\s+[\w\s\*]+?\b(fst_\w+)\s*\(", src)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return _ffi.lib()


def test_library_exports_every_declared_symbol(lib):
    names = _header_names()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    # and the binding declares exactly the header's entry points
    assert sorted(names) == sorted(_ffi.exported_names())


def _desc(tree):
    n = tree.n_bodies
    arr = (_ffi.BodyDesc * n)()
    for i in range(n):
        d = arr[i]
        d.parent, d.type = int(tree.parent[i]), int(tree.jtype[i])
        for k in range(3):
            d.axis[k], d.com[k] = tree.axis[i][k], tree.com[i][k]
        for k in range(12):
            d.T_joint[k], d.T_link[k] = tree.T_joint[i][k], tree.T_link[i][k]
        d.mass = tree.mass[i]
        for k in range(6):
            d.I_com[k] = tree.I_com[i][k]
    return arr


def _create(lib, tree, n=None):
    arr = _desc(tree)
    g = (ctypes.c_double * 3)(0, 0, -9.81)
    h = ctypes.c_void_p()
    st = lib.fst_model_create(arr, tree.n_bodies if n is None else n, g, ctypes.byref(h))
    if st == 0:
        lib.fst_model_destroy(h)
    return st, lib.fst_last_error().decode()


@pytest.mark.parametrize("mutate,status", [
    (lambda t: t.parent.__setitem__(2, 2), -2),          # own index as parent
    (lambda t: t.parent.__setitem__(1, 5), -2),          # parent after child
    (lambda t: t.parent.__setitem__(0, -3), -2),
    (lambda t: t.jtype.__setitem__(1, 9), -4),           # unknown joint type
    (lambda t: t.jtype.__setitem__(2, w.FREE), -2),      # free joint off the root
    (lambda t: t.mass.__setitem__(1, -1.0), -3),
    (lambda t: t.I_com.__setitem__(1, [1, 5, 1, 0, 0, 1]), -3),   # not PSD
    (lambda t: t.mass.__setitem__(1, np.nan), -3),
    (lambda t: t.axis.__setitem__(1, [0, 0, 0]), -1),    # zero axis
    (lambda t: t.T_joint.__setitem__(1, np.r_[2 * np.eye(3).ravel(), 0, 0, 0]), -1),  # not a rotation
], ids=["self-parent", "forward-parent", "bad-parent", "bad-type", "free-not-root", "neg-mass",
        "non-psd", "nan-mass", "zero-axis", "non-rotation"])
def test_model_create_rejects_bad_tables(lib, mutate, status):
    t = w.chain(5, seed=0)
    mutate(t)
    st, msg = _create(lib, t)
    assert st == status, msg
    assert msg.startswith("fst_model_create")


def test_model_create_limits(lib):
    t = w.chain(5, seed=0)
    assert _create(lib, t, n=0)[0] == -1
    big = w.chain(65, seed=0)
    assert _create(lib, big)[0] == -4


def test_free_joint_requires_identity_link(lib):
    t = w.humanoid(seed=0)
    t.T_link[0, 9] = 0.1
    assert _create(lib, t)[0] == -4


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.fst_model_create(None, 3, None, ctypes.byref(h)) == -1
    assert lib.fst_rnea(None, 10, None, None, None, None, None, None) == -1
    assert lib.fst_model_destroy(None) == 0
    assert lib.fst_version().decode().startswith("fst")


def test_valid_table_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, msg = _create(lib, w.spined_quadruped())
    assert st == -5 and "fst_model_create" in msg


def test_batch_size_bounds_are_checked_before_the_model_is_used(lib):
    """B < 0 and B > 2^31 - 1 are refused and B = 0 does nothing, all before
    the call reads the model, its device or any array (so an opaque stand-in
    handle suffices here)."""
    stand_in = ctypes.create_string_buffer(4096)
    h = ctypes.cast(stand_in, ctypes.c_void_p)
    for B in (-1, 2**31, 2**40):
        assert lib.fst_fk(h, ctypes.c_int64(B), None, None, None) == -1
        assert "B must" in lib.fst_last_error().decode()
        assert lib.fst_rnea(h, ctypes.c_int64(B), None, None, None, None, None, None) == -1
    assert lib.fst_fk(h, ctypes.c_int64(0), None, None, None) == 0


def test_plain_c_caller_compiles_links_and_reports_status(lib, tmp_path):
    """include/fst.h serves a C program (ISO C11, warnings as errors); run
    without a GPU, the example stops at model creation with FST_ERR_CUDA and
    the library's message."""
    import shutil
    import subprocess
    import torch
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if shutil.which("gcc") is None or not os.path.isdir(os.path.join(cuda, "include")):
        pytest.skip("needs gcc and the CUDA headers")
    pkg = os.path.dirname(_ffi.LIB_PATH)
    exe = str(tmp_path / "abi_example")
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        f"-I{os.path.join(ROOT, 'include')}", f"-I{cuda}/include",
                        os.path.join(ROOT, "tests", "host", "abi_example.c"), f"-L{pkg}", "-lfst",
                        f"-L{cuda}/lib64", "-lcudart", f"-Wl,-rpath,{pkg}", "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    if torch.cuda.is_available():
        return                                     # the GPU run belongs to the parity tests
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 1 and "fst_model_create" in r.stderr and "(-5)" in r.stderr
