"""fst_rnea_vjp_noalloc, the RNEA adjoint for callers that cannot allocate
device memory (memory owned by a pool or arena, real-time loops that may not
call cudaMalloc, plugins that only see their tensors): it must give the same
cotangents as fst_rnea_vjp with a caller-provided scratch buffer, call after
call, although every call reuses the library's one built-in scratch array.

This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2605_31481_gb300 import workloads as w

pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build, _ffi, api
    build.build(quiet=True)
    return torch, _ffi, api


def _t(x, torch):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float32).T)).cuda()


def _err(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1.0)


def test_noalloc_matches_allocating_entry_point_twice(setup):
    torch, _ffi, api = setup
    L = _ffi.lib()
    tree = w.spined_quadruped(seed=0)
    B = 4096 + 5
    s = w.random_state(tree, B, seed=21)
    m = api.Model(tree)
    q, qd, qdd, tb = (_t(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ref = api.rnea_vjp(m, q, qd, qdd, tb)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = {"q": torch.full_like(ref["q"], float("nan")), "qd": torch.full_like(ref["qd"], float("nan")),
               "qdd": torch.full_like(ref["qdd"], float("nan")),
               "theta": torch.full_like(ref["theta"], float("nan"))}
        st = L.fst_rnea_vjp_noalloc(m.handle, B, q.data_ptr(), qd.data_ptr(), qdd.data_ptr(), None, tb.data_ptr(),
                                    out["q"].data_ptr(), out["qd"].data_ptr(), out["qdd"].data_ptr(),
                                    out["theta"].data_ptr(), stream)
        assert st == 0, L.fst_last_error().decode()
        torch.cuda.synchronize()
        for k in ("q", "qd", "qdd", "theta"):
            assert _err(out[k], ref[k]) <= TOL, (call, k)


def test_noalloc_rejects_batches_beyond_its_scratch(setup):
    torch, _ffi, api = setup
    L = _ffi.lib()
    tree = w.spined_quadruped(seed=0)
    m = api.Model(tree)
    x = torch.zeros((tree.nv, 8), device="cuda")
    th = torch.zeros((tree.n_bodies, 10), device="cuda")
    B = 1 << 22                                  # far beyond 4 MiB of partial sums
    st = L.fst_rnea_vjp_noalloc(m.handle, B, x.data_ptr(), x.data_ptr(), x.data_ptr(), None, x.data_ptr(),
                                None, None, None, th.data_ptr(), None)
    assert st == -1
    assert "scratch" in L.fst_last_error().decode()
