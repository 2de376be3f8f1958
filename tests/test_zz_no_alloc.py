"""fst_rnea_vjp_noalloc, the RNEA adjoint for callers that cannot allocate
device memory (memory owned by a pool or arena, real-time loops that may not
call cudaMalloc, plugins that only see their tensors): it must give the same
cotangents as fst_rnea_vjp with a caller-provided scratch buffer, and the
oracle's, call after call, although every call reuses the library's one
built-in scratch array.

This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from oracle import derivs, rbd
from paper_2605_31481_gb300 import workloads as w

pytestmark = pytest.mark.gpu

TOL = 2e-4          # the adjoint parity bar of the other adjoint tests


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


def _env_err(gpu_soa, ref):
    g = np.moveaxis(gpu_soa.double().cpu().numpy(), -1, 0).reshape(ref.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    return (np.abs(g - r).max(1) / np.maximum(np.abs(r).max(1), 1.0)).max()


def _noalloc(L, torch, m, B, q, qd, qdd, tb, like, theta=None):
    out = {k: torch.full_like(v, float("nan")) for k, v in like.items()}
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.fst_rnea_vjp_noalloc(m.handle, B, q.data_ptr(), qd.data_ptr(), qdd.data_ptr(),
                                None if theta is None else theta.data_ptr(), tb.data_ptr(), out["q"].data_ptr(),
                                out["qd"].data_ptr(), out["qdd"].data_ptr(), out["theta"].data_ptr(), stream)
    assert st == 0, L.fst_last_error().decode()
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_allocating_entry_point_twice(setup):
    torch, _ffi, api = setup
    L = _ffi.lib()
    tree = w.spined_quadruped(seed=0)
    B = 4096 + 5
    s = w.random_state(tree, B, seed=21)
    m = api.Model(tree)
    q, qd, qdd, tb = (_t(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ref = api.rnea_vjp(m, q, qd, qdd, tb)
    for call in range(2):
        out = _noalloc(L, torch, m, B, q, qd, qdd, tb, ref)
        for k in ("q", "qd", "qdd", "theta"):
            assert _err(out[k], ref[k]) <= TOL, (call, k)


def test_noalloc_matches_oracle_after_a_larger_call(setup):
    """A call on a bigger tree and batch leaves more of the shared array
    written than the next, smaller call reads; the smaller call must not see
    any of it. Then a call with a theta override. Each against the oracle
    and against fst_rnea_vjp."""
    torch, _ffi, api = setup
    L = _ffi.lib()
    cases = [(w.humanoid(seed=0), 20000, None), (w.spined_quadruped(seed=0), 333, None),
             (w.spined_quadruped(seed=0), 333, 0.2)]
    for tree, B, pert in cases:
        s = w.random_state(tree, B, seed=5)
        rng = np.random.default_rng(3)
        tbn = rng.standard_normal((B, tree.nv))
        m = api.Model(tree)
        th = None
        th_np = rbd.Model(tree).theta()
        if pert:
            th_np = th_np * (1 + rng.uniform(-pert, pert, th_np.shape))
            th = torch.from_numpy(th_np.astype(np.float32)).cuda()
        q, qd, qdd, tb = (_t(x, torch) for x in (s["q"], s["qd"], s["qdd"], tbn))
        ref = api.rnea_vjp(m, q, qd, qdd, tb, theta=th)
        out = _noalloc(L, torch, m, B, q, qd, qdd, tb, ref, theta=th)
        for k in ("q", "qd", "qdd", "theta"):
            assert _err(out[k], ref[k]) <= TOL, (tree.name, B, k)
        idx = np.unique(np.r_[np.random.default_rng(1).choice(B, min(B, 64), replace=False), 0, B - 1])
        rq, rqd, rqdd, _ = derivs.rnea_vjp(tree, s["q"][idx], s["qd"][idx], s["qdd"][idx], tbn[idx], theta=th_np)
        for k, r in (("q", rq), ("qd", rqd), ("qdd", rqdd)):
            e = _env_err(out[k][..., idx], r)
            assert e <= TOL, (tree.name, B, k, e)
        if B <= 400:   # theta_bar over the whole batch through the regressor
            Y = derivs.regressor(tree, s["q"], s["qd"], s["qdd"])
            rth = np.einsum("bi,bink->nk", tbn, Y)
            g = out["theta"].double().cpu().numpy()
            assert np.abs(g - rth).max() / np.abs(rth).max() <= TOL, (tree.name, B)


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


def test_noalloc_applies_the_common_argument_checks(setup):
    """The checks every entry point makes, before anything is launched: B
    beyond 2^31 - 1 is refused even without theta_bar (no scratch limit
    applies then), and null inputs are refused."""
    torch, _ffi, api = setup
    L = _ffi.lib()
    tree = w.spined_quadruped(seed=0)
    m = api.Model(tree)
    x = torch.zeros((tree.nv, 8), device="cuda")
    st = L.fst_rnea_vjp_noalloc(m.handle, (1 << 31) + 5, x.data_ptr(), x.data_ptr(), x.data_ptr(), None,
                                x.data_ptr(), x.data_ptr(), None, None, None, None)
    assert st == -1 and "2^31" in L.fst_last_error().decode()
    st = L.fst_rnea_vjp_noalloc(m.handle, 8, None, x.data_ptr(), x.data_ptr(), None, x.data_ptr(),
                                x.data_ptr(), None, None, None, None)
    assert st == -1 and "null" in L.fst_last_error().decode()
    st = L.fst_rnea_vjp_noalloc(None, 8, x.data_ptr(), x.data_ptr(), x.data_ptr(), None, x.data_ptr(),
                                x.data_ptr(), None, None, None, None)
    assert st == -1
    # B = 0: nothing to launch; theta_bar is still overwritten with zeros
    th = torch.full((tree.n_bodies, 10), 7.0, device="cuda")
    st = L.fst_rnea_vjp_noalloc(m.handle, 0, None, None, None, None, None, None, None, None, th.data_ptr(),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == 0 and float(th.abs().max()) == 0.0
