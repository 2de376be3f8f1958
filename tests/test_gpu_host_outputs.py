"""Outputs in pinned host memory: fst_device_can_access tells which pointers
the device addresses with the same pointer, and the compute calls then write
their results straight to the host, bit-identical to device outputs."""
import ctypes

import numpy as np
import pytest

from paper_2605_31481_gb300 import workloads as w
from tests._helpers import to_soa_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


def _can(L, t):
    ok = ctypes.c_int32(-1)
    assert L.fst_device_can_access(ctypes.c_void_p(t.data_ptr() if t is not None else 0), ctypes.byref(ok)) == 0
    return ok.value


def test_device_can_access_classifies_pointers(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import _ffi
    L = _ffi.lib()
    assert _can(L, torch.empty(16, device="cuda")) == 1
    assert _can(L, torch.empty(16).pin_memory()) == 1
    assert _can(L, torch.empty(16)) == 0                   # pageable host memory: never passed to a kernel
    ok = ctypes.c_int32(-1)
    assert L.fst_device_can_access(None, ctypes.byref(ok)) == 0 and ok.value == 0


def test_fused_step_writes_pinned_host_outputs(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = w.spined_quadruped(seed=0)
    B = 500
    s = w.random_state(tree, B, seed=71)
    m = api.Model(tree)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ee = list(tree.ee)
    ref = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    host = {k: torch.full(tuple(v.shape), float("nan")).pin_memory() for k, v in ref.items()}
    api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True, out=host)
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(host[k], ref[k].cpu()), k
    with pytest.raises(ValueError):                        # pageable host memory is refused
        api.fk(m, q, out=torch.empty(tree.n_bodies, 12, B))
