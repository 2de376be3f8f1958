"""Dense dynamics derivatives through the C ABI (generic and specialised
kernels) against the FP64 oracle's complex-step derivatives along the same
tangent directions."""
import numpy as np
import pytest

from oracle import derivs, rbd
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import to_soa_cuda
from tests.test_gpu_parity import TREES

pytestmark = pytest.mark.gpu

DTOL = 2e-4      # per-environment normwise relative error of d tau / d (q, qd)
ATOL_FD = 2e-3   # forward-dynamics derivatives compose an M^-1 solve


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


def _mat(t):
    """(nv, nv, B) device tensor -> (B, nv, nv) numpy."""
    return np.moveaxis(t.cpu().numpy().astype(np.float64), -1, 0)


def _err(g, r):
    B = g.shape[0]
    g, r = g.reshape(B, -1), r.reshape(B, -1)
    return np.abs(g - r).max(1) / np.maximum(np.abs(r).max(1), 1.0)


@pytest.mark.parametrize("specialize", [False, True])
@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8", "urdf_arm6_tool"])
def test_rnea_derivatives_match_oracle(torch_cuda, name, specialize):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 70                                            # two tiles of 32 and a tail
    s = w.random_state(tree, B, seed=31)
    m = api.Model(tree, specialize=["rnea_derivatives"] if specialize else None)
    q, qd, qdd = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd"))
    res = api.rnea_derivatives(m, q, qd, qdd)
    only_qd = api.rnea_derivatives(m, q, qd, qdd, dq=False)
    torch.cuda.synchronize()
    rq, rqd = derivs.rnea_derivatives(tree, s["q"], s["qd"], s["qdd"])
    eq, eqd = _err(_mat(res["q"]), rq), _err(_mat(res["qd"]), rqd)
    assert eq.max() <= DTOL, f"{name} dtau/dq {eq.max():.3e}"
    assert eqd.max() <= DTOL, f"{name} dtau/dqd {eqd.max():.3e}"
    assert set(only_qd) == {"qd"} and torch.equal(only_qd["qd"], res["qd"])


@pytest.mark.parametrize("specialize", [False, True])
@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "urdf_arm6_tool"])
def test_aba_derivatives_match_oracle(torch_cuda, name, specialize):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 45
    s = w.random_state(tree, B, seed=32)
    m = api.Model(tree, specialize=["aba_derivatives"] if specialize else None)
    q, qd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "tau"))
    res = api.aba_derivatives(m, q, qd, tau, qdd=True)
    qdd_ref = api.aba(m, q, qd, tau)
    torch.cuda.synchronize()
    rq, rqd, rtau = derivs.aba_derivatives(tree, s["q"], s["qd"], s["tau"])
    M = rbd.crba(tree, s["q"])
    cond = np.linalg.cond(M)
    for key, ref in (("q", rq), ("qd", rqd), ("tau", rtau)):
        err = _err(_mat(res[key]), ref)
        # forward error of an M^-1 product grows with cond(M): scale the bar
        bar = ATOL_FD * np.maximum(cond / 1e3, 1.0)
        assert np.all(err <= bar), f"{name} d qdd / d {key}: {err.max():.3e}"
    np.testing.assert_allclose(res["qdd"].cpu().numpy(), qdd_ref.cpu().numpy(), rtol=1e-5,
                               atol=1e-5 * float(qdd_ref.abs().max()))
    Minv = _mat(res["tau"])
    np.testing.assert_allclose(Minv, np.swapaxes(Minv, 1, 2), rtol=0, atol=1e-6 * np.abs(Minv).max())


def test_derivative_edge_cases(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, _ffi
    tree = TREES["chain7"]()
    m = api.Model(tree)
    z = torch.empty(7, 0, device="cuda")
    assert api.rnea_derivatives(m, z, z, z)["q"].shape == (7, 7, 0)
    assert api.aba_derivatives(m, z, z, z)["tau"].shape == (7, 7, 0)
    s = w.random_state(tree, 1, seed=2)
    q, qd, qdd = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd"))
    one = api.rnea_derivatives(m, q, qd, qdd)
    torch.cuda.synchronize()
    rq, _ = derivs.rnea_derivatives(tree, s["q"], s["qd"], s["qdd"])
    assert _err(_mat(one["q"]), rq).max() <= DTOL
    # Minv is required (it is the factorisation's workspace)
    rc = _ffi.lib().fst_aba_derivatives(m.handle, 1, q.data_ptr(), qd.data_ptr(), qdd.data_ptr(), None, None, None,
                                        None, None, None)
    assert rc == -1
