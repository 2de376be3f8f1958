"""Dense dynamics derivatives through the C ABI (generic and specialised
kernels) against the FP64 oracle's complex-step derivatives along the same
tangent directions."""
import numpy as np
import pytest

from oracle import derivs, rbd
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import solve_backward_err, to_soa_cuda
from tests.test_gpu_parity import TREES

pytestmark = pytest.mark.gpu

DTOL = 2e-4      # per-environment normwise relative error of d tau / d (q, qd)
BWD_BAR = 1e-5   # normwise backward error of the M^-1 products (forward-dynamics derivatives): ~150 FP32 roundings
COND_MAX = 1e3   # forward-error checks of M^-1 products only where cond(M) is below this
FWD_BAR = 2e-3   # = COND_MAX x 2e-6, a backward error of about 30 FP32 roundings


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
    """d qdd / d (q, qd, tau) = -M^-1 d tau / d (q, qd) at qdd, and M^-1:
    products with M^-1, checked by their backward error, which a stable FP32
    solve keeps small whatever cond(M) is:
      ||M G_x + D_x|| <= BWD_BAR (||M|| ||G_x|| + ||D_x||)   for x = q, qd
      ||M G_tau - I|| <= BWD_BAR (||M|| ||G_tau|| + 1)
    with the oracle's FP64 M and D_x = d tau / d x evaluated at the kernel's
    own forward result qdd (which the call returns). The forward error
    against the oracle's complex-step derivatives is held to FWD_BAR only
    where cond(M) < COND_MAX."""
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
    M = rbd.crba(tree, s["q"])
    qdd_k = np.moveaxis(res["qdd"].cpu().numpy().astype(np.float64), -1, 0)
    Dq, Dqd = derivs.rnea_derivatives(tree, s["q"], s["qd"], qdd_k)
    eye = np.broadcast_to(np.eye(tree.nv), M.shape)
    meas = {}
    for key, rhs in (("q", -Dq), ("qd", -Dqd), ("tau", eye)):
        bwd = solve_backward_err(M, _mat(res[key]), rhs)
        meas["d qdd/d " + key + " backward"] = float(bwd.max())
        assert bwd.max() <= BWD_BAR, f"{name} d qdd / d {key}: backward error {bwd.max():.3e}"
    good = np.linalg.cond(M) < COND_MAX
    if good.any():
        idx = np.flatnonzero(good)
        rq, rqd, rtau = derivs.aba_derivatives(tree, s["q"][idx], s["qd"][idx], s["tau"][idx])
        for key, ref in (("q", rq), ("qd", rqd), ("tau", rtau)):
            err = _err(_mat(res[key])[idx], ref)
            meas["d qdd/d " + key + " forward (cond<1e3)"] = float(err.max())
            assert err.max() <= FWD_BAR, f"{name} d qdd / d {key}: forward error {err.max():.3e}"
    print(f"aba_derivatives {name} spec={specialize}: " + ", ".join(f"{k} {v:.2e}" for k, v in meas.items()))
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
