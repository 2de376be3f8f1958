"""System identification through the fused loss-gradient kernel (paper
Sec. 4.3): the loss it reports equals the oracle's, and Adam on the 70
parameters of the 7-DOF chain drives the loss down and the masses of the
well-excited distal links toward the truth."""
import numpy as np
import pytest

from oracle import rbd
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import to_soa_cuda

pytestmark = pytest.mark.gpu


def test_identification_recovers_masses(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    from paper_2605_31481_gb300 import api, sysid
    tree = w.chain(7, seed=0)
    B = 8192
    s = w.random_state(tree, B, seed=1)
    rng = np.random.default_rng(3)
    true = rbd.Model(tree).theta()
    tau_meas = rbd.rnea(tree, s["q"], s["qd"], s["qdd"]) * (1 + 0.05 * rng.standard_normal((B, tree.nv)))
    theta0 = true * (1 + rng.uniform(-0.3, 0.3, true.shape))
    m = api.Model(tree)
    q, qd, qdd, tm = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], tau_meas))
    th0 = torch.from_numpy(theta0.astype(np.float32)).cuda()
    # the model's own parameters match the oracle's conversion of the table
    assert np.abs(m.theta().cpu().numpy() - true).max() <= 1e-6 * np.abs(true).max()
    theta, losses = sysid.identify(m, q, qd, qdd, tm, th0, steps=500, history=True)
    r0 = rbd.rnea(tree, s["q"], s["qd"], s["qdd"], theta=theta0) - tau_meas
    assert abs(losses[0] - np.sum(r0 * r0)) / np.sum(r0 * r0) < 1e-4
    assert losses[-1] < 0.2 * losses[0]
    err = sysid.mass_errors(theta, true)
    err0 = sysid.mass_errors(theta0, true)
    assert err[3:].mean() < err0[3:].mean()



def test_least_squares_identification_matches_the_oracle_normal_equations():
    """identify_least_squares returns the minimiser of the quadratic loss:
    the same pseudo-inverse step computed in FP64 from the oracle's
    regressor, and the loss there is no larger than at the truth."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import derivs
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    from paper_2605_31481_gb300 import api, sysid
    tree = w.chain(7, seed=0)
    B = 4096
    s = w.random_state(tree, B, seed=2)
    rng = np.random.default_rng(5)
    true = rbd.Model(tree).theta()
    tau_meas = rbd.rnea(tree, s["q"], s["qd"], s["qdd"]) * (1 + 0.05 * rng.standard_normal((B, tree.nv)))
    theta0 = true * (1 + rng.uniform(-0.3, 0.3, true.shape))
    m = api.Model(tree)
    q, qd, qdd, tm = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], tau_meas))
    th0 = torch.from_numpy(theta0.astype(np.float32)).cuda()
    theta, loss = sysid.identify_least_squares(m, q, qd, qdd, tm, th0)
    theta = theta.cpu().numpy().astype(np.float64)
    # oracle: same scaled normal equations in FP64
    Y = derivs.regressor(tree, s["q"], s["qd"], s["qdd"]).reshape(B * tree.nv, -1) * theta0.reshape(-1)
    H = 2 * Y.T @ Y
    g = 2 * Y.T @ (Y @ np.ones(Y.shape[1]) - tau_meas.reshape(-1))
    lam, V = np.linalg.eigh(H)
    keep = lam > 1e-5 * np.abs(lam).max()
    step = V[:, keep] @ ((V[:, keep].T @ g) / lam[keep])
    ref = ((1 - step) * theta0.reshape(-1)).reshape(theta0.shape)
    # identifiable combinations agree: compare the predicted torques
    Yu = derivs.regressor(tree, s["q"], s["qd"], s["qdd"]).reshape(B * tree.nv, -1)
    pred, pred_ref = Yu @ theta.reshape(-1), Yu @ ref.reshape(-1)
    assert np.abs(pred - pred_ref).max() <= 1e-3 * np.abs(pred_ref).max()
    r_true = rbd.rnea(tree, s["q"], s["qd"], s["qdd"]) - tau_meas
    assert loss <= np.sum(r_true * r_true) * (1 + 1e-4)
    assert sysid.mass_errors(theta, true)[3:].mean() < 0.05
