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

