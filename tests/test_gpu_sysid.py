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
    # the step minimises the loss as well as the FP64 one does (FP64 loss)
    Yu = derivs.regressor(tree, s["q"], s["qd"], s["qdd"]).reshape(B * tree.nv, -1)
    L = lambda th: float(np.sum((Yu @ th.reshape(-1) - tau_meas.reshape(-1)) ** 2))
    assert L(theta) <= L(ref) * (1 + 1e-3)
    assert L(ref) <= L(true) and L(theta) < 0.5 * L(theta0)
    assert abs(loss - L(theta)) <= 1e-3 * L(theta)


def test_mass_only_identification_matches_oracle_least_squares():
    """Masses only, centres of mass and rotational inertias known (the
    paper's setting): the kernel-built normal equations give the FP64
    least-squares masses, within a few percent of the truth at 5% noise."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import derivs
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    from paper_2605_31481_gb300 import api, sysid
    tree = w.chain(7, seed=0)
    B = 4096
    s = w.random_state(tree, B, seed=3)
    rng = np.random.default_rng(6)
    true = rbd.Model(tree).theta()
    tau_meas = rbd.rnea(tree, s["q"], s["qd"], s["qdd"]) * (1 + 0.05 * rng.standard_normal((B, tree.nv)))
    m = api.Model(tree)
    q, qd, qdd, tm = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], tau_meas))
    masses, theta = sysid.identify_masses(m, q, qd, qdd, tm, torch.from_numpy(true.astype(np.float32)).cuda())
    masses = masses.cpu().numpy().astype(np.float64)
    # oracle: regressor columns combined along the same mass directions
    c = true[:, 1:4] / true[:, 0:1]
    x, y, z = c.T
    phi = np.concatenate([np.ones((len(c), 1)), c,
                          np.stack([y * y + z * z, -x * y, x * x + z * z, -x * z, -y * z, x * x + y * y], 1)], 1)
    Y = derivs.regressor(tree, s["q"], s["qd"], s["qdd"])                 # (B, nv, n_b, 10)
    A = np.einsum("bink,nk->bin", Y, phi).reshape(B * tree.nv, -1)
    base = np.einsum("bink,nk->bi", Y, true).reshape(-1) - A @ true[:, 0]
    ref, *_ = np.linalg.lstsq(A, tau_meas.reshape(-1) - base, rcond=None)
    np.testing.assert_allclose(masses, ref, rtol=2e-3)
    assert (np.abs(masses - true[:, 0]) / true[:, 0]).mean() < 0.05


def test_identification_checkpoint_and_resume(tmp_path):
    """250 steps, the optimiser state through torch.save / torch.load, 250
    more: bitwise the result of 500 uninterrupted steps."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    from paper_2605_31481_gb300 import api, sysid
    tree = w.chain(7, seed=0)
    B = 2048
    s = w.random_state(tree, B, seed=4)
    rng = np.random.default_rng(9)
    true = rbd.Model(tree).theta()
    tau_meas = rbd.rnea(tree, s["q"], s["qd"], s["qdd"]) * (1 + 0.05 * rng.standard_normal((B, tree.nv)))
    th0 = torch.from_numpy((true * (1 + rng.uniform(-0.3, 0.3, true.shape))).astype(np.float32)).cuda()
    m = api.Model(tree)
    q, qd, qdd, tm = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], tau_meas))
    full, _ = sysid.identify(m, q, qd, qdd, tm, th0, steps=500)
    _, _, st = sysid.identify(m, q, qd, qdd, tm, th0, steps=250, return_state=True)
    torch.save(st, tmp_path / "sysid.pt")
    st = torch.load(tmp_path / "sysid.pt")
    resumed, _ = sysid.identify(m, q, qd, qdd, tm, th0, steps=250, state=st)
    assert torch.equal(full, resumed)
