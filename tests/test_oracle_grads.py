"""Pins of the oracle's reference gradients: complex-step derivatives against
central finite differences (h = 1e-6), the regressor against the definition
of linearity, and exact identities (d tau / d qdd = M, d qdd / d tau = M^-1)."""
import numpy as np
import pytest

from oracle import rbd, derivs
from paper_2605_31481_gb300 import workloads as w


def _fd(f, xs, k, dx, h=1e-6):
    xp = [np.array(x, dtype=np.float64) for x in xs]
    xm = [np.array(x, dtype=np.float64) for x in xs]
    xp[k] = xp[k] + h * dx
    xm[k] = xm[k] - h * dx
    return (f(*xp) - f(*xm)) / (2 * h)


@pytest.mark.parametrize("tree", [w.chain(7), w.spined_quadruped(), w.humanoid()], ids=lambda t: t.name)
def test_complex_step_matches_central_differences(tree):
    s = w.random_state(tree, 6, seed=11)
    rng = np.random.default_rng(0)
    args = (s["q"], s["qd"], s["qdd"])
    for k in range(3):
        dx = rng.standard_normal(args[k].shape)
        cs = derivs.jvp_cs(lambda a, b, c: rbd.rnea(tree, a, b, c), args, k, dx)
        fd = _fd(lambda a, b, c: rbd.rnea(tree, a, b, c), args, k, dx)
        assert np.abs(cs - fd).max() < 1e-6 * max(1, np.abs(cs).max())
    args = (s["q"], s["qd"], s["tau"])
    for k in range(3):
        dx = rng.standard_normal(args[k].shape)
        cs = derivs.jvp_cs(lambda a, b, c: rbd.aba(tree, a, b, c), args, k, dx)
        fd = _fd(lambda a, b, c: rbd.aba(tree, a, b, c), args, k, dx)
        assert np.abs(cs - fd).max() < 1e-5 * max(1, np.abs(cs).max())


def test_regressor_reproduces_tau_and_fd():
    tree = w.chain(7)
    s = w.random_state(tree, 5, seed=12)
    Y = derivs.regressor(tree, s["q"], s["qd"], s["qdd"])
    th = rbd.Model(tree).theta()
    tau = rbd.rnea(tree, s["q"], s["qd"], s["qdd"])
    assert np.abs(np.einsum("bink,nk->bi", Y, th) - tau).max() < 1e-12
    # d tau / d theta by central differences in theta
    rng = np.random.default_rng(1)
    d = rng.standard_normal(th.shape)
    h = 1e-6
    fd = (rbd.rnea(tree, s["q"], s["qd"], s["qdd"], theta=th + h * d)
          - rbd.rnea(tree, s["q"], s["qd"], s["qdd"], theta=th - h * d)) / (2 * h)
    assert np.abs(np.einsum("bink,nk->bi", Y, d) - fd).max() < 1e-7


def test_exact_identities_of_the_vjps():
    tree = w.spined_quadruped()
    s = w.random_state(tree, 4, seed=13)
    rng = np.random.default_rng(2)
    tau_bar = rng.standard_normal(s["tau"].shape)
    M = rbd.crba(tree, s["q"])
    qb, qdb, qddb, thb = derivs.rnea_vjp(tree, s["q"], s["qd"], s["qdd"], tau_bar)
    assert np.abs(qddb - np.einsum("bij,bi->bj", M, tau_bar)).max() < 1e-12
    qdd = rbd.aba(tree, s["q"], s["qd"], s["tau"])
    qdd_bar = rng.standard_normal(qdd.shape)
    aq, aqd, atau, ath = derivs.aba_vjp(tree, s["q"], s["qd"], s["tau"], qdd_bar)
    lam = np.linalg.solve(M, qdd_bar[..., None])[..., 0]
    assert np.abs(atau - lam).max() < 1e-10
    # implicit-function identity: ABA cotangents = -RNEA cotangents at (qdd, lam)
    rq, rqd, _, rth = derivs.rnea_vjp(tree, s["q"], s["qd"], qdd, lam)
    assert np.abs(aq + rq).max() < 1e-9 * max(1, np.abs(rq).max())
    assert np.abs(aqd + rqd).max() < 1e-9 * max(1, np.abs(rqd).max())
    assert np.abs(ath + rth).max() < 1e-9 * max(1, np.abs(rth).max())


def test_fk_vjp_matches_fd():
    tree = w.humanoid()
    s = w.random_state(tree, 3, seed=14)
    rng = np.random.default_rng(3)
    pb = rng.standard_normal((3, tree.n_bodies, 12))
    qb = derivs.fk_vjp(tree, s["q"], pb)
    d = rng.standard_normal(s["q"].shape)

    def flat(q_):
        T = rbd.fk(tree, q_)
        return np.concatenate([T[..., :3, :3].reshape(T.shape[:2] + (9,)), T[..., :3, 3]], -1)

    fd = _fd(flat, (s["q"],), 0, d)
    assert np.abs(np.einsum("bnk,bnk->b", pb, fd) - np.einsum("bj,bj->b", qb, d)).max() < 1e-6
