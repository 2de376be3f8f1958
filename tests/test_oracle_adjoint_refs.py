"""Pins of the oracle's reference adjoints of the Jacobian and of the mass
matrix: central differences of the pinned forward functions, and the
linearity of M in the inertial parameters."""
import numpy as np
import pytest

from oracle import derivs, rbd
from paper_2605_31481_gb300 import workloads as w


@pytest.mark.parametrize("make", [lambda: w.spined_quadruped(seed=0), lambda: w.humanoid(seed=0)],
                         ids=["quadruped11", "humanoid29"])
def test_jacobian_vjp_matches_central_differences(make):
    tree = make()
    s = w.random_state(tree, 4, seed=3)
    links = list(tree.ee)[:2]
    rng = np.random.default_rng(0)
    Jb = rng.standard_normal((4, len(links), 6, tree.nv))
    qb = derivs.jacobian_vjp(tree, s["q"], links, Jb)
    L = lambda q_: np.einsum("blrc,blrc->b", Jb, np.stack([rbd.jacobian(tree, q_, l) for l in links], 1))
    h = 1e-6
    for j in range(tree.nq):
        e = np.zeros_like(s["q"])
        e[:, j] = h
        fd = (L(s["q"] + e) - L(s["q"] - e)) / (2 * h)
        assert np.abs(qb[:, j] - fd).max() <= 1e-6 * max(np.abs(fd).max(), 1.0), j


@pytest.mark.parametrize("make", [lambda: w.chain(7, seed=0), lambda: w.humanoid(seed=0)], ids=["chain7", "humanoid29"])
def test_crba_vjp_matches_central_differences_and_linearity(make):
    tree = make()
    s = w.random_state(tree, 3, seed=5)
    rng = np.random.default_rng(1)
    Mb = rng.standard_normal((3, tree.nv, tree.nv))
    th = rbd.Model(tree).theta() * (1 + rng.uniform(-0.2, 0.2, (tree.n_bodies, 10)))
    qb, thb = derivs.crba_vjp(tree, s["q"], Mb, theta=th)
    L = lambda q_, th_: np.sum(Mb * rbd.crba(tree, q_, theta=th_), axis=(1, 2))
    h = 1e-6
    for j in range(tree.nq):
        e = np.zeros_like(s["q"])
        e[:, j] = h
        fd = (L(s["q"] + e, th) - L(s["q"] - e, th)) / (2 * h)
        assert np.abs(qb[:, j] - fd).max() <= 1e-6 * max(np.abs(fd).max(), 1.0), j
    # M is linear in theta: sum M_bar : M(theta) = theta_bar . theta
    assert abs(np.sum(thb * th) - L(s["q"], th).sum()) <= 1e-10 * abs(L(s["q"], th).sum())
    d = rng.standard_normal(th.shape)
    fd = (L(s["q"], th + 1e-6 * d) - L(s["q"], th - 1e-6 * d)).sum() / 2e-6
    assert abs(np.sum(thb * d) - fd) <= 1e-6 * max(abs(fd), 1.0)
