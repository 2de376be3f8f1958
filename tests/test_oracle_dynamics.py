"""Pins of the oracle's dynamics (RNEA, CRBA, ABA) to closed forms, an
independent Lagrangian derivation, classical Newton-Euler for a free body,
and invariants any correct implementation must satisfy."""
import json
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import rbd, lagrange
from oracle import spatial as sp
from paper_2605_31481_gb300 import workloads as w

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_fp64_discrepancy.json")))
G0 = 9.81


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1.0)


def test_single_pendulum_closed_form():
    # one revolute joint about y through the origin, COM at (r, 0, 0),
    # gravity along -z: tau = (Iyy + m r^2) qdd - m g r cos q
    t = w.random_tree([-1], [w.REVOLUTE], seed=0)
    t.axis[0] = [0, 1, 0]
    t.T_joint[0, 9:] = 0
    r, m, Iyy = 0.4, 2.5, 0.07
    t.mass[0], t.com[0] = m, [r, 0, 0]
    t.I_com[0] = [0.05, 0.0, Iyy, 0.0, 0.0, 0.06]
    rng = np.random.default_rng(0)
    q, qd, qdd = (rng.uniform(-3, 3, (30, 1)) for _ in range(3))
    tau = rbd.rnea(t, q, qd, qdd)
    expect = (Iyy + m * r * r) * qdd - m * G0 * r * np.cos(q)
    assert np.abs(tau - expect).max() < 1e-13
    M = rbd.crba(t, q)
    assert np.abs(M[:, 0, 0] - (Iyy + m * r * r)).max() < 1e-14
    qdd2 = rbd.aba(t, q, qd, tau)
    assert np.abs(qdd2 - qdd).max() < 1e-12


def test_planar_two_link_closed_form():
    # textbook planar 2R arm in the x-y plane, gravity along -y
    m1, m2, l1, c1, c2, I1, I2 = 1.3, 0.9, 0.6, 0.25, 0.3, 0.04, 0.03
    t = w.random_tree([-1, 0], [w.REVOLUTE] * 2, seed=1)
    t.axis[:] = [0, 0, 1]
    t.T_joint[:, 9:] = 0
    t.T_joint[1, 9] = l1
    t.mass[:] = [m1, m2]
    t.com[:] = [[c1, 0, 0], [c2, 0, 0]]
    t.I_com[:] = [[0.02, 0.001, 0.03, 0.002, 0.003, I1], [0.01, -0.002, 0.02, 0.001, -0.001, I2]]
    t.gravity = np.array([0, -G0, 0])
    rng = np.random.default_rng(2)
    q, qd, qdd = (rng.uniform(-3, 3, (40, 2)) for _ in range(3))
    q1, q2 = q[:, 0], q[:, 1]
    M11 = I1 + I2 + m1 * c1 ** 2 + m2 * (l1 ** 2 + c2 ** 2 + 2 * l1 * c2 * np.cos(q2))
    M12 = I2 + m2 * (c2 ** 2 + l1 * c2 * np.cos(q2))
    M22 = I2 + m2 * c2 ** 2 + 0 * q2
    h = m2 * l1 * c2 * np.sin(q2)
    g1 = (m1 * c1 + m2 * l1) * G0 * np.cos(q1) + m2 * c2 * G0 * np.cos(q1 + q2)
    g2 = m2 * c2 * G0 * np.cos(q1 + q2)
    tau1 = M11 * qdd[:, 0] + M12 * qdd[:, 1] - h * (2 * qd[:, 0] * qd[:, 1] + qd[:, 1] ** 2) + g1
    tau2 = M12 * qdd[:, 0] + M22 * qdd[:, 1] + h * qd[:, 0] ** 2 + g2
    tau = rbd.rnea(t, q, qd, qdd)
    assert np.abs(tau - np.stack([tau1, tau2], -1)).max() < 1e-13
    M = rbd.crba(t, q)
    Mx = np.stack([np.stack([M11, M12], -1), np.stack([M12, M22], -1)], -2)
    assert np.abs(M - Mx).max() < 1e-14


def _mixed_tree(seed):
    t = w.random_tree([-1, 0, 0], [w.REVOLUTE, w.PRISMATIC, w.REVOLUTE], seed)
    rng = np.random.default_rng(seed + 50)
    for i in range(3):
        t.T_joint[i, :9] = Rotation.random(random_state=rng.integers(1 << 30)).as_matrix().ravel()
        t.T_link[i, :9] = Rotation.random(random_state=rng.integers(1 << 30)).as_matrix().ravel()
        t.T_link[i, 9:] = rng.uniform(-0.2, 0.2, 3)
    return t


@pytest.mark.parametrize("make", [
    lambda s: w.random_tree([-1, 0, 1], [w.REVOLUTE] * 3, s),
    lambda s: w.random_tree([-1, 0, 0], [w.REVOLUTE] * 3, s),
    lambda s: w.random_tree([-1, 0, 1], [w.REVOLUTE, w.FIXED, w.PRISMATIC], s),
    _mixed_tree,
], ids=["chain3", "branch3", "rev-fixed-prism", "general-frames"])
@pytest.mark.parametrize("seed", [0, 1])
def test_recursions_match_lagrangian(make, seed):
    t = make(seed)
    s = w.random_state(t, 6, seed=seed + 10)
    M = rbd.crba(t, s["q"])
    Ml = lagrange.mass_matrix(t, s["q"])
    assert _rel(M, Ml) < 1e-13
    tau = rbd.rnea(t, s["q"], s["qd"], s["qdd"])
    taul = lagrange.inverse_dynamics(t, s["q"], s["qd"], s["qdd"])
    assert _rel(tau, taul) < 1e-8          # central differences of M bound this
    g = rbd.rnea(t, s["q"], 0 * s["qd"], 0 * s["qdd"])
    assert _rel(g, lagrange.gravity_torque(t, s["q"])) < 1e-13
    qdd = rbd.aba(t, s["q"], s["qd"], taul)
    assert _rel(qdd, s["qdd"]) < 1e-6


TREES = [w.chain(7), w.spined_quadruped(), w.humanoid(), w.legged(6), w.humanoid(floating=False)]


@pytest.mark.parametrize("tree", TREES, ids=lambda t: t.name)
def test_invariants(tree):
    s = w.random_state(tree, 128, seed=3)
    q, qd, qdd, tau = s["q"], s["qd"], s["qdd"], s["tau"]
    M = rbd.crba(tree, q)
    assert np.abs(M - np.swapaxes(M, 1, 2)).max() <= 10 * GOLD["CRBA"]
    np.linalg.cholesky(M)                                   # positive definite
    # M e_k = RNEA(q, 0, e_k) with gravity off
    z = np.zeros_like(qd)
    for k in range(tree.nv):
        e = np.zeros_like(qd)
        e[:, k] = 1
        col = rbd.rnea(tree, q, z, e, gravity=[0, 0, 0])
        assert np.abs(col - M[:, :, k]).max() < 10 * GOLD["CRBA"] * max(1, np.abs(M).max())
    # ABA inverts RNEA, and equals the Cholesky solve of M qdd = tau - bias
    qdd_a = rbd.aba(tree, q, qd, tau)
    bias = rbd.rnea(tree, q, qd, z)
    qdd_s = np.linalg.solve(M, (tau - bias)[..., None])[..., 0]
    assert _rel(qdd_a, qdd_s) < GOLD["ABA"]
    back = rbd.rnea(tree, q, qd, qdd_a)
    assert _rel(back, tau) < GOLD["ABA"]
    # tau is linear in the inertial parameters
    th = rbd.Model(tree).theta()
    t1 = rbd.rnea(tree, q, qd, qdd, theta=th)
    t2 = rbd.rnea(tree, q, qd, qdd, theta=2.5 * th)
    assert _rel(t2, 2.5 * t1) < 1e-14
    assert _rel(t1, rbd.rnea(tree, q, qd, qdd)) < 1e-14


@pytest.mark.parametrize("tree", [w.chain(7), w.spined_quadruped(), w.legged(4)], ids=lambda t: t.name)
def test_power_balance(tree):
    # qd^T tau = d/dt (1/2 qd^T M qd + PE) along q(t) = q + t qd + t^2/2 qdd
    s = w.random_state(tree, 16, seed=4)
    q, qd, qdd = s["q"], s["qd"], s["qdd"]
    tau = rbd.rnea(tree, q, qd, qdd)

    def energy(h):
        qh = q + h * qd + 0.5 * h * h * qdd
        vh = qd + h * qdd
        M = rbd.crba(tree, qh)
        return 0.5 * np.einsum("bi,bij,bj->b", vh, M, vh) + lagrange.potential(tree, qh)

    h = 1e-5
    dE = (energy(h) - energy(-h)) / (2 * h)
    power = np.einsum("bi,bi->b", qd, tau)
    assert np.abs(dE - power).max() < 1e-6 * max(1, np.abs(power).max())


@pytest.mark.parametrize("tree", [w.humanoid(), w.spined_quadruped(), w.legged(6)], ids=lambda t: t.name)
def test_kinetic_energy_from_body_twists(tree):
    """1/2 qd^T M qd equals the sum over bodies of 1/2 m |v_com|^2 +
    1/2 w^T (R Ic R^T) w, each body's world twist [v_O; w] = J_i qd taken
    from the Jacobian and its pose from FK. This pins CRBA on full-size trees,
    the free base included (where qd is not dq/dt)."""
    s = w.random_state(tree, 16, seed=5)
    q, qd = s["q"], s["qd"]
    T = rbd.fk(tree, q)
    ke = np.zeros(len(q))
    for i in range(tree.n_bodies):
        tw = np.einsum("bij,bj->bi", rbd.jacobian(tree, q, i), qd)
        vO, om = tw[:, 0:3], tw[:, 3:6]
        R, p = T[:, i, :3, :3], T[:, i, :3, 3]
        pc = p + R @ np.asarray(tree.com[i], dtype=np.float64)
        vc = vO + np.cross(om, pc)
        Iw = R @ sp.sym6_to_3x3(np.asarray(tree.I_com[i], dtype=np.float64)) @ np.swapaxes(R, 1, 2)
        ke += 0.5 * tree.mass[i] * np.einsum("bi,bi->b", vc, vc) + 0.5 * np.einsum("bi,bij,bj->b", om, Iw, om)
    M = rbd.crba(tree, q)
    ref = 0.5 * np.einsum("bi,bij,bj->b", qd, M, qd)
    np.testing.assert_allclose(ke, ref, rtol=1e-12)


def _free_body(seed):
    t = w.random_tree([-1], [w.FREE], seed)
    return t


def _newton_euler_free_body(t, q, qd, qdd):
    """Classical Newton-Euler about the centre of mass, for one free body with
    body-frame twist [v; omega] of its origin and its derivative qdd."""
    m, c = t.mass[0], t.com[0]
    Ic = sp.sym6_to_3x3(t.I_com[0])
    R = sp.quat_to_R(q[:, 3:7])
    g_body = np.einsum("bji,j->bi", R, t.gravity)           # R^T g
    v, om = qd[:, 0:3], qd[:, 3:6]
    a, al = qdd[:, 0:3], qdd[:, 3:6]
    # classical acceleration of the origin, then of the COM (body coordinates)
    acc_o = a + np.cross(om, v)
    acc_c = acc_o + np.cross(al, c) + np.cross(om, np.cross(om, c))
    F = m * (acc_c - g_body)
    Nc = al @ Ic.T + np.cross(om, om @ Ic.T)
    n_o = Nc + np.cross(c, F)
    return np.concatenate([F, n_o], -1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_free_body_matches_classical_newton_euler(seed):
    t = _free_body(seed)
    s = w.random_state(t, 50, seed=seed)
    tau = rbd.rnea(t, s["q"], s["qd"], s["qdd"])
    expect = _newton_euler_free_body(t, s["q"], s["qd"], s["qdd"])
    assert np.abs(tau - expect).max() < 1e-12
    qdd = rbd.aba(t, s["q"], s["qd"], expect)
    assert np.abs(qdd - s["qdd"]).max() < 1e-11
    # M of a single free body is its spatial inertia, reordered to [v; omega]
    M = rbd.crba(t, s["q"])
    I = sp.mcI(t.mass[0], t.com[0], sp.sym6_to_3x3(t.I_com[0]))
    P = np.zeros((6, 6))
    P[0:3, 3:6] = np.eye(3)
    P[3:6, 0:3] = np.eye(3)
    assert np.abs(M - P.T @ I @ P).max() < 1e-15


def test_quaternion_scale_invariance():
    t = w.humanoid(seed=1)
    s = w.random_state(t, 20, seed=2)
    q2 = s["q"].copy()
    q2[:, 3:7] *= 3.7
    assert _rel(rbd.rnea(t, q2, s["qd"], s["qdd"]), rbd.rnea(t, s["q"], s["qd"], s["qdd"])) < 1e-14
