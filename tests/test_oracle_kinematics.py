"""Pins of the oracle's kinematics (FK and Jacobian) to facts that do not
come from the oracle itself: a library rotation routine, closed forms for a
planar arm, orthonormality, and derivatives of the pose."""
import json
import os

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

from oracle import rbd, derivs
from oracle import spatial as sp
from paper_2605_31481_gb300 import workloads as w

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_fp64_discrepancy.json")))


def _tree(parent, jtype, seed, rot_offsets=False, link_offsets=False):
    t = w.random_tree(parent, jtype, seed)
    rng = np.random.default_rng(seed + 100)
    if rot_offsets:
        for i in range(t.n_bodies):
            if t.jtype[i] != w.FREE:
                t.T_joint[i, :9] = Rotation.random(random_state=rng.integers(1 << 30)).as_matrix().ravel()
    if link_offsets:
        for i in range(t.n_bodies):
            t.T_link[i, :9] = Rotation.random(random_state=rng.integers(1 << 30)).as_matrix().ravel()
            t.T_link[i, 9:] = rng.uniform(-0.2, 0.2, 3)
    return t


def test_axis_angle_matches_library_rotation():
    rng = np.random.default_rng(0)
    ax = rng.standard_normal((50, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    ang = rng.uniform(-np.pi, np.pi, 50)
    R = sp.axis_angle_to_R(ax, ang)
    Rl = Rotation.from_rotvec(ax * ang[:, None]).as_matrix()
    assert np.abs(R - Rl).max() < 1e-14


def test_quaternion_matches_library_rotation():
    rng = np.random.default_rng(1)
    qv = rng.standard_normal((50, 4)) * 3.0           # deliberately not unit
    R = sp.quat_to_R(qv)
    Rl = Rotation.from_quat(qv).as_matrix()             # scalar-last (x, y, z, w)
    assert np.abs(R - Rl).max() < 1e-14


def test_planar_arm_closed_form():
    # three z-axis joints, each joint frame offset by l along the parent's x
    l = np.array([0.0, 0.7, 0.4])
    t = w.random_tree([-1, 0, 1], [w.REVOLUTE] * 3, seed=0)
    t.axis[:] = [0, 0, 1]
    t.T_joint[:, 9:] = 0
    t.T_joint[:, 9] = l
    rng = np.random.default_rng(3)
    q = rng.uniform(-np.pi, np.pi, (20, 3))
    T = rbd.fk(t, q)
    cum = np.cumsum(q, axis=1)
    p1 = l[1] * np.stack([np.cos(cum[:, 0]), np.sin(cum[:, 0])], -1)
    p2 = p1 + l[2] * np.stack([np.cos(cum[:, 1]), np.sin(cum[:, 1])], -1)
    assert np.abs(T[:, 1, :2, 3] - p1).max() < 1e-14
    assert np.abs(T[:, 2, :2, 3] - p2).max() < 1e-14
    for i in range(3):
        Rz = Rotation.from_euler("z", cum[:, i:i + 1]).as_matrix()
        assert np.abs(T[:, i, :3, :3] - Rz).max() < 1e-14


def test_prismatic_and_fixed_closed_form():
    t = w.random_tree([-1, 0], [w.PRISMATIC, w.FIXED], seed=4)
    q = np.array([[0.3], [-1.2]])
    T = rbd.fk(t, q)
    Tj0 = sp.T12_to_homog(t.T_joint[0])
    for b in range(2):
        expect0 = Tj0.copy()
        expect0[:3, 3] += Tj0[:3, :3] @ (t.axis[0] * q[b, 0])
        assert np.abs(T[b, 0] - expect0).max() < 1e-15
        expect1 = expect0 @ sp.T12_to_homog(t.T_joint[1])
        assert np.abs(T[b, 1] - expect1).max() < 1e-15


@pytest.mark.parametrize("tree", [w.chain(7), w.spined_quadruped(), w.humanoid()], ids=lambda t: t.name)
def test_fk_rotations_orthonormal(tree):
    s = w.random_state(tree, 200, seed=5)
    R = rbd.fk(tree, s["q"])[..., :3, :3]
    err = np.abs(R @ np.swapaxes(R, -1, -2) - np.eye(3)).max()
    assert err < 10 * GOLD["FK"]
    assert np.abs(np.linalg.det(R) - 1).max() < 10 * GOLD["FK"]


def _twist_from_dT(dT, T):
    """World twist [v_O; omega] of a moving frame from dT/dt and T."""
    R, p = T[..., :3, :3], T[..., :3, 3]
    dR, dp = dT[..., :3, :3], dT[..., :3, 3]
    W = dR @ np.swapaxes(R, -1, -2)
    om = np.stack([W[..., 2, 1], W[..., 0, 2], W[..., 1, 0]], -1)
    v0 = dp - np.cross(om, p)
    return np.concatenate([v0, om], -1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_jacobian_equals_pose_derivative(seed):
    # fixed-base tree with every joint type and non-trivial joint/link frames
    t = _tree([-1, 0, 1, 1, 3, 4], [w.REVOLUTE, w.PRISMATIC, w.REVOLUTE, w.FIXED, w.REVOLUTE, w.PRISMATIC],
              seed, rot_offsets=True, link_offsets=True)
    s = w.random_state(t, 8, seed=seed)
    q = s["q"]
    for body in range(t.n_bodies):
        J = rbd.jacobian(t, q, body)
        T = rbd.fk(t, q)[:, body]
        for k in range(t.nq):
            e = np.zeros_like(q)
            e[:, k] = 1
            dT = derivs.jvp_cs(lambda q_: rbd.fk(t, q_)[:, body], (q,), 0, e)
            tw = _twist_from_dT(dT, T)
            assert np.abs(J[:, :, k] - tw).max() < 1e-13
            # and by central differences, independent of the complex-step routine
            h = 1e-6
            dTf = (rbd.fk(t, q + h * e)[:, body] - rbd.fk(t, q - h * e)[:, body]) / (2 * h)
            assert np.abs(J[:, :, k] - _twist_from_dT(dTf, T)).max() < 1e-8


def test_jacobian_revolute_is_axis_cross_form():
    # paper Eq. 6: column = [o x z; z] with z the world axis, o a point on it
    t = _tree([-1, 0, 1], [w.REVOLUTE] * 3, 7, rot_offsets=True)
    q = w.random_state(t, 10, seed=3)["q"]
    J = rbd.jacobian(t, q, 2)
    T = rbd.fk(t, q)
    for k in range(3):
        Tp = np.eye(4) if k == 0 else T[:, k - 1]
        Tj = Tp @ sp.T12_to_homog(t.T_joint[k])
        a = t.axis[k] / np.linalg.norm(t.axis[k])
        z = Tj[..., :3, :3] @ a
        o = Tj[..., :3, 3]
        assert np.abs(J[:, 3:, k] - z).max() < 1e-15
        assert np.abs(J[:, :3, k] - np.cross(o, z)).max() < 1e-14


def _free_step(q, xi, h):
    """Advance a free-joint configuration by the body twist xi ([v; omega])
    for time h, by the exponential map (library expm)."""
    out = q.copy()
    for b in range(q.shape[0]):
        T = sp.homog(sp.quat_to_R(q[b, 3:7]), q[b, 0:3])
        Xi = np.zeros((4, 4))
        Xi[:3, :3] = sp.skew(xi[b, 3:6])
        Xi[:3, 3] = xi[b, 0:3]
        Tn = T @ expm(h * Xi)
        out[b, 0:3] = Tn[:3, 3]
        out[b, 3:7] = Rotation.from_matrix(Tn[:3, :3]).as_quat()
    return out


def test_free_joint_jacobian_by_exponential_map():
    t = w.humanoid(seed=2)
    s = w.random_state(t, 4, seed=9)
    q = s["q"]
    body = t.ee[0]
    J = rbd.jacobian(t, q, body)
    T = rbd.fk(t, q)[:, body]
    h = 1e-6
    for k in range(6):
        xi = np.zeros((4, 6))
        xi[:, k] = 1
        qp = _free_step(q, xi, h)
        qm = _free_step(q, xi, -h)
        dT = (rbd.fk(t, qp)[:, body] - rbd.fk(t, qm)[:, body]) / (2 * h)
        assert np.abs(J[:, :, k] - _twist_from_dT(dT, T)).max() < 1e-7
