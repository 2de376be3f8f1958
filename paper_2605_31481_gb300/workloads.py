"""Seeded synthetic kinematic trees and inputs.

This module only draws random numbers and lays them out; it holds none of the
dynamics arithmetic. Both the FP64 oracle and the CUDA path consume what it
produces, so it imports neither.

A tree is a body table in topological order (parent index < own index, -1 =
world). Each body is attached to its parent by one joint:

    pose of body i in its parent = T_joint[i] * J(q_i) * T_link[i]

where J is a rotation about `axis` (revolute), a translation along `axis`
(prismatic), the identity (fixed) or a full rigid pose taken from q (free).
Inertial data are given about the body's centre of mass, in the body frame:
mass, com (3) and I_com as (xx, xy, yy, xz, yz, zz).

Model distributions (the paper's robots are not available as assets, so these
trees stand in for the 7-23 DOF robots of the paper's Sec. 4.1/4.2):
  * unit joint axes uniform on the sphere (normalised 3-D Gaussian);
  * parent-to-joint offsets uniform in [-0.3, 0.3] m, identity rotation;
  * T_link = identity;
  * link masses uniform in [0.5, 5] kg, COM uniform in [-0.1, 0.1] m;
  * I_com = R diag(l) R^T with l uniform in [0.01, 0.1], all three redrawn
    until each pair-sum is >= the third, and R a Haar-uniform rotation taken
    from a normalised 4-D Gaussian quaternion.
Inputs: q uniform in [-pi, pi], qd and qdd from N(0, 1), tau from N(0, 5^2),
gravity (0, 0, -9.81). A free base takes a random unit quaternion and a
translation from N(0, 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FIXED, REVOLUTE, PRISMATIC, FREE = 0, 1, 2, 3
NQ_OF = {FIXED: 0, REVOLUTE: 1, PRISMATIC: 1, FREE: 7}
NV_OF = {FIXED: 0, REVOLUTE: 1, PRISMATIC: 1, FREE: 6}

IDENT12 = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], dtype=np.float64)


@dataclass
class Tree:
    """Body table of one kinematic tree (all float64, numpy)."""

    name: str
    parent: np.ndarray          # (n_b,) int32
    jtype: np.ndarray           # (n_b,) int32
    axis: np.ndarray            # (n_b, 3)
    T_joint: np.ndarray         # (n_b, 12) R row-major (9), t (3)
    T_link: np.ndarray          # (n_b, 12)
    mass: np.ndarray            # (n_b,)
    com: np.ndarray             # (n_b, 3)
    I_com: np.ndarray           # (n_b, 6) xx, xy, yy, xz, yz, zz
    gravity: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, -9.81]))
    ee: tuple = ()              # default end-effector bodies for Jacobians

    @property
    def n_bodies(self) -> int:
        return int(self.parent.shape[0])

    @property
    def nq(self) -> int:
        return int(sum(NQ_OF[int(t)] for t in self.jtype))

    @property
    def nv(self) -> int:
        return int(sum(NV_OF[int(t)] for t in self.jtype))

    def q_index(self) -> np.ndarray:
        out, k = [], 0
        for t in self.jtype:
            out.append(k)
            k += NQ_OF[int(t)]
        return np.array(out, dtype=np.int64)

    def v_index(self) -> np.ndarray:
        out, k = [], 0
        for t in self.jtype:
            out.append(k)
            k += NV_OF[int(t)]
        return np.array(out, dtype=np.int64)

    def depth(self) -> int:
        d = np.zeros(self.n_bodies, dtype=np.int64)
        for i, p in enumerate(self.parent):
            d[i] = 1 if p < 0 else d[p] + 1
        return int(d.max()) if self.n_bodies else 0


# ----------------------------------------------------------------------------
# random draws
# ----------------------------------------------------------------------------

def _unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _haar_rotation(rng):
    qv = rng.standard_normal(4)
    w, x, y, z = qv / np.linalg.norm(qv)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def _principal_moments(rng):
    while True:
        l = rng.uniform(0.01, 0.1, size=3)
        if l[0] + l[1] >= l[2] and l[0] + l[2] >= l[1] and l[1] + l[2] >= l[0]:
            return l


def _inertial(rng, n):
    mass = rng.uniform(0.5, 5.0, size=n)
    com = rng.uniform(-0.1, 0.1, size=(n, 3))
    I6 = np.zeros((n, 6))
    for i in range(n):
        l = _principal_moments(rng)
        R = _haar_rotation(rng)
        Ic = R @ np.diag(l) @ R.T
        I6[i] = [Ic[0, 0], Ic[0, 1], Ic[1, 1], Ic[0, 2], Ic[1, 2], Ic[2, 2]]
    return mass, com, I6


def random_tree(parent, jtype, seed, name="tree", ee=()):
    """Fill a topology with random joint axes, offsets and inertias."""
    parent = np.asarray(parent, dtype=np.int32)
    jtype = np.asarray(jtype, dtype=np.int32)
    n = parent.shape[0]
    rng = np.random.default_rng(seed)
    axis = _unit(rng, n)
    T_joint = np.tile(IDENT12, (n, 1))
    T_joint[:, 9:12] = rng.uniform(-0.3, 0.3, size=(n, 3))
    for i in range(n):
        if jtype[i] == FREE:
            T_joint[i] = IDENT12
    T_link = np.tile(IDENT12, (n, 1))
    mass, com, I6 = _inertial(rng, n)
    return Tree(name=name, parent=parent, jtype=jtype, axis=axis, T_joint=T_joint,
                T_link=T_link, mass=mass, com=com, I_com=I6, ee=tuple(ee))


# ----------------------------------------------------------------------------
# the workload topologies
# ----------------------------------------------------------------------------

def chain(n_dof=7, seed=0):
    """Serial chain of revolute joints on a fixed base (7-DOF arm shape)."""
    parent = [i - 1 for i in range(n_dof)]
    return random_tree(parent, [REVOLUTE] * n_dof, seed, name=f"chain{n_dof}", ee=(n_dof - 1,))


def spined_quadruped(seed=0):
    """11 revolute DOF, depth 5: spine s1-s2-s3 on a fixed base, a rear leg
    pair (hip, knee) hanging off s1 and a front pair off s3.
    Bodies: 0 s1, 1 s2, 2 s3, 3/4 rear-left hip/knee, 5/6 rear-right,
    7/8 front-left, 9/10 front-right. Feet = the four knees."""
    parent = [-1, 0, 1, 0, 3, 0, 5, 2, 7, 2, 9]
    return random_tree(parent, [REVOLUTE] * 11, seed, name="spined_quadruped11",
                       ee=(4, 6, 8, 10))


def legged(n_legs, seed=0, joints_per_leg=3):
    """n_legs legs of joints_per_leg revolute joints each, off a fixed base."""
    parent, k = [], 0
    for _ in range(n_legs):
        for j in range(joints_per_leg):
            parent.append(-1 if j == 0 else k - 1)
            k += 1
    ee = tuple(joints_per_leg * (l + 1) - 1 for l in range(n_legs))
    return random_tree(parent, [REVOLUTE] * k, seed, name=f"legged{k}", ee=ee)


def humanoid(seed=0, floating=True):
    """Humanoid shape: (free base) + 1-joint waist + 2 legs x 6 + 2 arms x 5
    (23 revolute DOF). Legs hang off the base, arms off the waist.
    With floating=True body 0 is a free joint (nq = 30, nv = 29, depth 7);
    otherwise the 23 revolute joints sit on a fixed base."""
    parent, jtype = [], []
    if floating:
        parent.append(-1)
        jtype.append(FREE)
        base = 0
    else:
        base = -1

    def add(p):
        parent.append(p)
        jtype.append(REVOLUTE)
        return len(parent) - 1

    waist = add(base)
    feet, hands = [], []
    for _ in range(2):
        p = base
        for _ in range(6):
            p = add(p)
        feet.append(p)
    for _ in range(2):
        p = waist
        for _ in range(5):
            p = add(p)
        hands.append(p)
    name = "humanoid_float29" if floating else "humanoid_fixed23"
    return random_tree(parent, jtype, seed, name=name, ee=tuple(feet + hands))


def mixed_trees(seeds=(0, 1, 2, 3, 4)):
    """The five trees of the mixed batch: 7, 11, 12, 18 and 23 revolute DOF."""
    return [chain(7, seeds[0]), spined_quadruped(seeds[1]), legged(4, seeds[2]),
            legged(6, seeds[3]), humanoid(seeds[4], floating=False)]


# ----------------------------------------------------------------------------
# inputs
# ----------------------------------------------------------------------------

def random_state(tree: Tree, B: int, seed=1, tau_std=5.0):
    """Returns a dict of float64 arrays with env as the leading axis:
    q (B, nq), qd (B, nv), qdd (B, nv), tau (B, nv)."""
    rng = np.random.default_rng(seed)
    nq, nv = tree.nq, tree.nv
    q = rng.uniform(-np.pi, np.pi, size=(B, nq))
    qd = rng.standard_normal((B, nv))
    qdd = rng.standard_normal((B, nv))
    tau = tau_std * rng.standard_normal((B, nv))
    qi = tree.q_index()
    for i, t in enumerate(tree.jtype):
        if t == FREE:
            k = qi[i]
            q[:, k:k + 3] = rng.standard_normal((B, 3))
            quat = rng.standard_normal((B, 4))
            q[:, k + 3:k + 7] = quat / np.linalg.norm(quat, axis=1, keepdims=True)
    return {"q": q, "qd": qd, "qdd": qdd, "tau": tau}
