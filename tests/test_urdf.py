"""URDF loader: the body table it builds, pinned through the FP64 oracle
against closed forms and scipy's Euler-angle convention."""
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import rbd
from paper_2605_31481_gb300 import urdf
from paper_2605_31481_gb300.workloads import FIXED, FREE, IDENT12, PRISMATIC, REVOLUTE

DATA = os.path.join(os.path.dirname(__file__), "data")


def _two_link(l1=0.7, c1=0.3, c2=0.25, m1=2.0, m2=1.3, I1=0.05, I2=0.03, rot_inertia=False):
    """Planar arm in the x-y plane (joints about z), URDF text."""
    # with rot_inertia the second link's tensor is given in a frame turned 90
    # degrees about x: its iyy then becomes the link-frame izz
    i2 = (f'<origin xyz="{c2} 0 0" rpy="1.5707963267948966 0 0"/><mass value="{m2}"/>'
          f'<inertia ixx="0.01" ixy="0" ixz="0" iyy="{I2}" iyz="0" izz="0.02"/>' if rot_inertia else
          f'<origin xyz="{c2} 0 0"/><mass value="{m2}"/>'
          f'<inertia ixx="0.01" ixy="0" ixz="0" iyy="0.02" iyz="0" izz="{I2}"/>')
    return f"""<robot name="two_link">
      <link name="base"/>
      <link name="a"><inertial><origin xyz="{c1} 0 0"/><mass value="{m1}"/>
        <inertia ixx="0.01" ixy="0" ixz="0" iyy="0.02" iyz="0" izz="{I1}"/></inertial></link>
      <link name="b"><inertial>{i2}</inertial></link>
      <joint name="j1" type="continuous"><parent link="base"/><child link="a"/><axis xyz="0 0 1"/></joint>
      <joint name="j2" type="revolute"><parent link="a"/><child link="b"/>
        <origin xyz="{l1} 0 0"/><axis xyz="0 0 1"/></joint>
    </robot>"""


@pytest.mark.parametrize("rot_inertia", [False, True])
def test_two_link_arm_mass_matrix_and_gravity_closed_form(rot_inertia):
    """Textbook planar two-link arm: M(q) and the gravity torques."""
    l1, c1, c2, m1, m2, I1, I2, g = 0.7, 0.3, 0.25, 2.0, 1.3, 0.05, 0.03, 9.81
    tree = urdf.load_urdf(_two_link(l1, c1, c2, m1, m2, I1, I2, rot_inertia), gravity=(0, -g, 0))
    assert tree.n_bodies == 2 and list(tree.parent) == [-1, 0] and list(tree.jtype) == [REVOLUTE, REVOLUTE]
    rng = np.random.default_rng(0)
    q = rng.uniform(-np.pi, np.pi, (16, 2))
    M = rbd.crba(tree, q)
    c = np.cos(q[:, 1])
    M11 = I1 + I2 + m1 * c1 ** 2 + m2 * (l1 ** 2 + c2 ** 2 + 2 * l1 * c2 * c)
    M12 = I2 + m2 * (c2 ** 2 + l1 * c2 * c)
    M22 = np.full_like(c, I2 + m2 * c2 ** 2)
    np.testing.assert_allclose(M[:, 0, 0], M11, rtol=1e-12)
    np.testing.assert_allclose(M[:, 0, 1], M12, rtol=1e-12)
    np.testing.assert_allclose(M[:, 1, 1], M22, rtol=1e-12)
    tau = rbd.rnea(tree, q, np.zeros_like(q), np.zeros_like(q))
    g1 = (m1 * c1 + m2 * l1) * g * np.cos(q[:, 0]) + m2 * c2 * g * np.cos(q[:, 0] + q[:, 1])
    g2 = m2 * c2 * g * np.cos(q[:, 0] + q[:, 1])
    np.testing.assert_allclose(tau[:, 0], g1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(tau[:, 1], g2, rtol=1e-12, atol=1e-12)


def test_joint_origin_rpy_follows_the_urdf_convention():
    """At q = 0 a body's pose is its joint origin: rpy about the fixed x, y,
    z axes, which is scipy's extrinsic "xyz"."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        rpy = rng.uniform(-np.pi, np.pi, 3)
        xyz = rng.standard_normal(3)
        text = f"""<robot name="r"><link name="w"/><link name="b"><inertial><mass value="1"/>
          <inertia ixx="1" ixy="0" ixz="0" iyy="1" iyz="0" izz="1"/></inertial></link>
          <joint name="j" type="revolute"><parent link="w"/><child link="b"/>
          <origin xyz="{xyz[0]} {xyz[1]} {xyz[2]}" rpy="{rpy[0]} {rpy[1]} {rpy[2]}"/><axis xyz="0 1 0"/></joint></robot>"""
        tree = urdf.load_urdf(text)
        T = rbd.fk(tree, np.zeros((1, 1)))[0, 0]
        np.testing.assert_allclose(T[:3, :3], Rotation.from_euler("xyz", rpy).as_matrix(), atol=1e-14)
        np.testing.assert_allclose(T[:3, 3], xyz, atol=1e-14)
        np.testing.assert_allclose(urdf.rpy_matrix(rpy), Rotation.from_euler("xyz", rpy).as_matrix(), atol=1e-14)


def test_inertial_frame_rotation():
    """One rigid body whose COM lies on its joint axis: the joint-space
    inertia is a^T I_link a, with I_link the URDF tensor rotated by the
    inertial origin's rpy."""
    rng = np.random.default_rng(2)
    rpy = rng.uniform(-1, 1, 3)
    L = rng.uniform(0.01, 0.1, 3)
    R0 = Rotation.from_euler("xyz", rng.uniform(-1, 1, 3)).as_matrix()
    I = R0 @ np.diag(L) @ R0.T
    text = f"""<robot name="r"><link name="w"/><link name="b"><inertial>
      <origin xyz="0 0 0" rpy="{rpy[0]} {rpy[1]} {rpy[2]}"/><mass value="2"/>
      <inertia ixx="{I[0,0]}" ixy="{I[0,1]}" ixz="{I[0,2]}" iyy="{I[1,1]}" iyz="{I[1,2]}" izz="{I[2,2]}"/></inertial></link>
      <joint name="j" type="revolute"><parent link="w"/><child link="b"/><axis xyz="1 2 2"/></joint></robot>"""
    tree = urdf.load_urdf(text)
    a = np.array([1.0, 2.0, 2.0]) / 3.0
    Rr = Rotation.from_euler("xyz", rpy).as_matrix()
    M = rbd.crba(tree, rng.uniform(-3, 3, (4, 1)))
    np.testing.assert_allclose(M[:, 0, 0], a @ (Rr @ I @ Rr.T) @ a, rtol=1e-12)


def test_arm_file_table():
    tree = urdf.load_urdf(os.path.join(DATA, "arm6_tool.urdf"))
    assert tree.name == "arm6_tool"
    assert tree.link_names == ("l1", "l2", "l3", "l4", "l5", "l6", "tool")
    assert list(tree.parent) == [-1, 0, 1, 2, 3, 4, 5]
    assert list(tree.jtype) == [REVOLUTE, REVOLUTE, REVOLUTE, PRISMATIC, REVOLUTE, REVOLUTE, FIXED]
    assert tree.nq == tree.nv == 6 and tree.ee == (6,)
    np.testing.assert_allclose(tree.axis[4], np.array([0, 1, 1]) / np.sqrt(2))
    np.testing.assert_allclose(tree.T_link, np.tile(IDENT12, (7, 1)))
    # total mass and the symmetric, positive definite mass matrix
    assert abs(tree.mass.sum() - 9.0) < 1e-12
    q = np.random.default_rng(3).uniform(-1, 1, (8, 6))
    M = rbd.crba(tree, q)
    np.testing.assert_allclose(M, np.swapaxes(M, 1, 2), atol=1e-14)
    assert np.all(np.linalg.eigvalsh(M) > 0)


def test_floating_base_and_named_end_effectors():
    text = open(os.path.join(DATA, "arm6_tool.urdf")).read().replace(
        '<link name="base"/>', '<link name="base"><inertial><mass value="5"/>'
        '<inertia ixx="0.1" ixy="0" ixz="0" iyy="0.1" iyz="0" izz="0.1"/></inertial></link>')
    tree = urdf.load_urdf(text, floating_base=True, ee=["tool", "l3"])
    assert tree.jtype[0] == FREE and tree.parent[0] == -1 and tree.mass[0] == 5.0
    assert tree.nq == 13 and tree.nv == 12 and tree.ee == (7, 3)
    s_q = np.zeros((2, 13))
    s_q[:, 6] = 1.0                      # identity quaternion
    M = rbd.crba(tree, s_q)
    np.testing.assert_allclose(M[:, 0, 0], tree.mass.sum(), rtol=1e-12)   # total mass on the base translation


@pytest.mark.parametrize("bad,msg", [
    ('<robot name="r"><link name="a"/><link name="b"/></robot>', "root"),
    ('<robot name="r"><link name="a"/><link name="b"/><joint name="j" type="planar"><parent link="a"/>'
     '<child link="b"/></joint></robot>', "not supported"),
    ('<robot name="r"><link name="a"/><link name="b"/><joint name="j" type="revolute"><parent link="a"/>'
     '<child link="c"/></joint></robot>', "unknown link"),
    ('<robot name="r"><link name="a"/><link name="b"/><joint name="j" type="revolute"><parent link="a"/>'
     '<child link="b"/><axis xyz="0 0 0"/></joint></robot>', "zero axis"),
    ('<notarobot/>', "<robot>"),
])
def test_rejects_what_is_not_a_tree(bad, msg):
    with pytest.raises(urdf.URDFError, match=msg):
        urdf.load_urdf(bad)
