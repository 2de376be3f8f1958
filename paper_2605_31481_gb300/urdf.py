"""URDF robot descriptions into the body table of a kinematic tree.

The paper parses a robot's URDF into a parent-indexed table of joints and
links before building its precomputed constants (Sec. 3.2). This module does
the same on the host and returns a `workloads.Tree`, the table that
`api.Model` uploads. It uses only the standard XML parser and numpy.

Mapping of URDF elements to the table:
  * one body per joint, in depth-first order from the root link (so every
    parent index is smaller than its child's); the body is the joint's child
    link, and its frame is that link's frame;
  * `<joint><origin xyz rpy>` -> T_joint (parent link frame to joint frame),
    T_link = identity (URDF puts the child link frame on the joint frame);
  * `<axis xyz>` (default 1 0 0) -> axis, normalised;
  * revolute and continuous -> REVOLUTE, prismatic -> PRISMATIC, fixed ->
    FIXED (kept as a body with no degree of freedom, so its frame still gets
    a pose and a Jacobian); floating is accepted only for the root, through
    floating_base=True; planar joints are rejected;
  * `<inertial>`: mass, the COM at `<origin xyz>`, and the inertia tensor of
    `<inertia>` rotated by `<origin rpy>` into the link frame (I_com about
    the COM, components xx, xy, yy, xz, yz, zz). A link without `<inertial>`
    is massless;
  * joint limits, dynamics, mimic tags, visuals and collisions are ignored.
The root link is welded to the world (its inertia plays no part) unless
floating_base=True, which gives it a free joint as body 0.

Rotations follow the URDF convention: rpy = (roll, pitch, yaw) about the
fixed x, y, z axes, R = Rz(yaw) Ry(pitch) Rx(roll).
"""
from __future__ import annotations

import os
import xml.etree.ElementTree as ET

import numpy as np

from .workloads import FIXED, FREE, IDENT12, PRISMATIC, REVOLUTE, Tree

_JOINT_TYPES = {"revolute": REVOLUTE, "continuous": REVOLUTE, "prismatic": PRISMATIC, "fixed": FIXED}


class URDFError(ValueError):
    """The description cannot be turned into a kinematic tree."""


def rpy_matrix(rpy) -> np.ndarray:
    """Rotation matrix of URDF roll-pitch-yaw angles (fixed axes x, y, z)."""
    r, p, y = (float(a) for a in rpy)
    cr, sr, cp, sp, cy, sy = np.cos(r), np.sin(r), np.cos(p), np.sin(p), np.cos(y), np.sin(y)
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _vec(el, attr, default):
    if el is None or el.get(attr) is None:
        return np.array(default, dtype=np.float64)
    v = np.array([float(x) for x in el.get(attr).split()], dtype=np.float64)
    if v.shape != (3,):
        raise URDFError(f"attribute {attr}={el.get(attr)!r} must hold 3 numbers")
    return v


def _origin(el):
    o = el.find("origin") if el is not None else None
    return _vec(o, "xyz", (0, 0, 0)), rpy_matrix(_vec(o, "rpy", (0, 0, 0)))


def _inertial(link):
    """(mass, com (3), I_com (6)) of a <link>, in the link frame."""
    it = link.find("inertial")
    if it is None:
        return 0.0, np.zeros(3), np.zeros(6)
    m_el = it.find("mass")
    mass = float(m_el.get("value", 0.0)) if m_el is not None else 0.0
    com, R = _origin(it)
    i_el = it.find("inertia")
    g = (lambda k: float(i_el.get(k, 0.0))) if i_el is not None else (lambda k: 0.0)
    I = np.array([[g("ixx"), g("ixy"), g("ixz")], [g("ixy"), g("iyy"), g("iyz")], [g("ixz"), g("iyz"), g("izz")]])
    I = R @ I @ R.T
    return mass, com, np.array([I[0, 0], I[0, 1], I[1, 1], I[0, 2], I[1, 2], I[2, 2]])


def load_urdf(source, floating_base=False, gravity=(0.0, 0.0, -9.81), ee=None) -> Tree:
    """Body table of a URDF given as a file path or as XML text.

    ee: names of links whose bodies become the tree's default Jacobian
    targets (default: every leaf body)."""
    text = source
    if not str(source).lstrip().startswith("<"):
        with open(os.fspath(source)) as fh:
            text = fh.read()
    try:
        robot = ET.fromstring(text)
    except ET.ParseError as exc:
        raise URDFError(f"not valid XML: {exc}") from None
    if robot.tag != "robot":
        raise URDFError("the root element must be <robot>")
    links = {l.get("name"): l for l in robot.findall("link")}
    joints = robot.findall("joint")
    children_of: dict[str, list] = {name: [] for name in links}
    child_links = set()
    for j in joints:
        p, c = j.find("parent"), j.find("child")
        if p is None or c is None:
            raise URDFError(f"joint {j.get('name')!r} needs <parent> and <child>")
        pl, cl = p.get("link"), c.get("link")
        if pl not in links or cl not in links:
            raise URDFError(f"joint {j.get('name')!r} names an unknown link")
        if cl in child_links:
            raise URDFError(f"link {cl!r} is the child of two joints (not a tree)")
        child_links.add(cl)
        children_of[pl].append(j)
    roots = [name for name in links if name not in child_links]
    if len(roots) != 1:
        raise URDFError(f"expected exactly one root link, found {roots}")
    root = roots[0]

    rows = []          # (parent body index, type, axis, T_joint (12), link name)
    index = {}         # link name -> body index
    if floating_base:
        index[root] = 0
        rows.append((-1, FREE, np.array([1.0, 0.0, 0.0]), IDENT12.copy(), root))
    stack = [(root, j) for j in reversed(children_of[root])]
    while stack:
        parent_link, j = stack.pop()
        kind = j.get("type")
        if kind not in _JOINT_TYPES:
            raise URDFError(f"joint {j.get('name')!r}: type {kind!r} is not supported")
        jt = _JOINT_TYPES[kind]
        xyz, R = _origin(j)
        axis = _vec(j.find("axis"), "xyz", (1, 0, 0))
        if jt != FIXED:
            nrm = np.linalg.norm(axis)
            if not nrm > 0:
                raise URDFError(f"joint {j.get('name')!r} has a zero axis")
            axis = axis / nrm
        else:
            axis = np.array([1.0, 0.0, 0.0])
        child = j.find("child").get("link")
        index[child] = len(rows)
        rows.append((index.get(parent_link, -1), jt, axis, np.concatenate([R.reshape(9), xyz]), child))
        stack.extend((child, cj) for cj in reversed(children_of[child]))
    if not rows:
        raise URDFError("the robot has no joints")

    n = len(rows)
    mass, com, I_com = np.zeros(n), np.zeros((n, 3)), np.zeros((n, 6))
    for i, (_, _, _, _, name) in enumerate(rows):
        mass[i], com[i], I_com[i] = _inertial(links[name])
    parents = np.array([r[0] for r in rows], dtype=np.int32)
    if ee is None:
        has_child = set(int(p) for p in parents if p >= 0)
        ee_idx = tuple(i for i in range(n) if i not in has_child)
    else:
        missing = [e for e in ee if e not in index]
        if missing:
            raise URDFError(f"unknown end-effector links {missing}")
        ee_idx = tuple(index[e] for e in ee)
    tree = Tree(name=robot.get("name", "urdf"), parent=parents,
                jtype=np.array([r[1] for r in rows], dtype=np.int32),
                axis=np.array([r[2] for r in rows]), T_joint=np.array([r[3] for r in rows]),
                T_link=np.tile(IDENT12, (n, 1)), mass=mass, com=com, I_com=I_com,
                gravity=np.asarray(gravity, dtype=np.float64), ee=ee_idx)
    tree.link_names = tuple(r[4] for r in rows)
    return tree
