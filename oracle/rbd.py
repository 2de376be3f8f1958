"""Textbook recursive rigid-body algorithms, FP64, batched over environments.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A tree is any object with the body-table fields parent, jtype, axis, T_joint,
T_link, mass, com, I_com, gravity (the seeded generators produce one). Bodies
are in topological order. Joint types: 0 fixed, 1 revolute, 2 prismatic,
3 free (6 DOF; q = [x, y, z, qx, qy, qz, qw]; velocity = twist of the moving
frame in its own coordinates, linear part first: [v; omega]).

Each body's pose in its parent is T_joint * J(q) * T_link (paper Sec. 3.2,
first equation). Plucker transforms, motion subspaces and inertias are plain
6x6 / 6xk matrices built from that definition; the paper's Rodrigues
constants (Eq. 2-5) are deliberately not used here.

Arrays: q (B, nq), qd/qdd/tau (B, nv); theta, if given, is (n_b, 10)
[m, m c, I_o(xx, xy, yy, xz, yz, zz)] about the body-frame origin and
replaces the table's inertias.
"""
import numpy as np

from . import spatial as sp

FIXED, REVOLUTE, PRISMATIC, FREE = 0, 1, 2, 3
_NQ = {FIXED: 0, REVOLUTE: 1, PRISMATIC: 1, FREE: 7}
_NV = {FIXED: 0, REVOLUTE: 1, PRISMATIC: 1, FREE: 6}


class Model:
    """Static per-body data derived from a body table."""

    def __init__(self, tree):
        self.tree = tree
        self.n = int(len(tree.parent))
        self.parent = [int(p) for p in tree.parent]
        self.jtype = [int(t) for t in tree.jtype]
        self.axis = [np.asarray(a, dtype=np.float64) / np.linalg.norm(a) if self.jtype[i] in (REVOLUTE, PRISMATIC)
                     else np.asarray(a, dtype=np.float64) for i, a in enumerate(tree.axis)]
        self.T_joint = [sp.T12_to_homog(np.asarray(t, dtype=np.float64)) for t in tree.T_joint]
        self.T_link = [sp.T12_to_homog(np.asarray(t, dtype=np.float64)) for t in tree.T_link]
        self.qi, self.vi, self.nqi, self.nvi = [], [], [], []
        kq = kv = 0
        for t in self.jtype:
            self.qi.append(kq)
            self.vi.append(kv)
            self.nqi.append(_NQ[t])
            self.nvi.append(_NV[t])
            kq += _NQ[t]
            kv += _NV[t]
        self.nq, self.nv = kq, kv
        # Motion subspace in child coordinates: S_i = X(T_link) s_J, with s_J
        # the joint's free modes in the joint's moving frame.
        self.S = []
        for i, t in enumerate(self.jtype):
            XL = sp.pose_to_X(self.T_link[i])
            if t == REVOLUTE:
                sJ = np.concatenate([self.axis[i], np.zeros(3)])[:, None]
            elif t == PRISMATIC:
                sJ = np.concatenate([np.zeros(3), self.axis[i]])[:, None]
            elif t == FREE:
                # velocity coordinates [v; omega] -> spatial [omega; v]
                sJ = np.zeros((6, 6))
                sJ[0:3, 3:6] = np.eye(3)
                sJ[3:6, 0:3] = np.eye(3)
            else:
                sJ = np.zeros((6, 0))
            self.S.append(XL @ sJ)
        self.gravity = np.asarray(tree.gravity, dtype=np.float64)

    def inertias(self, theta=None):
        """Spatial inertia of every body at its own frame origin."""
        if theta is not None:
            return [sp.inertia_from_theta(np.asarray(theta)[i]) for i in range(self.n)]
        t = self.tree
        return [sp.mcI(float(t.mass[i]), np.asarray(t.com[i], dtype=np.float64),
                       sp.sym6_to_3x3(np.asarray(t.I_com[i], dtype=np.float64)))
                for i in range(self.n)]

    def theta(self):
        """The table's inertias in the 10-parameter layout."""
        return np.stack([sp.theta_from_inertia(I) for I in self.inertias()])

    def joint_pose(self, i, q):
        """J(q) of body i's joint, as a batch of 4x4 transforms."""
        t = self.jtype[i]
        B = q.shape[0]
        seg = q[:, self.qi[i]:self.qi[i] + self.nqi[i]]
        if t == REVOLUTE:
            return sp.homog(sp.axis_angle_to_R(self.axis[i], seg[:, 0]), np.zeros((B, 3), dtype=q.dtype))
        if t == PRISMATIC:
            return sp.homog(np.broadcast_to(np.eye(3, dtype=q.dtype), (B, 3, 3)), seg[:, 0:1] * self.axis[i])
        if t == FREE:
            return sp.homog(sp.quat_to_R(seg[:, 3:7]), seg[:, 0:3])
        return sp.homog(np.broadcast_to(np.eye(3, dtype=q.dtype), (B, 3, 3)), np.zeros((B, 3), dtype=q.dtype))

    def local_pose(self, i, q):
        """Pose of body i in its parent: T_joint * J(q) * T_link."""
        return self.T_joint[i] @ self.joint_pose(i, q) @ self.T_link[i]

    def Xup(self, i, q):
        """Motion transform from the parent's frame to body i's frame."""
        return sp.pose_to_X(self.local_pose(i, q))

    def a0(self, B, dtype, gravity=None):
        # a complex gravity passes through, so complex steps can differentiate in it
        g = self.gravity if gravity is None else np.asarray(gravity)
        a = np.zeros((B, 6), dtype=np.result_type(dtype, g.dtype, np.float64))
        a[:, 3:6] = -g
        return a


def _mv(M, v):
    return np.einsum("...ij,...j->...i", M, v)


def _tv(M, v):
    return np.einsum("...ji,...j->...i", M, v)


def fk(tree, q):
    """World pose (B, n_b, 4, 4) of every body (tier 3 of paper Sec. 3.1)."""
    m = Model(tree)
    q = np.asarray(q)
    T = [None] * m.n
    for i in range(m.n):
        Tl = m.local_pose(i, q)
        p = m.parent[i]
        T[i] = Tl if p < 0 else T[p] @ Tl
    return np.stack(T, axis=1)


def jacobian(tree, q, body):
    """Geometric Jacobian (B, 6, nv) of `body`: world-frame twist measured at
    the world origin, rows [v; omega] (paper Eq. 6). Column block k is the
    adjoint of joint k's motion subspace, for joints on the support path."""
    m = Model(tree)
    q = np.asarray(q)
    T = fk(tree, q)
    B = q.shape[0]
    J = np.zeros((B, 6, m.nv), dtype=q.dtype)
    k = body
    while k >= 0:
        if m.nvi[k]:
            col = sp.pose_to_Xinv(T[:, k]) @ m.S[k]          # (B, 6, nv_k), [omega; v]
            J[:, 0:3, m.vi[k]:m.vi[k] + m.nvi[k]] = col[:, 3:6]
            J[:, 3:6, m.vi[k]:m.vi[k] + m.nvi[k]] = col[:, 0:3]
        k = m.parent[k]
    return J


def rnea(tree, q, qd, qdd, theta=None, gravity=None):
    """Inverse dynamics tau (B, nv) by recursive Newton-Euler.

    Forward sweep (paper Eq. 7 and its acceleration analogue):
        v_i = X_i v_p + S_i qd_i
        a_i = X_i a_p + S_i qdd_i + v_i x (S_i qd_i),   a_world = -g
        f_i = I_i a_i + v_i x* (I_i v_i)
    Backward sweep: tau_i = S_i^T f_i, f_p += X_i^T f_i."""
    m = Model(tree)
    q, qd, qdd = np.asarray(q), np.asarray(qd), np.asarray(qdd)
    dt = np.result_type(q, qd, qdd, np.float64 if theta is None else np.asarray(theta),
                        np.float64 if gravity is None else np.asarray(gravity))
    B = q.shape[0]
    I = m.inertias(theta)
    a0 = m.a0(B, dt, gravity)
    X, v, a, f = [None] * m.n, [None] * m.n, [None] * m.n, [None] * m.n
    for i in range(m.n):
        X[i] = m.Xup(i, q)
        S = m.S[i]
        s = slice(m.vi[i], m.vi[i] + m.nvi[i])
        vJ = _mv(S, qd[:, s])
        p = m.parent[i]
        vp = np.zeros((B, 6), dtype=dt) if p < 0 else v[p]
        ap = a0 if p < 0 else a[p]
        v[i] = _mv(X[i], vp) + vJ
        a[i] = _mv(X[i], ap) + _mv(S, qdd[:, s]) + _mv(sp.crm(v[i]), vJ)
        f[i] = _mv(I[i], a[i]) + _mv(sp.crf(v[i]), _mv(I[i], v[i]))
    tau = np.zeros((B, m.nv), dtype=dt)
    for i in reversed(range(m.n)):
        s = slice(m.vi[i], m.vi[i] + m.nvi[i])
        tau[:, s] = _tv(m.S[i], f[i])
        p = m.parent[i]
        if p >= 0:
            f[p] = f[p] + _tv(X[i], f[i])
    return tau


def crba(tree, q, theta=None):
    """Joint-space mass matrix M (B, nv, nv) by the composite-rigid-body
    algorithm: composite inertias I^c_p += X_i^T I^c_i X_i (the 6x6 update the
    paper names as the bottleneck, Sec. 3.5), then F = I^c_i S_i carried up
    the support path, M_ij = S_j^T F."""
    m = Model(tree)
    q = np.asarray(q)
    dt = np.result_type(q, np.float64 if theta is None else np.asarray(theta))
    B = q.shape[0]
    X = [m.Xup(i, q) for i in range(m.n)]
    Ic = [np.broadcast_to(Ii, (B, 6, 6)).astype(dt) for Ii in m.inertias(theta)]
    for i in reversed(range(m.n)):
        p = m.parent[i]
        if p >= 0:
            Ic[p] = Ic[p] + np.swapaxes(X[i], -1, -2) @ Ic[i] @ X[i]
    H = np.zeros((B, m.nv, m.nv), dtype=dt)
    for i in range(m.n):
        if m.nvi[i] == 0:
            continue
        si = slice(m.vi[i], m.vi[i] + m.nvi[i])
        F = Ic[i] @ m.S[i]
        H[:, si, si] = np.swapaxes(m.S[i], -1, -2) @ F
        j = i
        while m.parent[j] >= 0:
            F = np.swapaxes(X[j], -1, -2) @ F
            j = m.parent[j]
            if m.nvi[j] == 0:
                continue
            sj = slice(m.vi[j], m.vi[j] + m.nvi[j])
            Hij = np.swapaxes(F, -1, -2) @ m.S[j]
            H[:, si, sj] = Hij
            H[:, sj, si] = np.swapaxes(Hij, -1, -2)
    return H


def aba(tree, q, qd, tau, theta=None, gravity=None):
    """Forward dynamics qdd (B, nv) by the articulated-body algorithm, three
    passes (velocities and bias terms; articulated inertias leaf to root;
    accelerations root to leaf)."""
    m = Model(tree)
    q, qd, tau = np.asarray(q), np.asarray(qd), np.asarray(tau)
    dt = np.result_type(q, qd, tau, np.float64 if theta is None else np.asarray(theta),
                        np.float64 if gravity is None else np.asarray(gravity))
    B = q.shape[0]
    I = m.inertias(theta)
    a0 = m.a0(B, dt, gravity)
    X, v, c, IA, pA = ([None] * m.n for _ in range(5))
    for i in range(m.n):
        X[i] = m.Xup(i, q)
        s = slice(m.vi[i], m.vi[i] + m.nvi[i])
        vJ = _mv(m.S[i], qd[:, s])
        p = m.parent[i]
        vp = np.zeros((B, 6), dtype=dt) if p < 0 else v[p]
        v[i] = _mv(X[i], vp) + vJ
        c[i] = _mv(sp.crm(v[i]), vJ)
        IA[i] = np.broadcast_to(I[i], (B, 6, 6)).astype(dt)
        pA[i] = _mv(sp.crf(v[i]), _mv(I[i], v[i]))
    U, Dinv, u = [None] * m.n, [None] * m.n, [None] * m.n
    for i in reversed(range(m.n)):
        S = m.S[i]
        s = slice(m.vi[i], m.vi[i] + m.nvi[i])
        p = m.parent[i]
        if m.nvi[i]:
            U[i] = IA[i] @ S
            D = np.swapaxes(S, -1, -2) @ U[i]
            Dinv[i] = np.linalg.inv(D)
            u[i] = tau[:, s] - _tv(S, pA[i])
            Ia = IA[i] - U[i] @ Dinv[i] @ np.swapaxes(U[i], -1, -2)
            pa = pA[i] + _mv(Ia, c[i]) + _mv(U[i], _mv(Dinv[i], u[i]))
        else:
            Ia = IA[i]
            pa = pA[i] + _mv(Ia, c[i])
        if p >= 0:
            IA[p] = IA[p] + np.swapaxes(X[i], -1, -2) @ Ia @ X[i]
            pA[p] = pA[p] + _tv(X[i], pa)
    qdd = np.zeros((B, m.nv), dtype=dt)
    a = [None] * m.n
    for i in range(m.n):
        p = m.parent[i]
        ap = a0 if p < 0 else a[p]
        a_ = _mv(X[i], ap) + c[i]
        if m.nvi[i]:
            s = slice(m.vi[i], m.vi[i] + m.nvi[i])
            qdd[:, s] = _mv(Dinv[i], u[i] - _tv(U[i], a_))
            a_ = a_ + _mv(m.S[i], qdd[:, s])
        a[i] = a_
    return qdd
