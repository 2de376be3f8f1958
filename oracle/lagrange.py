"""Brute-force Lagrangian dynamics: an independent route to M, C qd and g.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Used only to pin the recursive algorithms. For a tree without a free joint
(so qd = dq/dt), with world poses from `rbd.fk`:

    M(q)  = sum_i  m_i Jv_i^T Jv_i + Jw_i^T (R_i Ic_i R_i^T) Jw_i
    g(q)  = d PE / dq,     PE = - sum_i m_i g . p_com,i
    (C qd)_k = sum_ij (dM_kj/dq_i - 1/2 dM_ij/dq_k) qd_i qd_j
    tau   = M qdd + C qd + g

Jv_i is the Jacobian of body i's centre of mass and Jw_i maps qd to its
world angular velocity (from dR_i/dq R_i^T). Derivatives of FK and PE use the
complex-step method; dM/dq uses central differences of M.
"""
import numpy as np

from . import rbd, derivs
from . import spatial as sp


def _com_world(tree, q):
    T = rbd.fk(tree, q)
    c = np.asarray(tree.com, dtype=np.float64)
    return np.einsum("bnij,nj->bni", T[..., :3, :3], c) + T[..., :3, 3]


def mass_matrix(tree, q):
    q = np.asarray(q, dtype=np.float64)
    n = len(tree.parent)
    Jv = derivs.jac_cs(lambda q_: _com_world(tree, q_), (q,), 0)             # (B, n, 3, nq)
    Rf = lambda q_: rbd.fk(tree, q_)[..., :3, :3].reshape(q_.shape[0], n, 9)
    dR = derivs.jac_cs(Rf, (q,), 0).reshape(q.shape[0], n, 3, 3, -1)        # (B, n, 3, 3, nq)
    R = rbd.fk(tree, q)[..., :3, :3]
    W = np.einsum("bnijk,bnlj->bnilk", dR, R)                                # dR R^T, skew
    Jw = np.stack([W[:, :, 2, 1], W[:, :, 0, 2], W[:, :, 1, 0]], axis=2)      # (B, n, 3, nq)
    Ic = sp.sym6_to_3x3(np.asarray(tree.I_com, dtype=np.float64))            # (n, 3, 3)
    Iw = R @ Ic[None] @ np.swapaxes(R, -1, -2)
    m = np.asarray(tree.mass, dtype=np.float64)
    M = np.einsum("n,bnik,bnil->bkl", m, Jv, Jv) + np.einsum("bnik,bnij,bnjl->bkl", Jw, Iw, Jw)
    return M


def potential(tree, q):
    g = np.asarray(tree.gravity, dtype=np.float64)
    m = np.asarray(tree.mass, dtype=np.float64)
    return -np.einsum("n,bni,i->b", m, _com_world(tree, q), g)


def gravity_torque(tree, q):
    return derivs.jac_cs(lambda q_: potential(tree, q_)[:, None], (q,), 0)[:, 0, :]


def coriolis_times_qd(tree, q, qd, h=1e-5):
    q = np.asarray(q, dtype=np.float64)
    nq = q.shape[1]
    dM = []
    for i in range(nq):
        e = np.zeros_like(q)
        e[:, i] = h
        dM.append((mass_matrix(tree, q + e) - mass_matrix(tree, q - e)) / (2 * h))
    dM = np.stack(dM, axis=1)                                                # (B, i, k, j) = dM_kj/dq_i
    term1 = np.einsum("bikj,bi,bj->bk", dM, qd, qd)
    term2 = 0.5 * np.einsum("bkij,bi,bj->bk", dM, qd, qd)
    return term1 - term2


def inverse_dynamics(tree, q, qd, qdd):
    return (np.einsum("bij,bj->bi", mass_matrix(tree, q), qdd)
            + coriolis_times_qd(tree, q, qd) + gravity_torque(tree, q))


def kinetic_energy(tree, q, qd):
    M = mass_matrix(tree, q)
    return 0.5 * np.einsum("bi,bij,bj->b", qd, M, qd)
