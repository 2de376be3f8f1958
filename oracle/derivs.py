"""Exact derivatives of the oracle's functions.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper obtains gradients by automatic differentiation through its
operators (Sec. 3.5, Sec. 4.3). The oracle needs reference gradients that do
not depend on any adjoint derivation, so it uses:

* the complex-step method: for a real-analytic f, f'(x) dx =
  Im f(x + i h dx) / h, exact to rounding for tiny h (no subtraction, so
  h = 1e-30 is fine). Every oracle routine is written with analytic
  operations only, so it runs unchanged on complex128 inputs;
* the inertial-parameter regressor: tau is linear in the 10 parameters of
  every body, tau = Y(q, qd, qdd) theta, so Y's columns are RNEA evaluated at
  unit parameter vectors.
"""
import numpy as np

from . import rbd
from . import spatial as sp

H_CS = 1e-30


def jvp_cs(f, xs, k, dx):
    """Directional derivative of f(*xs) along dx in argument k."""
    args = [np.asarray(x, dtype=np.complex128) for x in xs]
    args[k] = args[k] + 1j * H_CS * np.asarray(dx)
    return np.imag(f(*args)) / H_CS


def jac_cs(f, xs, k):
    """Per-environment Jacobian d f / d xs[k]: (B, out..., n_k) for a batched
    argument of shape (B, n_k)."""
    x = np.asarray(xs[k])
    cols = []
    for j in range(x.shape[-1]):
        e = np.zeros_like(x, dtype=np.float64)
        e[..., j] = 1.0
        cols.append(jvp_cs(f, xs, k, e))
    return np.stack(cols, axis=-1)


def regressor(tree, q, qd, qdd, gravity=None):
    """Y (B, nv, n_b, 10) with tau = sum Y[..., b, k] theta[b, k]."""
    n = len(tree.parent)
    B = np.asarray(q).shape[0]
    nv = np.asarray(qd).shape[1]
    Y = np.zeros((B, nv, n, 10))
    for b in range(n):
        for k in range(10):
            th = np.zeros((n, 10))
            th[b, k] = 1.0
            Y[:, :, b, k] = rbd.rnea(tree, q, qd, qdd, theta=th, gravity=gravity)
    return Y


# ---------------------------------------------------------------------------
# reference vector-Jacobian products (what the adjoint kernels must return)
# ---------------------------------------------------------------------------

def rnea_vjp(tree, q, qd, qdd, tau_bar, theta=None):
    """Cotangents of tau = RNEA(q, qd, qdd; theta) for an incoming tau_bar:
    q_bar, qd_bar, qdd_bar (per environment) and theta_bar (summed over
    environments)."""
    m = rbd.Model(tree)
    th = m.theta() if theta is None else np.asarray(theta, dtype=np.float64)
    f = lambda q_, qd_, qdd_: rbd.rnea(tree, q_, qd_, qdd_, theta=th)
    out = []
    for k in range(3):
        J = jac_cs(f, (q, qd, qdd), k)                   # (B, nv, n_k)
        out.append(np.einsum("bi,bij->bj", tau_bar, J))
    Y = regressor(tree, q, qd, qdd)
    th_bar = np.einsum("bi,bink->nk", tau_bar, Y)
    return out[0], out[1], out[2], th_bar


def aba_vjp(tree, q, qd, tau, qdd_bar, theta=None):
    """Cotangents of qdd = ABA(q, qd, tau; theta): q_bar, qd_bar, tau_bar
    (per environment) and theta_bar (summed over environments)."""
    m = rbd.Model(tree)
    th = m.theta() if theta is None else np.asarray(theta, dtype=np.float64)
    f = lambda q_, qd_, tau_: rbd.aba(tree, q_, qd_, tau_, theta=th)
    out = []
    for k in range(3):
        J = jac_cs(f, (q, qd, tau), k)
        out.append(np.einsum("bi,bij->bj", qdd_bar, J))
    g = lambda th_: rbd.aba(tree, np.asarray(q, np.complex128), np.asarray(qd, np.complex128),
                            np.asarray(tau, np.complex128), theta=th_)
    n = th.shape[0]
    th_bar = np.zeros((n, 10))
    for b in range(n):
        for k in range(10):
            d = np.zeros((n, 10), dtype=np.complex128)
            d[b, k] = 1j * H_CS
            dq = np.imag(g(th.astype(np.complex128) + d)) / H_CS
            th_bar[b, k] = np.sum(qdd_bar * dq)
    return out[0], out[1], out[2], th_bar


def fk_vjp(tree, q, poses_bar):
    """q_bar for the cotangent poses_bar (B, n_b, 12) of the FK output
    laid out as R row-major (9) then p (3) per body."""
    def f(q_):
        T = rbd.fk(tree, q_)
        return np.concatenate([T[..., :3, :3].reshape(T.shape[:2] + (9,)), T[..., :3, 3]], axis=-1)
    J = jac_cs(f, (q,), 0)                                # (B, n_b, 12, nq)
    return np.einsum("bnk,bnkj->bj", poses_bar, J)


# ---------------------------------------------------------------------------
# dense derivatives along the configuration's tangent space
# ---------------------------------------------------------------------------

def integrate(tree, q, dv):
    """q (+) dv: the configuration moved along a tangent vector dv (B, nv).

    Revolute and prismatic coordinates add. A free joint moves its frame by
    the displacement dv = [dp; dw] expressed in that moving frame: the
    position gains R(quat) dp and the quaternion is multiplied on the right
    by (dw / 2, 1), the rotation about the body-frame axis dw to first order.
    The map is exact to first order at dv = 0, the only place the
    derivatives below evaluate it. Analytic, so complex steps pass through."""
    m = rbd.Model(tree)
    q = np.asarray(q)
    dv = np.asarray(dv)
    dt = np.result_type(q.dtype, dv.dtype)
    out = np.array(q, dtype=dt, copy=True)
    for i, t in enumerate(m.jtype):
        a, b = m.qi[i], m.vi[i]
        if t in (rbd.REVOLUTE, rbd.PRISMATIC):
            out[:, a] = q[:, a] + dv[:, b]
        elif t == rbd.FREE:
            quat = q[:, a + 3:a + 7]
            R = sp.quat_to_R(quat)
            out[:, a:a + 3] = q[:, a:a + 3] + np.einsum("bij,bj->bi", R, dv[:, b:b + 3])
            x1, y1, z1, w1 = np.moveaxis(quat, -1, 0)
            x2, y2, z2 = np.moveaxis(dv[:, b + 3:b + 6] / 2, -1, 0)
            # Hamilton product (x1, y1, z1, w1) (x) (x2, y2, z2, 1)
            out[:, a + 3] = w1 * x2 + x1 + y1 * z2 - z1 * y2
            out[:, a + 4] = w1 * y2 + y1 + z1 * x2 - x1 * z2
            out[:, a + 5] = w1 * z2 + z1 + x1 * y2 - y1 * x2
            out[:, a + 6] = w1 - (x1 * x2 + y1 * y2 + z1 * z2)
    return out


def tangent_jac_cs(f, tree, q, nv):
    """d f(q (+) dv) / d dv at dv = 0, per environment: (B, out..., nv)."""
    B = np.asarray(q).shape[0]
    cols = []
    for j in range(nv):
        dv = np.zeros((B, nv), dtype=np.complex128)
        dv[:, j] = 1j * H_CS
        cols.append(np.imag(f(integrate(tree, np.asarray(q, np.complex128), dv))) / H_CS)
    return np.stack(cols, axis=-1)


def rnea_derivatives(tree, q, qd, qdd, theta=None):
    """Dense derivatives of inverse dynamics: d tau / d q along the tangent
    directions of `integrate` and d tau / d qd, each (B, nv, nv) with row =
    tau component, column = direction. (d tau / d qdd is the mass matrix.)"""
    m = rbd.Model(tree)
    th = m.theta() if theta is None else np.asarray(theta, dtype=np.float64)
    qdc, qddc = np.asarray(qd, np.complex128), np.asarray(qdd, np.complex128)
    dq = tangent_jac_cs(lambda q_: rbd.rnea(tree, q_, qdc, qddc, theta=th), tree, q, m.nv)
    dqd = jac_cs(lambda q_, qd_, qdd_: rbd.rnea(tree, q_, qd_, qdd_, theta=th), (q, qd, qdd), 1)
    return dq, dqd


def aba_derivatives(tree, q, qd, tau, theta=None):
    """Dense derivatives of forward dynamics qdd = ABA(q, qd, tau): d qdd / d q
    (tangent directions), d qdd / d qd and d qdd / d tau (= M^-1), each
    (B, nv, nv), by complex steps of the oracle's ABA."""
    m = rbd.Model(tree)
    th = m.theta() if theta is None else np.asarray(theta, dtype=np.float64)
    qdc, tauc = np.asarray(qd, np.complex128), np.asarray(tau, np.complex128)
    dq = tangent_jac_cs(lambda q_: rbd.aba(tree, q_, qdc, tauc, theta=th), tree, q, m.nv)
    f = lambda q_, qd_, tau_: rbd.aba(tree, q_, qd_, tau_, theta=th)
    return dq, jac_cs(f, (q, qd, tau), 1), jac_cs(f, (q, qd, tau), 2)


# ---------------------------------------------------------------------------
# adjoints of the Jacobian and of the mass matrix
# ---------------------------------------------------------------------------

def jacobian_vjp(tree, q, links, J_bar):
    """q_bar (B, nq) for the cotangent J_bar (B, n_links, 6, nv) of the
    Jacobians of `links` (rows [v; w], the layout of rbd.jacobian)."""
    def f(q_):
        return np.stack([rbd.jacobian(tree, q_, l) for l in links], axis=1)
    J = jac_cs(f, (q,), 0)                                # (B, L, 6, nv, nq)
    return np.einsum("blrc,blrcj->bj", J_bar, J)


def crba_vjp(tree, q, M_bar, theta=None):
    """Cotangents of M = CRBA(q; theta) for M_bar (B, nv, nv): q_bar (B, nq)
    by complex steps, and theta_bar (n_b, 10) summed over environments, exact
    because M is linear in theta (M = sum theta_bk CRBA(q; unit theta_bk))."""
    m = rbd.Model(tree)
    th = m.theta() if theta is None else np.asarray(theta, dtype=np.float64)
    J = jac_cs(lambda q_: rbd.crba(tree, q_, theta=th), (q,), 0)   # (B, nv, nv, nq)
    q_bar = np.einsum("brc,brcj->bj", M_bar, J)
    n = th.shape[0]
    th_bar = np.zeros((n, 10))
    for b in range(n):
        for k in range(10):
            u = np.zeros((n, 10))
            u[b, k] = 1.0
            th_bar[b, k] = np.sum(M_bar * rbd.crba(tree, q, theta=u))
    return q_bar, th_bar
