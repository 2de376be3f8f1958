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
