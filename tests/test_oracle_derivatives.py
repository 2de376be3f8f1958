"""Pins of the oracle's dense dynamics derivatives (d tau / d q, d tau / d qd,
d qdd / d q, d qdd / d qd, d qdd / d tau) and of its tangent-space map:
closed forms of the planar two-link arm, central differences along scipy's
exact rotations, the base-pose invariance of a floating body, and the
implicit-function identities between forward and inverse dynamics."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import derivs, rbd
from paper_2605_31481_gb300 import workloads as w

G0 = 9.81


def _two_link():
    m1, m2, l1, c1, c2, I1, I2 = 1.3, 0.9, 0.6, 0.25, 0.3, 0.04, 0.03
    t = w.random_tree([-1, 0], [w.REVOLUTE] * 2, seed=1)
    t.axis[:] = [0, 0, 1]
    t.T_joint[:, 9:] = 0
    t.T_joint[1, 9] = l1
    t.mass[:] = [m1, m2]
    t.com[:] = [[c1, 0, 0], [c2, 0, 0]]
    t.I_com[:] = [[0.02, 0.001, 0.03, 0.002, 0.003, I1], [0.01, -0.002, 0.02, 0.001, -0.001, I2]]
    t.gravity = np.array([0, -G0, 0])
    return t, (m1, m2, l1, c1, c2, I1, I2)


def test_two_link_closed_form_derivatives():
    """tau1 = M11 qdd1 + M12 qdd2 - h (2 qd1 qd2 + qd2^2) + g1,
    tau2 = M12 qdd1 + M22 qdd2 + h qd1^2 + g2, h = m2 l1 c2 sin q2,
    differentiated by hand."""
    t, (m1, m2, l1, c1, c2, I1, I2) = _two_link()
    rng = np.random.default_rng(3)
    q, qd, qdd = (rng.uniform(-3, 3, (25, 2)) for _ in range(3))
    dq, dqd = derivs.rnea_derivatives(t, q, qd, qdd)
    q1, q2 = q[:, 0], q[:, 1]
    s2, c2q = np.sin(q2), np.cos(q2)
    h, dh = m2 * l1 * c2 * s2, m2 * l1 * c2 * c2q
    dM11, dM12 = -2 * m2 * l1 * c2 * s2, -m2 * l1 * c2 * s2
    gs1, gs12 = np.sin(q1), np.sin(q1 + q2)
    A, Bc = (m1 * c1 + m2 * l1) * G0, m2 * c2 * G0
    w1 = 2 * qd[:, 0] * qd[:, 1] + qd[:, 1] ** 2
    ref_dq = np.stack([
        np.stack([-A * gs1 - Bc * gs12, dM11 * qdd[:, 0] + dM12 * qdd[:, 1] - dh * w1 - Bc * gs12], -1),
        np.stack([-Bc * gs12, dM12 * qdd[:, 0] + dh * qd[:, 0] ** 2 - Bc * gs12], -1)], -2)
    ref_dqd = np.stack([
        np.stack([-2 * h * qd[:, 1], -2 * h * (qd[:, 0] + qd[:, 1])], -1),
        np.stack([2 * h * qd[:, 0], 0 * h], -1)], -2)
    np.testing.assert_allclose(dq, ref_dq, atol=1e-12)
    np.testing.assert_allclose(dqd, ref_dqd, atol=1e-12)


def _fd_along(tree, f, q, j, h=1e-6):
    """Central difference of f along tangent direction j, moving a free
    joint with scipy's exact rotation composition (independent of
    derivs.integrate)."""
    m = rbd.Model(tree)

    def moved(sgn):
        out = np.array(q, dtype=np.float64, copy=True)
        for i, t in enumerate(m.jtype):
            a, b = m.qi[i], m.vi[i]
            if t in (rbd.REVOLUTE, rbd.PRISMATIC) and b == j:
                out[:, a] += sgn * h
            elif t == rbd.FREE and b <= j < b + 6:
                k = j - b
                R = Rotation.from_quat(q[:, a + 3:a + 7])
                if k < 3:
                    e = np.zeros((len(q), 3))
                    e[:, k] = sgn * h
                    out[:, a:a + 3] += R.apply(e)
                else:
                    v = np.zeros(3)
                    v[k - 3] = sgn * h
                    out[:, a + 3:a + 7] = (R * Rotation.from_rotvec(v)).as_quat()
        return out
    return (f(moved(1)) - f(moved(-1))) / (2 * h)


@pytest.mark.parametrize("make", [lambda: w.chain(7, seed=0), lambda: w.spined_quadruped(seed=0),
                                  lambda: w.humanoid(seed=0)], ids=["chain7", "quadruped11", "humanoid29"])
def test_tangent_derivatives_match_central_differences(make):
    tree = make()
    s = w.random_state(tree, 6, seed=2)
    dq, dqd = derivs.rnea_derivatives(tree, s["q"], s["qd"], s["qdd"])
    f = lambda q_: rbd.rnea(tree, q_, s["qd"], s["qdd"])
    for j in range(tree.nv):
        fd = _fd_along(tree, f, s["q"], j)
        assert np.abs(dq[..., j] - fd).max() <= 1e-6 * max(np.abs(fd).max(), 1.0), j
    for j in range(tree.nv):
        e = np.zeros_like(s["qd"])
        e[:, j] = 1e-6
        fd = (rbd.rnea(tree, s["q"], s["qd"] + e, s["qdd"]) - rbd.rnea(tree, s["q"], s["qd"] - e, s["qdd"])) / 2e-6
        assert np.abs(dqd[..., j] - fd).max() <= 1e-6 * max(np.abs(fd).max(), 1.0), j


def test_floating_base_pose_enters_only_through_gravity():
    """A floating tree's inverse dynamics in body coordinates ignore where
    the base is; turning the base by dw (body frame) acts like turning
    gravity the other way: d tau / d dw_k = d tau / d g along R (g_b x e_k),
    g_b = R^T g the gravity in the base frame."""
    tree = w.humanoid(seed=1)
    s = w.random_state(tree, 5, seed=4)
    dq, _ = derivs.rnea_derivatives(tree, s["q"], s["qd"], s["qdd"])
    assert np.abs(dq[..., 0:3]).max() < 1e-11 * np.abs(dq).max()          # base translation
    R = Rotation.from_quat(s["q"][:, 3:7]).as_matrix()
    g = np.asarray(tree.gravity, dtype=np.float64)
    gb = np.einsum("bji,j->bi", R, g)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        dg = np.einsum("bij,bj->bi", R, np.cross(gb, e))
        ref = np.stack([np.imag(rbd.rnea(tree, s["q"][b:b + 1], s["qd"][b:b + 1], s["qdd"][b:b + 1],
                                         gravity=g + 1j * 1e-30 * dg[b])) / 1e-30 for b in range(len(R))])[:, 0]
        np.testing.assert_allclose(dq[..., 3 + k], ref, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("make", [lambda: w.spined_quadruped(seed=0), lambda: w.humanoid(seed=0)],
                         ids=["quadruped11", "humanoid29"])
def test_forward_dynamics_derivatives_identities(make):
    """d qdd / d tau = M^-1 and, at qdd = ABA(q, qd, tau), the implicit
    function identities d qdd / d q = -M^-1 d tau / d q and
    d qdd / d qd = -M^-1 d tau / d qd."""
    tree = make()
    s = w.random_state(tree, 5, seed=6)
    dq, dqd, dtau = derivs.aba_derivatives(tree, s["q"], s["qd"], s["tau"])
    Minv = np.linalg.inv(rbd.crba(tree, s["q"]))
    np.testing.assert_allclose(dtau, Minv, rtol=1e-9, atol=1e-9 * np.abs(Minv).max())
    qdd = rbd.aba(tree, s["q"], s["qd"], s["tau"])
    rq, rqd = derivs.rnea_derivatives(tree, s["q"], s["qd"], qdd)
    for got, r in ((dq, rq), (dqd, rqd)):
        ref = -np.einsum("bij,bjk->bik", Minv, r)
        np.testing.assert_allclose(got, ref, atol=1e-8 * np.abs(ref).max())


def test_integrate_first_order_matches_exact_motion():
    """The tangent map's first derivative equals that of the exact motion
    (scipy rotation vector, body-frame displacement)."""
    tree = w.humanoid(seed=2)
    s = w.random_state(tree, 4, seed=1)
    rng = np.random.default_rng(0)
    dv = rng.standard_normal((4, tree.nv))
    h = 1e-7
    num = (derivs.integrate(tree, s["q"], h * dv) - derivs.integrate(tree, s["q"], -h * dv)) / (2 * h)
    R = Rotation.from_quat(s["q"][:, 3:7])
    plus = (R * Rotation.from_rotvec(h * dv[:, 3:6])).as_quat()
    minus = (R * Rotation.from_rotvec(-h * dv[:, 3:6])).as_quat()
    np.testing.assert_allclose(num[:, 3:7], (plus - minus) / (2 * h), atol=1e-7)
    np.testing.assert_allclose(num[:, 0:3], R.apply(dv[:, 0:3]), atol=1e-7)
    np.testing.assert_allclose(num[:, 7:], dv[:, 6:], atol=1e-7)


@pytest.mark.parametrize("make", [lambda: w.spined_quadruped(seed=0), lambda: w.humanoid(seed=0)],
                         ids=["quadruped11", "humanoid29"])
def test_forward_dynamics_derivatives_match_central_differences(make):
    """d qdd / d q along the tangent directions (a free base moved by scipy's
    exact rotations), d qdd / d qd and d qdd / d tau against central
    differences of ABA itself."""
    tree = make()
    s = w.random_state(tree, 4, seed=8)
    dq, dqd, dtau = derivs.aba_derivatives(tree, s["q"], s["qd"], s["tau"])
    f = lambda q_: rbd.aba(tree, q_, s["qd"], s["tau"])
    for j in range(tree.nv):
        fd = _fd_along(tree, f, s["q"], j)
        assert np.abs(dq[..., j] - fd).max() <= 1e-6 * max(np.abs(fd).max(), 1.0), j
    for name, got in (("qd", dqd), ("tau", dtau)):
        for j in range(tree.nv):
            e = np.zeros_like(s[name])
            e[:, j] = 1e-6
            lo, hi = dict(s), dict(s)
            lo[name], hi[name] = s[name] - e, s[name] + e
            fd = (rbd.aba(tree, hi["q"], hi["qd"], hi["tau"]) - rbd.aba(tree, lo["q"], lo["qd"], lo["tau"])) / 2e-6
            assert np.abs(got[..., j] - fd).max() <= 1e-6 * max(np.abs(fd).max(), 1.0), (name, j)
