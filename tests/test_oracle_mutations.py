"""The oracle's pins have teeth: plausible mistakes planted in the oracle (on
the CPU, through monkeypatching its building blocks) each make at least one
pin fail. The mistakes are the kinds a restatement of the textbook
recursions makes: a dropped term, a wrong sign, a transposed operand, a
rotation the wrong way round."""
import numpy as np
import pytest

from oracle import rbd
from oracle import spatial as sp
from paper_2605_31481_gb300 import workloads as w

import test_oracle_dynamics as dyn
import test_oracle_grads as grads
import test_oracle_kinematics as kin


def _battery():
    """The pins run against every mistake, as (name, call) pairs."""
    chain, quad = w.chain(7), w.spined_quadruped()
    return [
        ("single pendulum", dyn.test_single_pendulum_closed_form),
        ("planar two-link", dyn.test_planar_two_link_closed_form),
        ("free body", lambda: dyn.test_free_body_matches_classical_newton_euler(0)),
        ("Lagrangian", lambda: dyn.test_recursions_match_lagrangian(lambda s: dyn._mixed_tree(s), 0)),
        ("invariants", lambda: dyn.test_invariants(quad)),
        ("power balance", lambda: dyn.test_power_balance(chain)),
        ("kinetic energy", lambda: dyn.test_kinetic_energy_from_body_twists(quad)),
        ("axis-angle", kin.test_axis_angle_matches_library_rotation),
        ("quaternion", kin.test_quaternion_matches_library_rotation),
        ("planar arm FK", kin.test_planar_arm_closed_form),
        ("Jacobian = pose derivative", lambda: kin.test_jacobian_equals_pose_derivative(0)),
        ("regressor", grads.test_regressor_reproduces_tau_and_fd),
    ]


_crm, _mcI, _pose_to_X, _pose_to_Xinv, _quat_to_R, _axis_angle_to_R = (
    sp.crm, sp.mcI, sp.pose_to_X, sp.pose_to_Xinv, sp.quat_to_R, sp.axis_angle_to_R)
_tv = rbd._tv


def _crm_transposed_block(v):
    w_, u = v[..., :3], v[..., 3:]
    W = sp.skew(w_)
    return sp.block(W, np.zeros_like(W), np.swapaxes(sp.skew(u), -1, -2), W)


def _mcI_no_parallel_axis(m, c, Ic):
    C = sp.skew(c)
    Ct = np.swapaxes(C, -1, -2)
    one = np.eye(3, dtype=np.result_type(m, c, Ic))
    return sp.block(Ic, m * C, m * Ct, m * one)


def _pose_to_X_untransposed(T):
    R, t = T[..., :3, :3], T[..., :3, 3]
    return sp.block(R, np.zeros_like(R), -R @ sp.skew(t), R)


def _pose_to_Xinv_no_offset(T):
    R = T[..., :3, :3]
    return sp.block(R, np.zeros_like(R), np.zeros_like(R), R)


MUTATIONS = {
    "force cross product without its minus sign": ("crf", lambda v: np.swapaxes(_crm(v), -1, -2)),
    "motion cross product with a transposed block": ("crm", _crm_transposed_block),
    "spatial inertia without the parallel-axis term": ("mcI", _mcI_no_parallel_axis),
    "motion transform with R instead of R^T": ("pose_to_X", _pose_to_X_untransposed),
    "inverse motion transform without the t x R term": ("pose_to_Xinv", _pose_to_Xinv_no_offset),
    "quaternion rotation transposed": ("quat_to_R", lambda qq: np.swapaxes(_quat_to_R(qq), -1, -2)),
    "axis-angle rotation the wrong way": ("axis_angle_to_R", lambda ax, an: _axis_angle_to_R(ax, -np.asarray(an))),
    "force propagation with X instead of X^T": (
        "rbd._tv", lambda M, v: rbd._mv(M, v) if M.shape[-2:] == (6, 6) else _tv(M, v)),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_every_planted_mistake_fails_a_pin(monkeypatch, name):
    target, fake = MUTATIONS[name]
    if target.startswith("rbd."):
        monkeypatch.setattr(rbd, target[4:], fake)
    else:
        monkeypatch.setattr(sp, target, fake)
    caught = []
    for pin, call in _battery():
        try:
            call()
        except (AssertionError, np.linalg.LinAlgError):
            caught.append(pin)
    assert caught, f"no pin fails with: {name}"


def test_the_battery_passes_on_the_oracle_as_it_stands():
    for _, call in _battery():
        call()
