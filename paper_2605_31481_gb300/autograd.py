"""torch.autograd.Function wrappers: the forward calls the library's
operator, the backward its hand-written adjoint (fst_*_vjp). Tensors use the
binding's structure-of-arrays layout (field, B); theta is (n_b, 10) or None
(then the model's own inertias are used and get no gradient)."""
from __future__ import annotations

import torch

from . import api


class RNEAFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, model, q, qd, qdd, theta):
        ctx.model = model
        ctx.save_for_backward(q, qd, qdd, theta)
        return api.rnea(model, q, qd, qdd, theta=theta)

    @staticmethod
    def backward(ctx, tau_bar):
        q, qd, qdd, theta = ctx.saved_tensors
        need = ctx.needs_input_grad
        r = api.rnea_vjp(ctx.model, q, qd, qdd, tau_bar.contiguous(), theta=theta, q_bar=need[1], qd_bar=need[2],
                         qdd_bar=need[3], theta_bar=theta is not None and need[4])
        return None, r.get("q"), r.get("qd"), r.get("qdd"), r.get("theta")


class RNEAStoredFunction(torch.autograd.Function):
    """RNEA whose forward keeps the sweep state on a tape (fst_rnea_store)
    and whose backward reads it (fst_rnea_vjp_stored) instead of recomputing
    the forward sweep: 120 bytes per body and environment of memory and
    traffic traded for the forward sweep's arithmetic."""

    @staticmethod
    def forward(ctx, model, q, qd, qdd, theta):
        ctx.model = model
        tau, tape = api.rnea_store(model, q, qd, qdd, theta=theta)
        ctx.save_for_backward(q, qd, theta, tape)
        return tau

    @staticmethod
    def backward(ctx, tau_bar):
        q, qd, theta, tape = ctx.saved_tensors
        need = ctx.needs_input_grad
        r = api.rnea_vjp_stored(ctx.model, q, qd, tape, tau_bar.contiguous(), theta=theta, q_bar=need[1],
                                qd_bar=need[2], qdd_bar=need[3], theta_bar=theta is not None and need[4])
        return None, r.get("q"), r.get("qd"), r.get("qdd"), r.get("theta")


class ABAFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, model, q, qd, tau, theta):
        qdd = api.aba(model, q, qd, tau, theta=theta)
        ctx.model = model
        ctx.save_for_backward(q, qd, qdd, theta)
        return qdd

    @staticmethod
    def backward(ctx, qdd_bar):
        q, qd, qdd, theta = ctx.saved_tensors
        need = ctx.needs_input_grad
        r = api.aba_vjp(ctx.model, q, qd, qdd, qdd_bar.contiguous(), theta=theta, q_bar=need[1], qd_bar=need[2],
                        tau_bar=need[3], theta_bar=theta is not None and need[4])
        return None, r.get("q"), r.get("qd"), r.get("tau"), r.get("theta")


class FKFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, model, q):
        ctx.model = model
        ctx.save_for_backward(q)
        return api.fk(model, q)

    @staticmethod
    def backward(ctx, poses_bar):
        (q,) = ctx.saved_tensors
        return None, api.fk_vjp(ctx.model, q, poses_bar.contiguous())


def rnea(model, q, qd, qdd, theta=None, store=False):
    """Differentiable inverse dynamics tau (nv, B). store=True keeps the
    forward sweep's state for the backward (store variant) instead of
    recomputing it there."""
    if store:
        return RNEAStoredFunction.apply(model, q, qd, qdd, theta)
    return RNEAFunction.apply(model, q, qd, qdd, theta)


def aba(model, q, qd, tau, theta=None):
    """Differentiable forward dynamics qdd (nv, B)."""
    return ABAFunction.apply(model, q, qd, tau, theta)


def fk(model, q):
    """Differentiable forward kinematics (n_b, 12, B)."""
    return FKFunction.apply(model, q)
