"""Gradient-based identification of link inertial parameters (paper Sec. 4.3).

The paper recovers link masses by minimising
    sum_k || RNEA(q_k, qd_k, qdd_k; theta) - tau_meas_k ||^2
through autograd with L-BFGS. Here every iteration is one fused kernel
(fst_rnea_loss_grad: the loss and its gradient with respect to all 10
inertial parameters of every link, deterministic) followed by an Adam step on
the normalised parameters s = theta / theta_init, as plain torch ops on 10*n
numbers; or, since the loss is quadratic in theta, its exact minimiser from
10*n + 2 kernel calls (identify_least_squares). With world_size > 1 (torch.distributed initialised), each rank holds
a contiguous shard of the environments and the gradients and losses are
summed with one all-reduce per step.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


def shard(B: int, rank: int, world: int):
    """Contiguous environment range [lo, hi) of one rank."""
    base, extra = divmod(B, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_sum(t: torch.Tensor) -> torch.Tensor:
    """Sums t over ranks in place when torch.distributed is initialised."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def identify(model, q, qd, qdd, tau_meas, theta_init, steps=500, lr=1e-2, betas=(0.9, 0.999), eps=1e-8,
             history=False, state=None, return_state=False):
    """Adam on s = theta / theta_init minimising the squared torque error.

    q, qd, qdd, tau_meas: this rank's environments, (field, B) CUDA tensors.
    theta_init: (n_b, 10) float32 CUDA tensor (entries must be non-zero).
    Returns (theta, losses) with losses the per-step total loss if history.
    With return_state=True, also the optimiser state (a dict of tensors and
    the step count, suitable for torch.save); passing it back as `state`
    continues the run exactly where it stopped (checkpoint and resume: the
    loss-gradient reduction is deterministic, so a resumed run equals an
    uninterrupted one bit for bit)."""
    B = q.shape[1]
    if state is None:
        scale = theta_init.clone()
        s = torch.ones_like(theta_init)
        m = torch.zeros_like(s)
        v = torch.zeros_like(s)
        t0 = 0
    else:
        scale, s, m, v = (state[k].to(theta_init.device).clone() for k in ("scale", "s", "m", "v"))
        t0 = int(state["step"])
    scratch = api.adjoint_scratch(model, B)
    buf = torch.empty(theta_init.numel() + 1, device=theta_init.device)
    losses = []
    b1, b2 = betas
    for t in range(t0 + 1, t0 + steps + 1):
        theta = (s * scale).contiguous()
        api.rnea_loss_grad(model, q, qd, qdd, tau_meas, theta=theta, scratch=scratch, out=buf)
        allreduce_sum(buf)
        if history:
            losses.append(float(buf[-1]))
        g = buf[:-1].view_as(s) * scale            # d loss / d s
        m.mul_(b1).add_(g, alpha=1 - b1)
        v.mul_(b2).addcmul_(g, g, value=1 - b2)
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        s.sub_(lr * mh / (vh.sqrt() + eps))
    theta = (s * scale).contiguous()
    if return_state:
        return theta, losses, {"scale": scale, "s": s, "m": m, "v": v, "step": t0 + steps}
    return theta, losses


def identify_least_squares(model, q, qd, qdd, tau_meas, theta_init, rcond=1e-5):
    """Exact minimiser of the same loss, which is quadratic in theta (tau is
    linear in the inertial parameters): with s = theta / theta_init,
    L(s) = |Y D s - tau_meas|^2, D = diag(theta_init). Its Hessian
    H = 2 D Y^T Y D is built column by column from the fused loss-gradient
    kernel with zero measured torques (then grad = H s exactly, so column k
    is the gradient at s = e_k: 10 n_b kernel calls), the gradient g at the
    initial guess from one more call, and the step s = 1 - H^+ g is solved in
    FP64 with a pseudo-inverse that drops eigenvalues below rcond times the
    largest. Parameter combinations the data cannot determine (H's null
    space) keep their initial values. With torch.distributed initialised each
    rank passes its shard and every gradient is summed across ranks.
    Returns (theta, loss at theta) with the loss evaluated by the kernel."""
    n = theta_init.numel()
    scale = theta_init.reshape(-1).double()
    scratch = api.adjoint_scratch(model, q.shape[1])
    buf = torch.empty(n + 1, device=theta_init.device)
    zero_tau = torch.zeros_like(tau_meas)

    def grad(s_vec, tau):
        theta = (s_vec * scale).float().view_as(theta_init).contiguous()
        api.rnea_loss_grad(model, q, qd, qdd, tau, theta=theta, scratch=scratch, out=buf)
        allreduce_sum(buf)
        return buf[:-1].double() * scale, float(buf[-1])

    H = torch.empty(n, n, dtype=torch.float64, device=theta_init.device)
    for k in range(n):
        e = torch.zeros(n, dtype=torch.float64, device=theta_init.device)
        e[k] = 1.0
        H[:, k] = grad(e, zero_tau)[0]
    H = 0.5 * (H + H.T)
    ones = torch.ones(n, dtype=torch.float64, device=theta_init.device)
    g, _ = grad(ones, tau_meas)
    lam, V = torch.linalg.eigh(H)
    keep = lam > rcond * lam.abs().max()
    inv = torch.where(keep, 1.0 / torch.where(keep, lam, torch.ones_like(lam)), torch.zeros_like(lam))
    s_vec = ones - V @ (inv * (V.T @ g))
    theta = (s_vec * scale).float().view_as(theta_init).contiguous()
    _, loss = grad(s_vec, tau_meas)
    return theta, loss


def mass_directions(theta_known):
    """(n_b, 10) rows d theta / d m per link with the centre of mass and the
    rotational inertia about it held fixed: [1, c, S(c)], S(c) the
    parallel-axis term (xx, xy, yy, xz, yz, zz) of a unit mass at c."""
    th = theta_known.double()
    c = th[:, 1:4] / th[:, 0:1]
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    S = torch.stack([y * y + z * z, -x * y, x * x + z * z, -x * z, -y * z, x * x + y * y], dim=1)
    return torch.cat([torch.ones_like(x)[:, None], c, S], dim=1)


def identify_masses(model, q, qd, qdd, tau_meas, theta_known):
    """The paper's identification setting (Sec. 4.3): only the link masses
    are unknown, each link's centre of mass and rotational inertia about it
    are known (taken from theta_known). theta(m) is affine in the masses, so
    the least-squares masses solve a n_b x n_b system whose matrix and
    right-hand side come from n_b + 1 calls of the fused loss-gradient
    kernel (zero torques give the columns, the measured ones the gradient at
    the known parameters). Returns (masses (n_b,), theta at those masses)."""
    nb = theta_known.shape[0]
    phi = mass_directions(theta_known)                       # (n_b, 10)
    scratch = api.adjoint_scratch(model, q.shape[1])
    buf = torch.empty(nb * 10 + 1, device=theta_known.device)
    zero_tau = torch.zeros_like(tau_meas)

    def grad(theta64, tau):
        api.rnea_loss_grad(model, q, qd, qdd, tau, theta=theta64.float().contiguous(), scratch=scratch, out=buf)
        allreduce_sum(buf)
        return buf[:-1].double().view(nb, 10)

    H = torch.empty(nb, nb, dtype=torch.float64, device=theta_known.device)
    for k in range(nb):
        d = torch.zeros(nb, 10, dtype=torch.float64, device=theta_known.device)
        d[k] = phi[k]
        H[:, k] = (grad(d, zero_tau) * phi).sum(dim=1)        # Phi^T (2 Y^T Y) Phi e_k
    H = 0.5 * (H + H.T)
    base = theta_known.double()
    g = (grad(base, tau_meas) * phi).sum(dim=1)              # gradient in the masses at theta_known
    dm = torch.linalg.solve(H, -g)
    m = base[:, 0] + dm
    theta = base + dm[:, None] * phi
    return m.float(), theta.float().contiguous()


def mass_errors(theta, true_theta):
    """Per-link relative mass error |m_hat - m| / m (numpy)."""
    th = np.asarray(theta.detach().cpu() if isinstance(theta, torch.Tensor) else theta, dtype=np.float64)
    tr = np.asarray(true_theta, dtype=np.float64)
    return np.abs(th[:, 0] - tr[:, 0]) / tr[:, 0]
