"""The parity tests' error measures, on the CPU: the backward-error check
that the forward-dynamics adjoint and derivative tests use must accept a
stable FP32 solve however badly M is conditioned, and must reject the
mistakes a wrong kernel would make (a dropped term, a transposed operand, a
wrong sign)."""
import numpy as np

from oracle import rbd
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import env_err, solve_backward_err

BWD_BAR = 1e-5          # the bar of the forward-dynamics adjoint and derivative tests


def _fp32_solve(M, R):
    return np.linalg.solve(M.astype(np.float32), R.astype(np.float32)).astype(np.float64)


def test_backward_error_accepts_fp32_solves_at_any_conditioning():
    rng = np.random.default_rng(0)
    n, B = 12, 64
    U = np.linalg.qr(rng.standard_normal((B, n, n)))[0]
    for cond in (1e1, 1e4, 1e6):
        d = np.geomspace(1.0, 1.0 / cond, n)
        M = U @ (d[None, :, None] * np.swapaxes(U, 1, 2))
        r = rng.standard_normal((B, n))
        x = _fp32_solve(M, r[..., None])[..., 0]
        assert solve_backward_err(M, x, r).max() < 1e-5, cond
        # the forward error of the same solve grows with cond(M): that is why
        # the tests bound the backward error instead
        x64 = np.linalg.solve(M, r[..., None])[..., 0]
        if cond >= 1e6:
            assert env_err(x, x64).max() > 1e-4
        X = _fp32_solve(M, np.broadcast_to(np.eye(n), M.shape))
        assert solve_backward_err(M, X, np.broadcast_to(np.eye(n), M.shape)).max() < 1e-5


def test_backward_error_rejects_planted_mistakes():
    tree = w.humanoid(seed=0)
    s = w.random_state(tree, 16, seed=3)
    M = rbd.crba(tree, s["q"])
    rng = np.random.default_rng(1)
    r = rng.standard_normal((16, tree.nv))
    x = np.linalg.solve(M, r[..., None])[..., 0]
    assert solve_backward_err(M, x, r).max() < 1e-12
    wrong = {
        "sign": -x,
        "transposed operand": np.einsum("bji,bj->bi", np.linalg.inv(M) + 1e-2 * np.triu(np.ones_like(M), 1), r),
        "dropped entry": np.where(np.arange(tree.nv) == 7, 0.0, x),
        "1e-2 relative perturbation": x * (1 + 1e-2 * rng.standard_normal(x.shape)),
    }
    # a normwise backward error of a wrong answer can be as small as about
    # 1/cond(M) (here cond(M) is 2e3 to 4e3): the bar must sit well below it
    for name, xw in wrong.items():
        assert solve_backward_err(M, xw, r).min() > 3 * BWD_BAR, name
