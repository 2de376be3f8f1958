"""Shared helpers of the parity tests: run the oracle and the CUDA path on
the same seeded inputs and measure the per-environment error."""
import numpy as np

from oracle import rbd

# Per-output tolerances on the per-environment normwise relative error
#   err_e = max|x_gpu - x_ref| / max(max|x_ref|, 1)
# FP32 kernels against the FP64 oracle: 1e-5 for poses and Jacobians,
# 1e-4 for tau, M and qdd.
TOL = {"poses": 1e-5, "J": 1e-5, "tau": 1e-4, "M": 1e-4, "qdd": 1e-4}


def env_err(gpu, ref):
    """gpu, ref: (B, ...) arrays -> (B,) normwise relative error."""
    B = ref.shape[0]
    g = np.asarray(gpu, dtype=np.float64).reshape(B, -1)
    r = np.asarray(ref, dtype=np.float64).reshape(B, -1)
    if g.shape[1] == 0:
        return np.zeros(B)
    num = np.abs(g - r).max(axis=1)
    den = np.maximum(np.abs(r).max(axis=1), 1.0)
    return num / den


def to_soa_cuda(x, torch):
    """(B, n) float64 numpy -> (n, B) float32 CUDA tensor."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float32).T)).cuda()


def from_soa(t):
    """(..., B) tensor -> (B, ...) float64 numpy."""
    a = t.detach().cpu().numpy().astype(np.float64)
    return np.moveaxis(a, -1, 0)


def oracle_poses(tree, q):
    T = rbd.fk(tree, q)
    return np.concatenate([T[..., :3, :3].reshape(T.shape[:2] + (9,)), T[..., :3, 3]], axis=-1)


def _inf_norm(x):
    """Per-environment infinity norm: max |x| of a (B, n) vector, max row sum
    of |x| of a (B, n, m) matrix."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    return x.max(axis=1) if x.ndim == 2 else x.sum(axis=2).max(axis=1)


def solve_backward_err(M, X, R):
    """Normwise backward error of X as a solution of M X = R, per
    environment: ||M X - R|| / (||M|| ||X|| + ||R||) in the infinity norm.
    M (B, n, n); X, R both (B, n) or both (B, n, k). A backward-stable FP32
    solve keeps it at a small multiple of n times the unit roundoff 6e-8,
    whatever the conditioning of M (Higham, Accuracy and Stability of
    Numerical Algorithms, Sec. 7.1)."""
    M = np.asarray(M, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    vec = X.ndim == 2
    MX = np.einsum("bij,bj->bi", M, X) if vec else M @ X
    return _inf_norm(MX - R) / (_inf_norm(M) * _inf_norm(X) + _inf_norm(R))
