"""Spatial (Plucker) algebra in Featherstone's convention.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Motion vectors are [omega; v] and force vectors [n; f] (angular first). All
functions broadcast over leading axes and keep the input dtype, so they work
unchanged under the complex-step method.
"""
import numpy as np


def skew(v):
    """3-vector -> 3x3 cross-product matrix, so that skew(a) @ b = a x b."""
    v = np.asarray(v)
    z = np.zeros_like(v[..., 0])
    return np.stack([
        np.stack([z, -v[..., 2], v[..., 1]], axis=-1),
        np.stack([v[..., 2], z, -v[..., 0]], axis=-1),
        np.stack([-v[..., 1], v[..., 0], z], axis=-1),
    ], axis=-2)


def block(A, B, C, D):
    """Assemble [[A, B], [C, D]] from four (..., 3, 3) blocks."""
    top = np.concatenate([A, B], axis=-1)
    bot = np.concatenate([C, D], axis=-1)
    return np.concatenate([top, bot], axis=-2)


def crm(v):
    """Motion cross-product operator v x (Featherstone eq. 2.31)."""
    w, u = v[..., :3], v[..., 3:]
    W = skew(w)
    return block(W, np.zeros_like(W), skew(u), W)


def crf(v):
    """Force cross-product operator v x* = -crm(v)^T (Featherstone eq. 2.32)."""
    return -np.swapaxes(crm(v), -1, -2)


def pose_to_X(T):
    """Motion transform from frame a to frame b, where T (4x4) is the pose of
    b expressed in a: E = R^T, r = t, X = [[E, 0], [-E r x, E]]."""
    R = T[..., :3, :3]
    t = T[..., :3, 3]
    E = np.swapaxes(R, -1, -2)
    return block(E, np.zeros_like(E), -E @ skew(t), E)


def pose_to_Xinv(T):
    """Motion transform from frame b back to frame a (inverse of pose_to_X):
    [[R, 0], [t x R, R]]."""
    R = T[..., :3, :3]
    t = T[..., :3, 3]
    return block(R, np.zeros_like(R), skew(t) @ R, R)


def mcI(m, c, Ic):
    """Rigid-body spatial inertia at the frame origin from mass m, centre of
    mass c and rotational inertia Ic about the centre of mass (Featherstone
    eq. 2.63): [[Ic + m C C^T, m C], [m C^T, m 1]] with C = c x."""
    C = skew(c)
    Ct = np.swapaxes(C, -1, -2)
    one = np.eye(3, dtype=np.result_type(m, c, Ic))
    return block(Ic + m * C @ Ct, m * C, m * Ct, m * one)


def inertia_from_theta(theta):
    """Spatial inertia from the 10 linear parameters
    [m, hx, hy, hz, Ixx, Ixy, Iyy, Ixz, Iyz, Izz] with h = m c and I the
    rotational inertia about the frame origin: [[I, h x], [(h x)^T, m 1]]."""
    th = np.asarray(theta)
    m = th[..., 0]
    h = th[..., 1:4]
    Ixx, Ixy, Iyy, Ixz, Iyz, Izz = (th[..., 4 + k] for k in range(6))
    I = np.stack([np.stack([Ixx, Ixy, Ixz], -1),
                  np.stack([Ixy, Iyy, Iyz], -1),
                  np.stack([Ixz, Iyz, Izz], -1)], -2)
    H = skew(h)
    one = np.eye(3, dtype=th.dtype)
    return block(I, H, np.swapaxes(H, -1, -2), m[..., None, None] * one)


def sym6_to_3x3(s):
    """(xx, xy, yy, xz, yz, zz) -> symmetric 3x3."""
    s = np.asarray(s)
    return np.stack([np.stack([s[..., 0], s[..., 1], s[..., 3]], -1),
                     np.stack([s[..., 1], s[..., 2], s[..., 4]], -1),
                     np.stack([s[..., 3], s[..., 4], s[..., 5]], -1)], -2)


def theta_from_inertia(I6x6):
    """Inverse of inertia_from_theta for a rigid-body inertia."""
    I6 = np.asarray(I6x6)
    m = I6[..., 5, 5]
    h = np.stack([I6[..., 2, 4], I6[..., 0, 5], I6[..., 1, 3]], -1)
    Ir = I6[..., :3, :3]
    return np.concatenate([m[..., None], h,
                           np.stack([Ir[..., 0, 0], Ir[..., 0, 1], Ir[..., 1, 1],
                                     Ir[..., 0, 2], Ir[..., 1, 2], Ir[..., 2, 2]], -1)], -1)


def quat_to_R(quat):
    """Rotation matrix of the unit quaternion (x, y, z, w) after normalising
    it by sqrt(x^2 + y^2 + z^2 + w^2) (an analytic function, so the
    complex-step method passes through it)."""
    quat = np.asarray(quat)
    n = np.sqrt(np.sum(quat * quat, axis=-1, keepdims=True))
    x, y, z, w = np.moveaxis(quat / n, -1, 0)
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def axis_angle_to_R(axis, angle):
    """Rotation by `angle` about the unit `axis`, built from the quaternion
    (sin(angle/2) axis, cos(angle/2))."""
    angle = np.asarray(angle)
    s = np.sin(angle / 2)[..., None]
    c = np.cos(angle / 2)[..., None]
    quat = np.concatenate([s * np.asarray(axis), c], axis=-1)
    return quat_to_R(quat)


def homog(R, t):
    """4x4 homogeneous transform from R (..., 3, 3) and t (..., 3)."""
    R = np.asarray(R)
    t = np.asarray(t)
    dt = np.result_type(R, t)
    shape = np.broadcast_shapes(R.shape[:-2], t.shape[:-1])
    T = np.zeros(shape + (4, 4), dtype=dt)
    T[..., :3, :3] = R
    T[..., :3, 3] = t
    T[..., 3, 3] = 1
    return T


def T12_to_homog(T12):
    """(R row-major 9, t 3) -> 4x4."""
    T12 = np.asarray(T12)
    return homog(T12[..., :9].reshape(T12.shape[:-1] + (3, 3)), T12[..., 9:12])
