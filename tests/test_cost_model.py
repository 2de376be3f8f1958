"""The FP32 flop model of `costs.py` against a count.

The operator bodies of the kernels (world poses, Jacobian columns, the RNEA
sweeps, CRBA with 10-parameter composite inertias, ABA with 21-entry
articulated inertias) are restated here over a counting scalar, operation for
operation as the device code evaluates them: + - * / and sqrt count one flop,
a fused multiply-add two, a sign flip nothing; sin/cos pairs are counted
apart. The restatement's results are first held to the FP64 oracle, so the
count is of arithmetic that computes the right thing; the counts must then
equal `costs.flops` for every operator on chains, branched and floating
trees, and trees with prismatic and fixed joints."""
import math

import numpy as np
import pytest

from oracle import rbd
from paper_2605_31481_gb300 import costs
from paper_2605_31481_gb300 import workloads as w

FIXED, REVOLUTE, PRISMATIC, FREE = w.FIXED, w.REVOLUTE, w.PRISMATIC, w.FREE
COUNT = {"flops": 0, "sincos": 0}


def _v(x):
    return x.x if isinstance(x, F) else x


class F:
    """A float that counts the arithmetic done on it."""
    __slots__ = ("x",)

    def __init__(self, x):
        self.x = float(_v(x))

    def _op(self, other, f):
        COUNT["flops"] += 1
        return F(f(self.x, _v(other)))

    def __add__(self, o): return self._op(o, lambda a, b: a + b)
    def __radd__(self, o): return self._op(o, lambda a, b: b + a)
    def __sub__(self, o): return self._op(o, lambda a, b: a - b)
    def __rsub__(self, o): return self._op(o, lambda a, b: b - a)
    def __mul__(self, o): return self._op(o, lambda a, b: a * b)
    def __rmul__(self, o): return self._op(o, lambda a, b: b * a)
    def __truediv__(self, o): return self._op(o, lambda a, b: a / b)
    def __rtruediv__(self, o): return self._op(o, lambda a, b: b / a)
    def __neg__(self): return F(-self.x)


def fma(a, b, c):
    COUNT["flops"] += 2
    return F(_v(a) * _v(b) + _v(c))


def sqrt(a):
    COUNT["flops"] += 1
    return F(math.sqrt(_v(a)))


def rsqrt(a):
    COUNT["flops"] += 1
    return F(1.0 / math.sqrt(_v(a)))


def sincos(a):
    COUNT["sincos"] += 1
    return F(math.sin(_v(a))), F(math.cos(_v(a)))


Z = F(0.0)      # zeros the kernels hold in registers and compute with


# 3-vectors are lists of 3, spatial vectors pairs (w, v) of 3-vectors.
def add3(a, b): return [a[k] + b[k] for k in range(3)]
def sub3(a, b): return [a[k] - b[k] for k in range(3)]
def scale3(s, a): return [s * a[k] for k in range(3)]
def dot3(a, b): return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]))


def cross(a, b):
    return [fma(a[1], b[2], -(a[2] * b[1])), fma(a[2], b[0], -(a[0] * b[2])), fma(a[0], b[1], -(a[1] * b[0]))]


def Rmul(R, x): return [fma(R[3 * r], x[0], fma(R[3 * r + 1], x[1], R[3 * r + 2] * x[2])) for r in range(3)]
def RTmul(R, x): return [fma(R[r], x[0], fma(R[3 + r], x[1], R[6 + r] * x[2])) for r in range(3)]
def sadd(a, b): return (add3(a[0], b[0]), add3(a[1], b[1]))
def ssub(a, b): return (sub3(a[0], b[0]), sub3(a[1], b[1]))
def sscale(s, a): return (scale3(s, a[0]), scale3(s, a[1]))
def sdot(a, b): return dot3(a[0], b[0]) + dot3(a[1], b[1])
def szero(): return ([Z] * 3, [Z] * 3)


def X_motion(X, m):
    R, t = X
    return (RTmul(R, m[0]), RTmul(R, sub3(m[1], cross(t, m[0]))))


def XT_force(X, f):
    R, t = X
    fl = Rmul(R, f[1])
    return (add3(Rmul(R, f[0]), cross(t, fl)), fl)


def crm(v, m): return (cross(v[0], m[0]), add3(cross(v[0], m[1]), cross(v[1], m[0])))
def crf(v, f): return (add3(cross(v[0], f[0]), cross(v[1], f[1])), cross(v[0], f[1]))


def sym_mul(I, x):
    return [fma(I[0], x[0], fma(I[1], x[1], I[3] * x[2])), fma(I[1], x[0], fma(I[2], x[1], I[4] * x[2])),
            fma(I[3], x[0], fma(I[4], x[1], I[5] * x[2]))]


def in_mul(I, m):
    mass, h, Io = I
    return (add3(sym_mul(Io, m[0]), cross(h, m[1])), sub3(scale3(mass, m[1]), cross(h, m[0])))


def in_add(a, b): return (a[0] + b[0], add3(a[1], b[1]), [a[2][k] + b[2][k] for k in range(6)])


def sym_rot(R, S):
    P = []
    for r in range(3):
        P += sym_mul(S, [R[3 * r], R[3 * r + 1], R[3 * r + 2]])
    pairs = ((0, 0), (0, 1), (1, 1), (0, 2), (1, 2), (2, 2))
    return [fma(P[3 * a], R[3 * b], fma(P[3 * a + 1], R[3 * b + 1], P[3 * a + 2] * R[3 * b + 2])) for a, b in pairs]


def in_to_parent(X, I):
    R, t = X
    mass, h, Io = I
    y = Rmul(R, h)
    ho = add3(y, scale3(mass, t))
    o = sym_rot(R, Io)
    d = fma(2.0, dot3(y, t), mass * dot3(t, t))
    z = add3(y, scale3(0.5 * mass, t))
    o[0] = o[0] + (d - 2.0 * z[0] * t[0])
    o[1] = o[1] - fma(z[0], t[1], t[0] * z[1])
    o[2] = o[2] + (d - 2.0 * z[1] * t[1])
    o[3] = o[3] - fma(z[0], t[2], t[0] * z[2])
    o[4] = o[4] - fma(z[1], t[2], t[1] * z[2])
    o[5] = o[5] + (d - 2.0 * z[2] * t[2])
    return (mass, ho, o)


def sym6_from_in(I):
    mass, h, Io = I
    Bk = [Z, -h[2], h[1], h[2], Z, -h[0], -h[1], h[0], Z]
    return (list(Io), Bk, [mass, Z, mass, Z, Z, mass])


def sym6_mul(s, m):
    A, Bk, C = s
    return (add3(sym_mul(A, m[0]), Rmul(Bk, m[1])), add3(RTmul(Bk, m[0]), sym_mul(C, m[1])))


def sym6_add(a, b):
    return ([a[0][k] + b[0][k] for k in range(6)], [a[1][k] + b[1][k] for k in range(9)],
            [a[2][k] + b[2][k] for k in range(6)])


def sym6_rank1_sub(s, U, invD):
    A, Bk, C = [list(x) for x in s]
    n, f = U
    ns, fs = scale3(invD, n), scale3(invD, f)
    pairs = ((0, 0), (0, 1), (1, 1), (0, 2), (1, 2), (2, 2))
    for k, (a, b) in enumerate(pairs):
        A[k] = A[k] - ns[a] * n[b]
        C[k] = C[k] - fs[a] * f[b]
    for a in range(3):
        for b in range(3):
            Bk[3 * a + b] = Bk[3 * a + b] - ns[a] * f[b]
    return (A, Bk, C)


def full_rot(R, M):
    P = [fma(R[3 * r], M[c], fma(R[3 * r + 1], M[3 + c], R[3 * r + 2] * M[6 + c])) for r in range(3) for c in range(3)]
    return [fma(P[3 * r], R[3 * c], fma(P[3 * r + 1], R[3 * c + 1], P[3 * r + 2] * R[3 * c + 2]))
            for r in range(3) for c in range(3)]


def sym6_to_parent(X, s):
    R, (tx, ty, tz) = X
    A, Bk, C = s
    oA, oC, Bp = sym_rot(R, A), sym_rot(R, C), full_rot(R, Bk)
    Cf = [oC[0], oC[1], oC[3], oC[1], oC[2], oC[4], oC[3], oC[4], oC[5]]
    W = [None] * 9
    for c in range(3):
        W[c] = fma(-tz, Cf[3 + c], ty * Cf[6 + c])
        W[3 + c] = fma(tz, Cf[c], -(tx * Cf[6 + c]))
        W[6 + c] = fma(-ty, Cf[c], tx * Cf[3 + c])
    oB = [Bp[k] + W[k] for k in range(9)]
    Zm = [fma(0.5, W[k], Bp[k]) for k in range(9)]
    Y = []
    for r in range(3):
        Y += [fma(Zm[3 * r + 1], tz, -(Zm[3 * r + 2] * ty)), fma(-Zm[3 * r], tz, Zm[3 * r + 2] * tx),
              fma(Zm[3 * r], ty, -(Zm[3 * r + 1] * tx))]
    oA = [oA[0] - 2.0 * Y[0], oA[1] - (Y[1] + Y[3]), oA[2] - 2.0 * Y[4], oA[3] - (Y[2] + Y[6]),
          oA[4] - (Y[5] + Y[7]), oA[5] - 2.0 * Y[8]]
    return (oA, oB, oC)


def sym6_solve(s, rhs):
    A6, Bk, C = s
    Af = [A6[0], A6[1], A6[3], A6[1], A6[2], A6[4], A6[3], A6[4], A6[5]]
    Cf = [C[0], C[1], C[3], C[1], C[2], C[4], C[3], C[4], C[5]]
    A = [[None] * 6 for _ in range(6)]
    for r in range(3):
        for c in range(3):
            A[r][c], A[r][3 + c], A[3 + r][c], A[3 + r][3 + c] = Af[3 * r + c], Bk[3 * r + c], Bk[3 * c + r], Cf[3 * r + c]
    L = [[None] * 6 for _ in range(6)]
    inv = [None] * 6
    for j in range(6):
        d = A[j][j]
        for k in range(j):
            d = fma(-L[j][k], L[j][k], d)
        ljj = sqrt(d)
        inv[j] = 1.0 / ljj
        L[j][j] = ljj
        for i in range(j + 1, 6):
            x = A[i][j]
            for k in range(j):
                x = fma(-L[i][k], L[j][k], x)
            L[i][j] = x * inv[j]
    y = list(rhs[0]) + list(rhs[1])
    for i in range(6):
        for k in range(i):
            y[i] = fma(-L[i][k], y[k], y[i])
        y[i] = y[i] * inv[i]
    for i in range(5, -1, -1):
        for k in range(i + 1, 6):
            y[i] = fma(-L[k][i], y[k], y[i])
        y[i] = y[i] * inv[i]
    return (y[0:3], y[3:6])


def quat_R(x, y, z, w):
    s = rsqrt(fma(x, x, fma(y, y, fma(z, z, w * w))))
    x, y, z, w = x * s, y * s, z * s, w * s
    return [1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
            2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
            2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)]


def skew(a): return np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])


class Body:
    """The per-joint constants the kernels read (paper Sec. 3.2, Eq. 2-5),
    in FP64 from the body table."""

    def __init__(self, tree, i, qi, vi):
        self.parent, self.type, self.qi, self.vi = int(tree.parent[i]), int(tree.jtype[i]), qi, vi
        Rpre, tpre = tree.T_joint[i, :9].reshape(3, 3), tree.T_joint[i, 9:]
        Rpost, tpost = tree.T_link[i, :9].reshape(3, 3), tree.T_link[i, 9:]
        ax = np.asarray(tree.axis[i], dtype=np.float64)
        ax = ax / np.linalg.norm(ax) if self.type in (REVOLUTE, PRISMATIC) else ax
        K = skew(ax)
        self.R0 = list((Rpre if self.type == FREE else Rpre @ Rpost).ravel())
        self.t0 = list(tpre if self.type == FREE else Rpre @ tpost + tpre)
        self.A = list((Rpre @ K @ Rpost).ravel())
        self.Bm = list((Rpre @ K @ K @ Rpost).ravel())
        self.a = list(Rpre @ ax if self.type == PRISMATIC else Rpre @ K @ tpost)
        self.b = list(Rpre @ K @ K @ tpost)
        w_ = Rpost.T @ ax
        self.S = ([0.0] * 3, list(w_)) if self.type == PRISMATIC else (list(w_), list(np.cross(-Rpost.T @ tpost, w_)))
        m, c = float(tree.mass[i]), np.asarray(tree.com[i], dtype=np.float64)
        Ic = tree.I_com[i]
        cc = c @ c
        # the inertial parameters are run-time loads in every kernel variant
        Io = [Ic[0] + m * (cc - c[0] ** 2), Ic[1] - m * c[0] * c[1], Ic[2] + m * (cc - c[1] ** 2),
              Ic[3] - m * c[0] * c[2], Ic[4] - m * c[1] * c[2], Ic[5] + m * (cc - c[2] ** 2)]
        self.theta = (F(m), [F(x) for x in m * c], [F(x) for x in Io])
        self.nv = {FIXED: 0, REVOLUTE: 1, PRISMATIC: 1, FREE: 6}[self.type]


def bodies_of(tree):
    out, qi, vi = [], 0, 0
    for i in range(tree.n_bodies):
        b = Body(tree, i, qi, vi)
        qi += {FIXED: 0, REVOLUTE: 1, PRISMATIC: 1, FREE: 7}[b.type]
        vi += b.nv
        out.append(b)
    for i, b in enumerate(out):
        b.anc = {i} | (out[b.parent].anc if b.parent >= 0 else set())
    return out


def joint_X(b, q):
    if b.type == REVOLUTE:
        sh, ch = sincos(0.5 * q[b.qi])
        s, omc = 2.0 * sh * ch, 2.0 * sh * sh
        return ([fma(omc, b.Bm[k], fma(s, b.A[k], b.R0[k])) for k in range(9)],
                [fma(omc, b.b[k], fma(s, b.a[k], b.t0[k])) for k in range(3)])
    if b.type == PRISMATIC:
        return ([F(x) for x in b.R0], [fma(q[b.qi], b.a[k], b.t0[k]) for k in range(3)])
    if b.type == FREE:
        p, Rq = q[b.qi:b.qi + 3], quat_R(*q[b.qi + 3:b.qi + 7])
        R0, t0 = b.R0, b.t0
        return ([fma(R0[3 * r], Rq[c], fma(R0[3 * r + 1], Rq[3 + c], R0[3 * r + 2] * Rq[6 + c]))
                 for r in range(3) for c in range(3)],
                [fma(R0[3 * r], p[0], fma(R0[3 * r + 1], p[1], fma(R0[3 * r + 2], p[2], t0[r]))) for r in range(3)])
    return ([F(x) for x in b.R0], [F(x) for x in b.t0])


def S_times(b, x):
    if b.type in (REVOLUTE, PRISMATIC):
        return sscale(x[b.vi], b.S)
    if b.type == FREE:
        return (x[b.vi + 3:b.vi + 6], x[b.vi:b.vi + 3])
    return szero()


def ST(b, f):
    if b.type in (REVOLUTE, PRISMATIC):
        return [sdot(b.S, f)]
    if b.type == FREE:
        return list(f[1]) + list(f[0])
    return []


def world_poses(bs, q):
    Rw, pw = [], []
    for b in bs:
        R, t = joint_X(b, q)
        if b.parent < 0:
            Rw.append(R)
            pw.append(t)
        else:
            Rp, pp = Rw[b.parent], pw[b.parent]
            Rw.append([fma(Rp[3 * r], R[c], fma(Rp[3 * r + 1], R[3 + c], Rp[3 * r + 2] * R[6 + c]))
                       for r in range(3) for c in range(3)])
            pw.append([fma(Rp[3 * r], t[0], fma(Rp[3 * r + 1], t[1], fma(Rp[3 * r + 2], t[2], pp[r]))) for r in range(3)])
    return Rw, pw


def rnea(bs, a0, q, qd, qdd):
    X, v, a, f = [], [], [], []
    for i, b in enumerate(bs):
        X.append(joint_X(b, q))
        vJ, aJ = S_times(b, qd), S_times(b, qdd)
        if b.parent < 0:
            vi, ai = vJ, sadd(X_motion(X[i], a0), aJ)
        else:
            vi = sadd(X_motion(X[i], v[b.parent]), vJ)
            ai = sadd(sadd(X_motion(X[i], a[b.parent]), aJ), crm(vi, vJ))
        v.append(vi)
        a.append(ai)
        f.append(sadd(in_mul(b.theta, ai), crf(vi, in_mul(b.theta, vi))))
    tau = {}
    for i in range(len(bs) - 1, -1, -1):
        b = bs[i]
        for r, x in enumerate(ST(b, f[i])):
            tau[b.vi + r] = x
        if b.parent >= 0:
            f[b.parent] = sadd(f[b.parent], XT_force(X[i], f[i]))
    return [_v(tau[k]) for k in range(len(tau))]


def crba(bs, q, nv):
    X = [joint_X(b, q) for b in bs]
    Ic = [b.theta for b in bs]
    for i in range(len(bs) - 1, 0, -1):
        p = bs[i].parent
        if p >= 0:
            Ic[p] = in_add(Ic[p], in_to_parent(X[i], Ic[i]))
    M = np.zeros((nv, nv))
    for i, b in enumerate(bs):
        if b.nv == 1:
            Fv = in_mul(Ic[i], b.S)
            M[b.vi, b.vi] = _v(sdot(b.S, Fv))
            k = i
            for j in range(i - 1, -1, -1):
                if j not in b.anc:
                    continue
                Fv = XT_force(X[k], Fv)
                k = j
                bj = bs[j]
                if bj.nv == 1:
                    M[b.vi, bj.vi] = M[bj.vi, b.vi] = _v(sdot(bj.S, Fv))
                elif bj.nv == 6:
                    col = [_v(x) for x in Fv[1] + Fv[0]]
                    M[bj.vi:bj.vi + 6, b.vi] = M[b.vi, bj.vi:bj.vi + 6] = col
        elif b.nv == 6:
            m, h, Io = (_v(Ic[i][0]), [_v(x) for x in Ic[i][1]], [_v(x) for x in Ic[i][2]])
            M[b.vi:b.vi + 6, b.vi:b.vi + 6] = [
                [m, 0, 0, 0, h[2], -h[1]], [0, m, 0, -h[2], 0, h[0]], [0, 0, m, h[1], -h[0], 0],
                [0, -h[2], h[1], Io[0], Io[1], Io[3]], [h[2], 0, -h[0], Io[1], Io[2], Io[4]],
                [-h[1], h[0], 0, Io[3], Io[4], Io[5]]]
    return M


def aba(bs, a0, q, qd, tau):
    n = len(bs)
    X, va, cb, pA, IA = [None] * n, [None] * n, [None] * n, [None] * n, [None] * n
    U, invD, u = [None] * n, [None] * n, [None] * n
    for i, b in enumerate(bs):
        X[i] = joint_X(b, q)
        IA[i] = sym6_from_in(b.theta)
        vJ = S_times(b, qd)
        if b.parent < 0:
            vi, cb[i] = vJ, szero()
        else:
            vi = sadd(X_motion(X[i], va[b.parent]), vJ)
            cb[i] = crm(vi, vJ)
        va[i] = vi
        pA[i] = crf(vi, in_mul(b.theta, vi))
    for i in range(n - 1, -1, -1):
        b = bs[i]
        if b.type == FREE:
            continue
        Ia, pa = IA[i], pA[i]
        if b.type != FIXED:
            Ui = sym6_mul(IA[i], b.S)
            iD = 1.0 / sdot(b.S, Ui)
            ui = tau[b.vi] - sdot(b.S, pA[i])
            U[i], invD[i], u[i] = Ui, iD, ui
            if b.parent < 0:
                continue
            Ia = sym6_rank1_sub(Ia, Ui, iD)
            pa = sadd(sadd(pa, sym6_mul(Ia, cb[i])), sscale(ui * iD, Ui))
        else:
            if b.parent < 0:
                continue
            pa = sadd(pa, sym6_mul(Ia, cb[i]))
        IA[b.parent] = sym6_add(IA[b.parent], sym6_to_parent(X[i], Ia))
        pA[b.parent] = sadd(pA[b.parent], XT_force(X[i], pa))
    qdd = {}
    for i, b in enumerate(bs):
        ap = a0 if b.parent < 0 else va[b.parent]
        ai = sadd(X_motion(X[i], ap), cb[i])
        if b.type in (REVOLUTE, PRISMATIC):
            qi = (u[i] - sdot(U[i], ai)) * invD[i]
            qdd[b.vi] = qi
            ai = sadd(ai, sscale(qi, b.S))
        elif b.type == FREE:
            tf = (tau[b.vi + 3:b.vi + 6], tau[b.vi:b.vi + 3])
            anew = sym6_solve(IA[i], ssub(tf, pA[i]))
            x = ssub(anew, ai)
            for r, val in enumerate(list(x[1]) + list(x[0])):
                qdd[b.vi + r] = val
            ai = anew
        va[i] = ai
    return [_v(qdd[k]) for k in range(len(qdd))]


def _mixed_tree():
    """Revolute, prismatic and fixed joints with rotated joint and link
    frames."""
    t = w.random_tree([-1, 0, 1, 1, 3, 2], [REVOLUTE, PRISMATIC, REVOLUTE, FIXED, REVOLUTE, PRISMATIC], seed=7,
                      ee=(4, 5))
    rng = np.random.default_rng(3)
    for i in range(t.n_bodies):
        for T in (t.T_joint, t.T_link):
            qv = rng.standard_normal(4)
            qv /= np.linalg.norm(qv)
            x, y, z, s = qv
            T[i, :9] = [1 - 2 * (y * y + z * z), 2 * (x * y - s * z), 2 * (x * z + s * y),
                        2 * (x * y + s * z), 1 - 2 * (x * x + z * z), 2 * (y * z - s * x),
                        2 * (x * z - s * y), 2 * (y * z + s * x), 1 - 2 * (x * x + y * y)]
            T[i, 9:] = 0.2 * rng.standard_normal(3)
    return t


TREES = {"chain7": lambda: w.chain(7, seed=0), "quadruped11": lambda: w.spined_quadruped(seed=0),
         "humanoid29": lambda: w.humanoid(seed=0), "mixed": _mixed_tree}


def _counted(fn, *args):
    COUNT["flops"] = COUNT["sincos"] = 0
    out = fn(*args)
    return out, COUNT["flops"], COUNT["sincos"]


@pytest.mark.parametrize("name", list(TREES))
def test_flop_model_equals_a_count_of_the_kernels_arithmetic(name):
    tree = TREES[name]()
    bs = bodies_of(tree)
    s = w.random_state(tree, 2, seed=4)
    a0 = ([F(0.0)] * 3, [F(-g) for g in tree.gravity])
    links = list(tree.ee)
    for e in range(2):
        q, qd, qdd, tau = ([F(x) for x in s[k][e]] for k in ("q", "qd", "qdd", "tau"))
        one = {k: s[k][e:e + 1] for k in s}
        # FK
        (Rw, pw), n_fk, sc = _counted(world_poses, bs, q)
        T = rbd.fk(tree, one["q"])[0]
        assert np.abs(np.array([[_v(x) for x in R] for R in Rw]) - T[:, :3, :3].reshape(-1, 9)).max() < 1e-12
        assert np.abs(np.array([[_v(x) for x in p] for p in pw]) - T[:, :3, 3]).max() < 1e-12
        assert n_fk == costs.flops(tree, "fk") and sc == costs.sincos(tree, "fk")
        # Jacobians of the end-effector links (one world-pose pass per link
        # list: the kernel computes the poses once)
        COUNT["flops"] = 0
        Rw, pw = world_poses(bs, q)
        Js = [jacobian_columns(bs, Rw, pw, l, tree.nv) for l in links]
        assert COUNT["flops"] == costs.flops(tree, "jacobian", links=links)
        for l, J in zip(links, Js):
            assert np.abs(J - rbd.jacobian(tree, one["q"], l)[0]).max() < 1e-12
        # RNEA, CRBA, ABA
        t_, n_rnea, _ = _counted(rnea, bs, a0, q, qd, qdd)
        assert np.abs(np.array(t_) - rbd.rnea(tree, one["q"], one["qd"], one["qdd"])[0]).max() < 1e-10
        assert n_rnea == costs.flops(tree, "rnea")
        M, n_crba, _ = _counted(crba, bs, q, tree.nv)
        assert np.abs(M - rbd.crba(tree, one["q"])[0]).max() < 1e-12
        assert n_crba == costs.flops(tree, "crba")
        x, n_aba, _ = _counted(aba, bs, a0, q, qd, tau)
        ref = rbd.aba(tree, one["q"], one["qd"], one["tau"])[0]
        assert np.abs(np.array(x) - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())
        assert n_aba == costs.flops(tree, "aba")


def jacobian_columns(bs, Rw, pw, link, nv):
    """Jacobian columns of one link from world poses already computed."""
    J = np.zeros((6, nv))
    for k, b in enumerate(bs):
        if b.nv == 0 or k not in bs[link].anc:
            continue
        p = pw[k]
        if b.nv == 1:
            wk = Rmul(Rw[k], b.S[0])
            vk = add3(Rmul(Rw[k], b.S[1]), cross(p, wk))
            J[:, b.vi] = [_v(x) for x in vk + wk]
        else:
            for j in range(6):
                a = j % 3
                Re = [Rw[k][a], Rw[k][3 + a], Rw[k][6 + a]]
                col = Re + [0.0] * 3 if j < 3 else cross(p, Re) + Re
                J[:, b.vi + j] = [_v(x) for x in col]
    return J
