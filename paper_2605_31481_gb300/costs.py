"""Algorithmic cost model of the kernels: bytes moved and FP32 flops per
environment, for the roofline report.

Bytes are the operator's FP32 inputs and outputs only (the model constants
are read once per block from L2 and are amortised away). Flops count the
arithmetic of the formulation the kernels use, one FMA = 2 flops, add/mul/
div/sqrt = 1; sin/cos are counted separately as `sincos` (they run on the
special-function path, not the FMA pipe).

Per-primitive counts (f3 = 3-vector, SV = spatial 6-vector):
  dot3 5, cross 9, f3 add 3, R*x 15, SV dot 11,
  X*m (motion to child) 42, X^T f (force to parent) 42, crm/crf 30,
  I*m (10-parameter inertia) 42, rigid inertia to parent 140,
  6x6 symmetric times SV 66, rank-1 downdate 48, symmetric 6x6 to parent 333,
  6x6 Cholesky solve 169,
  revolute joint transform (paper Eq. 4-5) 53 + one sincos,
  prismatic 6, free joint 114 (unit quaternion to R: 51).
"""
from __future__ import annotations

FIXED, REVOLUTE, PRISMATIC, FREE = 0, 1, 2, 3

JX = {FIXED: 0, REVOLUTE: 53, PRISMATIC: 6, FREE: 114}
NV = {FIXED: 0, REVOLUTE: 1, PRISMATIC: 1, FREE: 6}


def _path(tree, i):
    out = []
    while i >= 0:
        out.append(i)
        i = int(tree.parent[i])
    return out


def io_bytes(tree, op, n_links=1):
    n, nv, nb = tree.nq, tree.nv, tree.n_bodies
    f = {
        "fk": n + 12 * nb,
        "jacobian": n + 6 * nv * n_links,
        "rnea": n + 3 * nv,
        "crba": n + nv * nv,
        "aba": n + 3 * nv,
    }[op]
    return 4 * f


def flops(tree, op, links=()):
    """FP32 flops per environment of one operator."""
    nb = tree.n_bodies
    jt = [int(t) for t in tree.jtype]
    par = [int(p) for p in tree.parent]
    total = 0
    if op in ("fk", "jacobian"):
        for i in range(nb):
            total += JX[jt[i]] + (0 if par[i] < 0 else 63)
        if op == "jacobian":
            for l in links:
                for k in _path(tree, l):
                    total += 42 if NV[jt[k]] == 1 else (27 if jt[k] == FREE else 0)
        return total
    if op == "rnea":
        for i in range(nb):
            dof = NV[jt[i]] > 0
            total += JX[jt[i]] + (12 if NV[jt[i]] == 1 else 0)   # S qd, S qdd (a free joint's is a copy)
            total += 42 + 6 if par[i] < 0 else 84 + 18 + 30
            total += 84 + 30 + 6
            total += (11 if NV[jt[i]] == 1 else 0) + (48 if par[i] >= 0 else 0)
        return total
    if op == "crba":
        for i in range(nb):
            total += JX[jt[i]] + (150 if par[i] >= 0 else 0)
            if NV[jt[i]] == 1:
                # F = I^c S and its projection, then one force transform per
                # ancestor, projected where the ancestor has a 1-DOF joint
                total += 53 + sum(42 + (11 if NV[jt[k]] == 1 else 0) for k in _path(tree, i)[1:])
        return total
    if op == "aba":
        for i in range(nb):
            root = par[i] < 0
            dof1 = NV[jt[i]] == 1
            # pass 1: velocity, bias acceleration, bias force
            total += JX[jt[i]] + (6 if dof1 else 0) + (0 if root else 42 + 6 + 30) + 72
            # pass 2: U, D, u, then the articulated inertia and bias force to the parent
            if dof1:
                total += 90 + (0 if root else 48 + 85 + 333 + 21 + 48)
            elif jt[i] == FIXED and not root:
                total += 66 + 6 + 333 + 21 + 48
            # pass 3: the acceleration, then qdd (1-DOF) or the 6x6 solve (free root)
            total += 48
            if dof1:
                total += 25
            elif jt[i] == FREE:
                total += 169 + 12
        return total
    raise ValueError(op)


def sincos(tree, op, links=()):
    return sum(1 for t in tree.jtype if int(t) == REVOLUTE)
