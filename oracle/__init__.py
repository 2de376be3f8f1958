"""FP64 CPU oracle for batched rigid-body dynamics.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check in
`__graft_entry__.smoke()`, and the CPU-baseline leg and the reference arm
(`--impl reference`) of `bench.py` may import this package. The product (the CUDA library and its Python binding) never
calls it, and it shares no code with the product.

What it computes, and where the definitions come from:

* `rbd.fk`        forward kinematics, world pose of every body as the plain
                  product of homogeneous transforms T_joint * J(q) * T_link
                  (paper Sec. 3.2, first equation; tier 3 of Sec. 3.1).
* `rbd.jacobian`  geometric Jacobian, world-frame twist at the world origin,
                  linear part first (paper Sec. 3.4, Eq. 6), built here as the
                  adjoint of each joint's motion subspace.
* `rbd.rnea`      recursive Newton-Euler inverse dynamics (paper Sec. 3.3,
                  Eq. 7 for the forward sweep; Featherstone 2008 Table 5.1).
* `rbd.crba`      composite-rigid-body mass matrix (paper Sec. 3.5;
                  Featherstone 2008 Table 6.2).
* `rbd.aba`       articulated-body forward dynamics, three passes (paper
                  Sec. 4.1; Featherstone 2008 Table 7.1).
* `derivs`        exact derivatives by the complex-step method and the
                  inertial-parameter regressor (the paper differentiates with
                  autograd, Sec. 3.5 and Sec. 4.3); the dense derivatives
                  d tau / d q, d tau / d qd, d qdd / d q, d qdd / d qd and
                  M^-1 along the configuration's tangent space; the
                  reference cotangents of the Jacobian and of CRBA.
* `lagrange`      an independent route to M(q), C(q, qd) qd and g(q) from the
                  Lagrangian of the bodies, used only to pin the recursions.

All arithmetic is float64 (or complex128 under the complex-step method).
Environments are a leading batch axis; there is no blocking, fusion or
reordering across bodies beyond the textbook recursions.
"""
from . import spatial, rbd, derivs, lagrange  # noqa: F401
