"""Run one operator of a workload tree at a fixed launch configuration, a
few times, for a profiler to capture its kernel, or time it:

    python -m paper_2605_31481_gb300.run_op <tree> <B> <op> <variant> <block> [calls] [--time]

tree: chain7 | quadruped11 | humanoid29; op: fk | jacobian | rnea | crba |
aba, or eval:<roles> for one fused launch of the roles joined by "+" among
kin (FK and the Jacobians), rnea, crba and aba; variant and block as
Model.set_launch takes them (for eval:..., the eval kind's). Inputs are the
seeded states of workloads.random_state(tree, B, seed=1). --time prints the
device time per call of a CUDA graph of 20 calls replayed (best of three
measurements, hot inputs).
"""
from __future__ import annotations

import sys

import numpy as np


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    timed = "--time" in argv
    argv = [a for a in argv if a != "--time"]
    if len(argv) < 5:
        raise SystemExit(__doc__)
    import torch

    from . import api, build, workloads as w
    build.build(quiet=True)
    name, B, op, variant, block = argv[0], int(argv[1]), argv[2], argv[3], int(argv[4])
    calls = int(argv[5]) if len(argv) > 5 else 4
    tree = {"chain7": lambda: w.chain(7, seed=0), "quadruped11": lambda: w.spined_quadruped(seed=0),
            "humanoid29": lambda: w.humanoid(seed=0)}[name]()
    kind = "eval" if op.startswith("eval:") else op
    m = api.Model(tree, specialize=[kind] if variant in ("specialized", "path", "pathwarp", "pinned") else None)
    m.set_launch([kind], block, variant)
    s = w.random_state(tree, B, seed=1)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x.T.astype(np.float32))).cuda()
    q, qd, qdd, tau = cu(s["q"]), cu(s["qd"]), cu(s["qdd"]), cu(s["tau"])
    links = list(tree.ee) or [tree.n_bodies - 1]
    if kind == "eval":
        roles = set(op[5:].split("+"))
        if not roles <= {"kin", "rnea", "crba", "aba"}:
            raise SystemExit(f"unknown roles in {op}")
        f = lambda: api.eval(m, q, qd, qdd, tau, fk="kin" in roles, links=links if "kin" in roles else None,
                             rnea="rnea" in roles, crba="crba" in roles, aba="aba" in roles)
    else:
        f = {"fk": lambda: api.fk(m, q), "jacobian": lambda: api.jacobian(m, q, links),
             "rnea": lambda: api.rnea(m, q, qd, qdd), "crba": lambda: api.crba(m, q),
             "aba": lambda: api.aba(m, q, qd, tau)}[op]
    for _ in range(calls):
        f()
    torch.cuda.synchronize()
    if timed:
        from .autotune import graph_time_us
        print(f"{name} B={B} {op} {variant}/{block}: {graph_time_us(f, n=20, reps=5):.2f} us per call")
    else:
        print(f"{name} B={B} {op} {variant}/{block}: {calls} calls")


if __name__ == "__main__":
    main()
