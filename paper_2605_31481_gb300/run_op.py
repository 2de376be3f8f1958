"""Run one operator of a workload tree at a fixed launch configuration, a
few times, for a profiler to capture its kernel:

    python -m paper_2605_31481_gb300.run_op <tree> <B> <op> <variant> <block> [calls]

tree: chain7 | quadruped11 | humanoid29; op: fk | jacobian | rnea | crba |
aba; variant and block as Model.set_launch takes them. Inputs are the seeded
states of workloads.random_state(tree, B, seed=1).
"""
from __future__ import annotations

import sys

import numpy as np


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) < 5:
        raise SystemExit(__doc__)
    import torch

    from . import api, build, workloads as w
    build.build(quiet=True)
    name, B, op, variant, block = argv[0], int(argv[1]), argv[2], argv[3], int(argv[4])
    calls = int(argv[5]) if len(argv) > 5 else 4
    tree = {"chain7": lambda: w.chain(7, seed=0), "quadruped11": lambda: w.spined_quadruped(seed=0),
            "humanoid29": lambda: w.humanoid(seed=0)}[name]()
    m = api.Model(tree, specialize=[op] if variant in ("specialized", "path", "pathwarp") else None)
    m.set_launch([op], block, variant)
    s = w.random_state(tree, B, seed=1)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x.T.astype(np.float32))).cuda()
    q, qd, qdd, tau = cu(s["q"]), cu(s["qd"]), cu(s["qdd"]), cu(s["tau"])
    links = list(tree.ee) or [tree.n_bodies - 1]
    f = {"fk": lambda: api.fk(m, q), "jacobian": lambda: api.jacobian(m, q, links),
         "rnea": lambda: api.rnea(m, q, qd, qdd), "crba": lambda: api.crba(m, q),
         "aba": lambda: api.aba(m, q, qd, tau)}[op]
    for _ in range(calls):
        f()
    torch.cuda.synchronize()
    print(f"{name} B={B} {op} {variant}/{block}: {calls} calls")


if __name__ == "__main__":
    main()
