"""Randomised trees (random topology, every joint type, floating roots,
forests, non-identity joint and link frames) through every operator and
every environment-to-thread mapping, against the FP64 oracle."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2605_31481_gb300 import workloads as w
from tests._helpers import TOL, env_err, from_soa, to_soa_cuda
from tests.test_gpu_parity import _assert_close, _oracle_all

pytestmark = pytest.mark.gpu

KINDS = ["fk", "jacobian", "rnea", "crba", "aba", "eval"]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


def random_tree(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 25))
    floating = seed % 3 == 0
    parent, jtype = [], []
    for i in range(n):
        if i == 0:
            parent.append(-1)
        elif rng.random() < 0.08 and not floating:
            parent.append(-1)                                    # another root: a forest
        else:
            parent.append(int(rng.integers(0 if not floating else 0, i)))
        if i == 0 and floating:
            jtype.append(w.FREE)
        else:
            jtype.append(int(rng.choice([w.REVOLUTE] * 6 + [w.PRISMATIC] * 2 + [w.FIXED])))
    t = w.random_tree(parent, jtype, seed=seed, name=f"random{seed}")
    for i in range(n):
        if jtype[i] == w.FREE:
            continue
        t.T_joint[i, :9] = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix().ravel()
        t.T_link[i, :9] = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix().ravel()
        t.T_link[i, 9:] = rng.uniform(-0.2, 0.2, 3)
    has_child = set(p for p in parent if p >= 0)
    t.ee = tuple(i for i in range(n) if i not in has_child)[:4]
    return t


@pytest.mark.parametrize("seed", range(6))
def test_random_tree_every_mapping_matches_oracle(torch_cuda, seed):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, _ffi, autotune
    tree = random_tree(seed)
    m = api.Model(tree, specialize=KINDS)
    B = 197
    s = w.random_state(tree, B, seed=seed)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ee = list(tree.ee)
    ref = _oracle_all(tree, s, ee)
    configs = [("generic", 64), ("specialized", 128), ("level", 128), ("path", 64), ("pathwarp", 0)]
    ran = []
    for variant, block in configs:
        try:
            m.set_launch(KINDS if variant in ("generic", "specialized") else None, block, variant)
        except _ffi.FstError:
            continue                       # no such kernel for this tree (too many leaves, too large)
        out = {"poses": api.fk(m, q), "J": api.jacobian(m, q, ee), "tau": api.rnea(m, q, qd, qdd),
               "M": api.crba(m, q), "qdd": api.aba(m, q, qd, tau)}
        ev = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
        torch.cuda.synchronize()
        _assert_close({k: from_soa(v) for k, v in out.items()}, ref, f"random{seed}/{variant}")
        _assert_close({k: from_soa(v) for k, v in ev.items()}, ref, f"random{seed}/{variant}/eval")
        ran.append(variant)
    # the lean level-parallel CRBA and ABA (fixed and prismatic joints, free roots)
    m.set_launch(["crba", "aba"], 128, "levellean")
    lean = {"M": api.crba(m, q), "qdd": api.aba(m, q, qd, tau)}
    torch.cuda.synchronize()
    for k in lean:
        err = env_err(from_soa(lean[k]), ref[k])
        assert np.all(np.isfinite(err)) and err.max() <= TOL[k], f"random{seed}/levellean/{k}: {err.max():.3e}"
    m.set_sm_roles(autotune.StepPlan.pin_roles([60, 30, 30, 32]))
    try:
        m.set_launch(["eval"], 256, "pinned")
        pinned = True
    except _ffi.FstError:
        pinned = False                     # two level-parallel ABA tiles of this tree do not fit
    if pinned:
        ev = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
        torch.cuda.synchronize()
        _assert_close({k: from_soa(v) for k, v in ev.items()}, ref, f"random{seed}/pinned/eval")
    assert {"generic", "specialized"} <= set(ran)
