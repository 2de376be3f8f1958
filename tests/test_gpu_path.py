"""Path-parallel kernels (FST_VARIANT_PATH: one lane per root-to-leaf path,
shuffles where paths merge) against the FP64 oracle on every tree, at several
block sizes and a ragged batch, and the fused evaluation against the
per-operator calls."""
import numpy as np
import pytest

from paper_2605_31481_gb300 import workloads as w
from tests._helpers import TOL, env_err, from_soa, to_soa_cuda
from tests.test_gpu_parity import TREES, _assert_close, _oracle_all

pytestmark = pytest.mark.gpu

PATH_KINDS = ["fk", "jacobian", "rnea", "crba", "aba", "eval"]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


@pytest.fixture(scope="module")
def models(torch_cuda):
    from paper_2605_31481_gb300 import api
    return {name: api.Model(make(), specialize=PATH_KINDS) for name, make in TREES.items()}


@pytest.mark.parametrize("name", list(TREES))
@pytest.mark.parametrize("variant,block", [("path", 32), ("path", 128), ("path", 256), ("pathwarp", 0)])
def test_path_parallel_matches_oracle(torch_cuda, models, name, variant, block):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    m = models[name]
    m.set_launch(None, block, variant)
    B = 333                                    # ragged against every block's environment count
    s = w.random_state(tree, B, seed=8)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ee = list(tree.ee) or [tree.n_bodies - 1]
    out = {"poses": api.fk(m, q), "J": api.jacobian(m, q, ee), "tau": api.rnea(m, q, qd, qdd), "M": api.crba(m, q),
           "qdd": api.aba(m, q, qd, tau)}
    ev = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    torch.cuda.synchronize()
    ref = _oracle_all(tree, s, ee)
    _assert_close({k: from_soa(v) for k, v in out.items()}, ref, f"{variant}/{name}/{block}")
    for k in out:
        assert torch.equal(ev[k], out[k]), k


@pytest.mark.parametrize("variant", ["path", "pathwarp"])
def test_path_parallel_theta_override_and_small_batches(torch_cuda, models, variant):
    torch = torch_cuda
    from oracle import rbd
    from paper_2605_31481_gb300 import api
    tree = TREES["humanoid29"]()
    m = models["humanoid29"]
    m.set_launch(None, 64, variant)
    rng = np.random.default_rng(3)
    th = rbd.Model(tree).theta() * (1 + rng.uniform(-0.2, 0.2, (tree.n_bodies, 10)))
    tht = torch.from_numpy(th.astype(np.float32)).cuda()
    for B in (1, 7):
        s = w.random_state(tree, B, seed=B)
        q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
        got = {"tau": api.rnea(m, q, qd, qdd, theta=tht), "M": api.crba(m, q, theta=tht),
               "qdd": api.aba(m, q, qd, tau, theta=tht)}
        torch.cuda.synchronize()
        ref = {"tau": rbd.rnea(tree, s["q"], s["qd"], s["qdd"], theta=th), "M": rbd.crba(tree, s["q"], theta=th),
               "qdd": rbd.aba(tree, s["q"], s["qd"], s["tau"], theta=th)}
        for k, v in got.items():
            assert env_err(from_soa(v), ref[k]).max() <= TOL[k], (B, k)


def test_path_variant_needs_the_kernels(torch_cuda):
    from paper_2605_31481_gb300 import api, _ffi
    m = api.Model(TREES["quadruped11"]())
    with pytest.raises(_ffi.FstError):
        m.set_launch(["aba"], 64, "path")                       # not specialised
    wide = api.Model(w.legged(9, seed=1), specialize=["aba"])   # 9 leaves: no path-parallel kernel
    for v in ("path", "pathwarp"):
        with pytest.raises(_ffi.FstError):
            wide.set_launch(["aba"], 64, v)
    wide.set_launch(["aba"], 64, "specialized")
