"""CUDA path (through the C ABI) against the FP64 oracle, element by
element, on seeded inputs: several tiles plus a ragged tail, the full
workload sizes on sampled environments, and the edge cases (B = 0, B = 1,
inertia override, NaN isolation, every joint type)."""
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import rbd
from paper_2605_31481_gb300 import urdf, workloads as w
from tests._helpers import TOL, env_err, from_soa, oracle_poses, to_soa_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


def _general_tree(seed=5):
    """Every joint type, non-identity joint and link frames."""
    t = w.random_tree([-1, 0, 1, 1, 3, 4, 0, 6], [w.REVOLUTE, w.PRISMATIC, w.REVOLUTE, w.FIXED, w.REVOLUTE,
                                                  w.PRISMATIC, w.REVOLUTE, w.REVOLUTE], seed)
    rng = np.random.default_rng(seed)
    for i in range(t.n_bodies):
        t.T_joint[i, :9] = Rotation.random(random_state=rng.integers(1 << 30)).as_matrix().ravel()
        t.T_link[i, :9] = Rotation.random(random_state=rng.integers(1 << 30)).as_matrix().ravel()
        t.T_link[i, 9:] = rng.uniform(-0.2, 0.2, 3)
    t.ee = (5, 7, 2)
    return t


TREES = {
    "chain7": lambda: w.chain(7, seed=0),
    "quadruped11": lambda: w.spined_quadruped(seed=0),
    "humanoid29": lambda: w.humanoid(seed=0),
    "general8": _general_tree,
    "legged18": lambda: w.legged(6, seed=3),
    "urdf_arm6_tool": lambda: urdf.load_urdf(os.path.join(os.path.dirname(__file__), "data", "arm6_tool.urdf")),
}


def _run_all(torch, api, tree, s, theta=None):
    m = api.Model(tree)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    th = None if theta is None else torch.from_numpy(theta.astype(np.float32)).cuda()
    ee = list(tree.ee) if tree.ee else [tree.n_bodies - 1]
    out = {
        "poses": from_soa(api.fk(m, q)),
        "J": from_soa(api.jacobian(m, q, ee)),
        "tau": from_soa(api.rnea(m, q, qd, qdd, theta=th)),
        "M": from_soa(api.crba(m, q, theta=th)),
        "qdd": from_soa(api.aba(m, q, qd, tau, theta=th)),
    }
    torch.cuda.synchronize()
    return out, ee


def _oracle_all(tree, s, ee, theta=None, idx=None):
    sl = (lambda x: x) if idx is None else (lambda x: x[idx])
    q, qd, qdd, tau = (sl(s[k]) for k in ("q", "qd", "qdd", "tau"))
    return {
        "poses": oracle_poses(tree, q),
        "J": np.stack([rbd.jacobian(tree, q, e) for e in ee], axis=1),
        "tau": rbd.rnea(tree, q, qd, qdd, theta=theta),
        "M": rbd.crba(tree, q, theta=theta),
        "qdd": rbd.aba(tree, q, qd, tau, theta=theta),
    }


def _assert_close(gpu, ref, label):
    for k, tol in TOL.items():
        err = env_err(gpu[k], ref[k])
        assert np.all(np.isfinite(err)), f"{label}/{k}: non-finite output"
        assert err.max() <= tol, f"{label}/{k}: max err {err.max():.3e} (p99.9 {np.quantile(err, 0.999):.3e}) > {tol}"


@pytest.mark.parametrize("name", list(TREES))
def test_all_ops_match_oracle_ragged_batch(torch_cuda, name):
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 1000                                   # 31 full 32-env tiles plus a tail of 8
    s = w.random_state(tree, B, seed=1)
    gpu, ee = _run_all(torch_cuda, api, tree, s)
    _assert_close(gpu, _oracle_all(tree, s, ee), name)


@pytest.mark.parametrize("name,B", [("quadruped11", 4096), ("chain7", 8192), ("humanoid29", 65536)])
def test_full_size_sampled(torch_cuda, name, B):
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    s = w.random_state(tree, B, seed=1)
    gpu, ee = _run_all(torch_cuda, api, tree, s)
    idx = np.unique(np.r_[np.random.default_rng(0).choice(B, 512, replace=False), 0, B - 1])
    ref = _oracle_all(tree, s, ee, idx=idx)
    _assert_close({k: v[idx] for k, v in gpu.items()}, ref, f"{name}@{B}")


def test_theta_override(torch_cuda):
    from paper_2605_31481_gb300 import api
    tree = w.spined_quadruped(seed=2)
    s = w.random_state(tree, 333, seed=4)
    rng = np.random.default_rng(7)
    th = rbd.Model(tree).theta() * (1 + rng.uniform(-0.3, 0.3, (tree.n_bodies, 10)))
    gpu, ee = _run_all(torch_cuda, api, tree, s, theta=th)
    ref = _oracle_all(tree, s, ee, theta=th)
    for k in ("tau", "M"):
        assert env_err(gpu[k], ref[k]).max() <= TOL[k]
    # the perturbed parameters need not be physical, so ABA may be badly
    # conditioned here; check it against the oracle where M stays well-posed
    good = np.linalg.cond(rbd.crba(tree, s["q"], theta=th)) < 1e4
    assert good.sum() > 100
    assert env_err(gpu["qdd"][good], ref["qdd"][good]).max() <= TOL["qdd"]


def test_batch_of_one_and_zero(torch_cuda):
    import torch
    from paper_2605_31481_gb300 import api
    tree = w.humanoid(seed=1)
    s = w.random_state(tree, 1, seed=9)
    gpu, ee = _run_all(torch_cuda, api, tree, s)
    _assert_close(gpu, _oracle_all(tree, s, ee), "B=1")
    m = api.Model(tree)
    z = torch.empty((tree.nq, 0), device="cuda")
    assert api.fk(m, z).shape == (tree.n_bodies, 12, 0)
    assert api.rnea(m, z, torch.empty((tree.nv, 0), device="cuda"), torch.empty((tree.nv, 0), device="cuda")).numel() == 0


def test_nan_stays_in_its_environment(torch_cuda):
    from paper_2605_31481_gb300 import api
    tree = w.chain(7, seed=0)
    s = w.random_state(tree, 64, seed=3)
    s["q"][10, 3] = np.nan
    gpu, ee = _run_all(torch_cuda, api, tree, s)
    for k in ("poses", "tau", "M", "qdd"):
        bad = ~np.isfinite(gpu[k].reshape(64, -1)).all(axis=1)
        assert bad[10] and bad.sum() == 1, k


def test_invalid_calls_return_errors(torch_cuda):
    import torch
    from paper_2605_31481_gb300 import api, _ffi
    tree = w.chain(7, seed=0)
    m = api.Model(tree)
    q = torch.zeros((7, 16), device="cuda")
    with pytest.raises(_ffi.FstError):
        api.jacobian(m, q, [99])
    with pytest.raises(ValueError):
        api.fk(m, torch.zeros((6, 16), device="cuda"))
    L = _ffi.lib()
    assert L.fst_fk(m.handle, 16, None, None, None) == -1
    assert L.fst_fk(m.handle, -1, None, None, None) == -1


@pytest.mark.parametrize("name", ["quadruped11", "humanoid29", "general8"])
def test_fused_eval_is_bitwise_equal_to_per_op_calls(torch_cuda, name):
    import torch
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 777
    s = w.random_state(tree, B, seed=2)
    m = api.Model(tree)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ee = list(tree.ee)
    res = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    ref = {"poses": api.fk(m, q), "J": api.jacobian(m, q, ee), "tau": api.rnea(m, q, qd, qdd),
           "M": api.crba(m, q), "qdd": api.aba(m, q, qd, tau)}
    for k in ref:
        assert torch.equal(res[k], ref[k]), k
    # subsets: only the requested outputs are produced
    only = api.eval(m, q, qd, qdd, tau, rnea=True)
    assert set(only) == {"tau"} and torch.equal(only["tau"], ref["tau"])
    kin = api.eval(m, q, links=ee)
    assert set(kin) == {"J"} and torch.equal(kin["J"], ref["J"])


@pytest.mark.parametrize("name", list(TREES))
@pytest.mark.parametrize("variant,block", [("level", 32), ("level", 64), ("level", 256), ("level2", 64),
                                           ("level2", 256)])
def test_level_parallel_variant_matches_oracle(torch_cuda, name, variant, block):
    """Level-parallel kernels (warps split each tree level) on every tree:
    one tile of 32 environments per block with 1, 2 and 8 warps, and two
    tiles per block with 1 and 4 warps each (a 333-environment batch leaves
    the last block's second tile partly and wholly past B)."""
    import torch
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 333
    s = w.random_state(tree, B, seed=6)
    m = api.Model(tree)
    m.set_launch(["fk", "jacobian", "rnea", "crba", "aba", "eval"], block, variant)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ee = list(tree.ee)
    out = {"poses": api.fk(m, q), "J": api.jacobian(m, q, ee), "tau": api.rnea(m, q, qd, qdd), "M": api.crba(m, q),
           "qdd": api.aba(m, q, qd, tau)}
    ev = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    torch.cuda.synchronize()
    ref = _oracle_all(tree, s, ee)
    _assert_close({k: from_soa(v) for k, v in out.items()}, ref, f"{variant}/{name}/{block}")
    if variant == "level":
        for k in out:
            assert torch.equal(ev[k], out[k]), k
    else:
        # two ABA-sized tiles need not fit where one operator's tiles do: the
        # fused launch may then run another kernel than the per-operator one
        _assert_close({k: from_soa(v) for k, v in ev.items()}, ref, f"{variant}/{name}/{block}/eval")


@pytest.mark.parametrize("name", list(TREES))
@pytest.mark.parametrize("block", [32, 128, 256])
def test_lean_level_crba_aba_match_oracle(torch_cuda, name, block):
    """The lean level-parallel CRBA (X and I^c S per body, q from global
    memory) and ABA (14 floats per body, transforms recomputed), both with
    contributions in a two-level ring, on every tree, 1, 4 and 8 warps per
    tile, a ragged 333-environment batch: the oracle's M and accelerations,
    and those of the standard level-parallel kernels within rounding."""
    import torch
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 333
    s = w.random_state(tree, B, seed=16)
    m = api.Model(tree)
    q, qd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "tau"))
    M_out = torch.full((tree.nv, tree.nv, B), float("nan"), device="cuda")  # every entry must be written
    m.set_launch(["crba", "aba"], block, "levellean")
    lean = {"M": api.crba(m, q, out=M_out), "qdd": api.aba(m, q, qd, tau)}
    m.set_launch(["crba", "aba"], block, "level")
    std = {"M": api.crba(m, q), "qdd": api.aba(m, q, qd, tau)}
    torch.cuda.synchronize()
    ref = {"M": rbd.crba(tree, s["q"]), "qdd": rbd.aba(tree, s["q"], s["qd"], s["tau"])}
    for k in ref:
        err = env_err(from_soa(lean[k]), ref[k])
        assert np.all(np.isfinite(err)) and err.max() <= TOL[k], f"levellean/{name}/{block}/{k}: {err.max():.3e}"
        scale = 1.0 + std[k].abs().max().item()
        assert (lean[k] - std[k]).abs().max().item() <= 1e-4 * scale, (name, k)


def test_lean_level_aba_full_size_sampled(torch_cuda):
    """humanoid29 at B = 65536 with the lean kernels at the block the tuner
    tries (256): sampled environments against the oracle, and the NaN of one
    environment's input stays in that environment."""
    import torch
    from paper_2605_31481_gb300 import api
    tree = TREES["humanoid29"]()
    B = 65536
    s = w.random_state(tree, B, seed=17)
    m = api.Model(tree)
    m.set_launch(["crba", "aba"], 256, "levellean")
    q, qd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "tau"))
    q[7, 777] = float("nan")                  # the waist joint (q of the free base do not enter M)
    out = {"qdd": from_soa(api.aba(m, q, qd, tau)), "M": from_soa(api.crba(m, q))}
    idx = np.r_[np.arange(0, B, 997), B - 1]
    idx = idx[idx != 777]
    ref = {"qdd": rbd.aba(tree, s["q"][idx], s["qd"][idx], s["tau"][idx]), "M": rbd.crba(tree, s["q"][idx])}
    for k in ref:
        err = env_err(out[k][idx], ref[k])
        assert np.all(np.isfinite(err)) and err.max() <= TOL[k], f"levellean/humanoid29/65536/{k}: {err.max():.3e}"
        assert np.isnan(out[k][777]).any()
        assert np.isfinite(out[k][np.r_[776, 778]]).all()


def test_lean_variant_is_for_crba_and_aba_only(torch_cuda):
    from paper_2605_31481_gb300 import api, _ffi
    m = api.Model(TREES["quadruped11"]())
    for kind in ("fk", "jacobian", "rnea", "eval"):
        with pytest.raises(_ffi.FstError):
            m.set_launch([kind], 128, "levellean")
    m.set_launch(None, 128, "levellean")        # "all kinds" means CRBA and ABA


def test_carveout_change_keeps_shared_memory_limit(torch_cuda):
    """A change of the shared-memory carveout re-prepares each kernel; a
    smaller model prepared after it must not shrink the dynamic shared-memory
    limit that a larger model's launch of the same kernel needs."""
    import torch
    from paper_2605_31481_gb300 import api
    big, small = TREES["humanoid29"](), TREES["quadruped11"]()
    models = {}
    for name, tree in (("big", big), ("small", small)):
        m = api.Model(tree)
        m.set_launch(None, 32, "level")
        s = w.random_state(tree, 64, seed=3)
        models[name] = (m, [to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau")], list(tree.ee))
    try:
        for carveout, order in ((100, ("big",)), (-1, ("small", "big")), (50, ("small", "big", "small"))):
            api.set_smem_carveout(carveout)
            for name in order:
                m, (q, qd, qdd, tau), ee = models[name]
                api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
                api.aba(m, q, qd, tau)
        torch.cuda.synchronize()
    finally:
        api.set_smem_carveout(-1)
