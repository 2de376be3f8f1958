"""The autotuner: every candidate launch configuration gives oracle-correct
results, the chosen one is applied and cached, and the multi-operator step
plan reproduces the per-operator calls."""
import json

import numpy as np
import pytest

from oracle import rbd
from paper_2605_31481_gb300 import workloads as w
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


def test_every_launch_configuration_is_correct(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = w.spined_quadruped(seed=3)
    B = 300
    s = w.random_state(tree, B, seed=4)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ref = {"poses": oracle_poses(tree, s["q"]), "J": np.stack([rbd.jacobian(tree, s["q"], e) for e in tree.ee], 1),
           "tau": rbd.rnea(tree, s["q"], s["qd"], s["qdd"]), "M": rbd.crba(tree, s["q"]),
           "qdd": rbd.aba(tree, s["q"], s["qd"], s["tau"])}
    m = api.Model(tree, specialize=True)
    for variant in ("generic", "specialized", "level"):
        for block in (32, 64, 128, 256):
            m.set_launch(None, block, variant)
            out = api.eval(m, q, qd, qdd, tau, fk=True, links=tree.ee, rnea=True, crba=True, aba=True)
            per = {"poses": api.fk(m, q), "J": api.jacobian(m, q, tree.ee), "tau": api.rnea(m, q, qd, qdd),
                   "M": api.crba(m, q), "qdd": api.aba(m, q, qd, tau)}
            for k, tol in TOL.items():
                assert env_err(from_soa(out[k]), ref[k]).max() <= tol, (variant, block, k)
                assert torch.equal(out[k], per[k]), (variant, block, k)


def test_tune_sets_and_caches(torch_cuda, tmp_path, monkeypatch):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autotune
    monkeypatch.setenv("FST_TUNE_CACHE", str(tmp_path / "tune.json"))
    tree = w.chain(7, seed=0)
    m = api.Model(tree, specialize=["rnea", "aba"])
    res = autotune.tune(m, 2048, kinds=("rnea", "aba", "crba"))
    # not specialised: no specialised candidates
    assert res["crba"]["variant"] in ("generic", "level", "level2", "levellean")
    # generic x4, level x4, level2 x3 (block >= 64), for CRBA also levellean x2 (blocks 128, 256), and for
    # the specialised RNEA also specialised x4, path x4 and pathwarp
    assert len(res["rnea"]["candidates"]) == 20 and len(res["crba"]["candidates"]) == 13
    assert not any(k.startswith("mixed") for k in res["rnea"]["candidates"])
    data = json.load(open(tmp_path / "tune.json"))
    assert len(data) == 3
    again = autotune.tune(m, 2048, kinds=("rnea", "aba", "crba"))     # served from the cache
    assert {k: (v["variant"], v["block"]) for k, v in again.items()} == \
           {k: (v["variant"], v["block"]) for k, v in res.items()}


def test_step_plan_matches_per_operator_calls(torch_cuda, tmp_path, monkeypatch):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autotune
    monkeypatch.setenv("FST_TUNE_CACHE", str(tmp_path / "tune.json"))
    tree = w.spined_quadruped(seed=0)
    B = 1024
    s = w.random_state(tree, B, seed=5)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    m = api.Model(tree, specialize=True)
    plan = autotune.StepPlan(m, B)
    out = {"poses": torch.empty(tree.n_bodies, 12, B, device="cuda"),
           "J": torch.empty(4, 6, tree.nv, B, device="cuda"), "tau": torch.empty(tree.nv, B, device="cuda"),
           "M": torch.empty(tree.nv, tree.nv, B, device="cuda"), "qdd": torch.empty(tree.nv, B, device="cuda")}
    for mode in plan.MODES:
        plan.mode = mode
        for v in out.values():
            v.zero_()
        plan(q, qd, qdd, tau, out)
        torch.cuda.synchronize()
        ref = {"poses": api.fk(m, q), "J": api.jacobian(m, q, tree.ee), "tau": api.rnea(m, q, qd, qdd),
               "M": api.crba(m, q), "qdd": api.aba(m, q, qd, tau)}
        for k, tol in TOL.items():
            assert env_err(from_soa(out[k]), from_soa(ref[k])).max() <= tol, (mode, k)
    assert set(plan.MODES) <= {k.split("[")[0].split("@")[0].split("+")[0] for k in plan.describe()["us"]}
    from paper_2605_31481_gb300 import api as _api
    _api.set_smem_carveout(-1)
    ref = {"poses": api.fk(m, q), "J": api.jacobian(m, q, tree.ee), "tau": api.rnea(m, q, qd, qdd),
           "M": api.crba(m, q), "qdd": api.aba(m, q, qd, tau)}
    for k, tol in TOL.items():
        assert env_err(from_soa(out[k]), from_soa(ref[k])).max() <= tol, k


def test_bench_step_at_full_size_matches_oracle(torch_cuda, tmp_path, monkeypatch):
    """The timed step exactly as bench.py runs it (the 11-DOF tree, B = 4096,
    specialised model, tuned step plan, replayed from a CUDA graph) against
    the oracle on sampled environments, element by element."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autotune
    monkeypatch.setenv("FST_TUNE_CACHE", str(tmp_path / "tune.json"))
    tree = w.spined_quadruped(seed=0)
    B = 4096
    s = w.random_state(tree, B, seed=1)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    m = api.Model(tree, specialize=True)
    plan = autotune.StepPlan(m, B, links=list(tree.ee))
    out = {"poses": torch.empty(tree.n_bodies, 12, B, device="cuda"),
           "J": torch.empty(4, 6, tree.nv, B, device="cuda"), "tau": torch.empty(tree.nv, B, device="cuda"),
           "M": torch.empty(tree.nv, tree.nv, B, device="cuda"), "qdd": torch.empty(tree.nv, B, device="cuda")}
    g = torch.cuda.CUDAGraph()
    plan(q, qd, qdd, tau, out)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        plan(q, qd, qdd, tau, out)
    for v in out.values():
        v.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    idx = np.unique(np.r_[np.random.default_rng(2).choice(B, 256, replace=False), 0, 31, 32, B - 1])
    ref = {"poses": oracle_poses(tree, s["q"][idx]),
           "J": np.stack([rbd.jacobian(tree, s["q"][idx], e) for e in tree.ee], 1),
           "tau": rbd.rnea(tree, s["q"][idx], s["qd"][idx], s["qdd"][idx]), "M": rbd.crba(tree, s["q"][idx]),
           "qdd": rbd.aba(tree, s["q"][idx], s["qd"][idx], s["tau"][idx])}
    for k, tol in TOL.items():
        err = env_err(from_soa(out[k])[idx], ref[k])
        assert np.all(np.isfinite(err)) and err.max() <= tol, (plan.describe()["mode"], k, err.max())
