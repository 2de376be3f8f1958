"""Kernels specialised at run time for one tree (fst_model_specialize)
against the FP64 oracle, at the same tolerances as the generic kernels, and
against the generic kernels themselves."""
import numpy as np
import pytest

from oracle import rbd, derivs
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import TOL, env_err, from_soa, oracle_poses, to_soa_cuda
from tests.test_gpu_parity import TREES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8"])
def test_specialized_forward_ops_match_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, _ffi
    tree = TREES[name]()
    B = 1000
    s = w.random_state(tree, B, seed=11)
    m = api.Model(tree, specialize=True)
    assert set(m.specialized()) == set(_ffi.SPEC_KINDS)
    g = api.Model(tree)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ee = list(tree.ee)
    out = {"poses": api.fk(m, q), "J": api.jacobian(m, q, ee), "tau": api.rnea(m, q, qd, qdd), "M": api.crba(m, q),
           "qdd": api.aba(m, q, qd, tau)}
    ev = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    gen = api.eval(g, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    torch.cuda.synchronize()
    ref = {"poses": oracle_poses(tree, s["q"]), "J": np.stack([rbd.jacobian(tree, s["q"], e) for e in ee], 1),
           "tau": rbd.rnea(tree, s["q"], s["qd"], s["qdd"]), "M": rbd.crba(tree, s["q"]),
           "qdd": rbd.aba(tree, s["q"], s["qd"], s["tau"])}
    for k, tol in TOL.items():
        assert env_err(from_soa(out[k]), ref[k]).max() <= tol, k
        assert torch.equal(ev[k], out[k]), k                   # fused and per-op specialised agree bitwise
        assert env_err(from_soa(gen[k]), from_soa(out[k])).max() <= tol, k


@pytest.mark.parametrize("name", ["chain7", "humanoid29", "general8"])
def test_specialized_adjoints_match_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 129
    s = w.random_state(tree, B, seed=12)
    rng = np.random.default_rng(5)
    tb = rng.standard_normal((B, tree.nv))
    m = api.Model(tree, specialize=True)
    q, qd, qdd, tau, tbar = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], s["tau"], tb))
    r = api.rnea_vjp(m, q, qd, qdd, tbar)
    rq, rqd, rqdd, rth = derivs.rnea_vjp(tree, s["q"], s["qd"], s["qdd"], tb)
    for k, ref in (("q", rq), ("qd", rqd), ("qdd", rqdd)):
        assert env_err(from_soa(r[k]), ref).max() <= 2e-4, k
    th = r["theta"].cpu().numpy()
    assert np.abs(th - rth).max() / np.abs(rth).max() <= 2e-4
    qdd_f = api.aba(m, q, qd, tau)
    a = api.aba_vjp(m, q, qd, qdd_f, tbar)
    aq, aqd, atau, ath = derivs.aba_vjp(tree, s["q"], s["qd"], s["tau"], tb)
    for k, ref in (("q", aq), ("qd", aqd), ("tau", atau)):
        assert env_err(from_soa(a[k]), ref).max() <= 2e-3, k
    pb = rng.standard_normal((B, tree.n_bodies, 12))
    pbt = torch.from_numpy(np.ascontiguousarray(np.moveaxis(pb, 0, -1).astype(np.float32))).cuda()
    assert env_err(from_soa(api.fk_vjp(m, q, pbt)), derivs.fk_vjp(tree, s["q"], pb)).max() <= 2e-4
    L, thb, qb, _ = api.rnea_loss_grad(m, q, qd, qdd, tau, q_bar=True)
    res = rbd.rnea(tree, s["q"], s["qd"], s["qdd"]) - s["tau"]
    assert abs(float(L) - np.sum(res * res)) / np.sum(res * res) < 1e-4
    lq, _, _, lth = derivs.rnea_vjp(tree, s["q"], s["qd"], s["qdd"], 2 * res)
    assert env_err(from_soa(qb), lq).max() <= 2e-4
    assert np.abs(thb.cpu().numpy() - lth).max() / np.abs(lth).max() <= 2e-4


def test_specialized_theta_override(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES["quadruped11"]()
    s = w.random_state(tree, 300, seed=13)
    th = rbd.Model(tree).theta() * (1 + np.random.default_rng(9).uniform(-0.2, 0.2, (tree.n_bodies, 10)))
    m = api.Model(tree, specialize=["rnea", "crba"])
    assert set(m.specialized()) == {"rnea", "crba"}
    q, qd, qdd = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd"))
    tht = torch.from_numpy(th.astype(np.float32)).cuda()
    assert env_err(from_soa(api.rnea(m, q, qd, qdd, theta=tht)),
                   rbd.rnea(tree, s["q"], s["qd"], s["qdd"], theta=th)).max() <= TOL["tau"]
    assert env_err(from_soa(api.crba(m, q, theta=tht)), rbd.crba(tree, s["q"], theta=th)).max() <= TOL["M"]


@pytest.mark.parametrize("name", ["quadruped11", "humanoid29", "general8"])
@pytest.mark.parametrize("level_kinds", [("aba",), ("aba", "crba", "rnea", "jacobian"), ("crba",), ("jacobian",),
                                         ("crba", "jacobian"), ("aba:levellean",), ("aba:levellean", "crba:levellean"),
                                         ("aba:level2", "rnea:level2")])
def test_specialized_eval_with_level_parallel_roles(torch_cuda, name, level_kinds):
    """The specialised fused kernel runs roles whose operator is tuned
    level-parallel that way (32 environments per block, warps splitting
    levels) and the others one environment per thread, in one launch. The
    cases without ABA have a CRBA or Jacobian role set the launch's shared
    memory: its state sits after the nq + 2 nv staged rows of the kernel's
    layout, which the launch must allocate even though the role stages only
    q. Any level-parallel setting of an operator (level, level2,
    levellean) makes its role level-parallel in the fused kernel."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 1000
    s = w.random_state(tree, B, seed=14)
    m = api.Model(tree, specialize=["eval_mixed"])
    for kv in level_kinds:
        kind, _, variant = kv.partition(":")
        m.set_launch([kind], 128, variant or "level")
    m.set_launch(["eval"], 64, "mixed")
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ee = list(tree.ee)
    ev = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    torch.cuda.synchronize()
    ref = {"poses": oracle_poses(tree, s["q"]), "J": np.stack([rbd.jacobian(tree, s["q"], e) for e in ee], 1),
           "tau": rbd.rnea(tree, s["q"], s["qd"], s["qdd"]), "M": rbd.crba(tree, s["q"]),
           "qdd": rbd.aba(tree, s["q"], s["qd"], s["tau"])}
    for k, tol in TOL.items():
        assert env_err(from_soa(ev[k]), ref[k]).max() <= tol, k
