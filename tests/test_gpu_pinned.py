"""SM-pinned launches (FST_VARIANT_PINNED): the pinned fused step (all five
operators in one launch of one block per SM, ABA level-parallel inside it)
and the pinned ABA give the oracle's results whatever the SM role table,
including tables that give some role no SM at all (the last block then does
that role's work), and the pinned step replayed from a CUDA graph equals the
plain calls."""
import numpy as np
import pytest

from paper_2605_31481_gb300 import workloads as w
from tests._helpers import from_soa, to_soa_cuda
from tests.test_gpu_parity import TREES, _assert_close, _oracle_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


TABLES = {
    "interleaved": lambda: __import__("paper_2605_31481_gb300.autotune",
                                      fromlist=["StepPlan"]).StepPlan.pin_roles([64, 32, 24, 32]),
    "few_sms": lambda: __import__("paper_2605_31481_gb300.autotune",
                                  fromlist=["StepPlan"]).StepPlan.pin_roles([3, 2, 1, 2]),
    "no_roles": lambda: ["none"] * 256,
    "aba_only": lambda: ["aba"] * 256,
    "kin_only": lambda: ["kin"] * 256,
}


@pytest.mark.parametrize("name", ["quadruped11", "humanoid29", "general8"])
@pytest.mark.parametrize("table", list(TABLES))
def test_pinned_matches_oracle(torch_cuda, name, table):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    from paper_2605_31481_gb300 import _ffi
    tree = TREES[name]()
    m = api.Model(tree, specialize=["eval"])
    m.set_sm_roles(TABLES[table]())
    if name == "humanoid29":
        # two level-parallel ABA tiles of the 24-body tree exceed shared memory
        with pytest.raises(_ffi.FstError):
            m.set_launch(["eval"], 256, "pinned")
    else:
        m.set_launch(["eval"], 256, "pinned")
    m.set_launch(["aba"], 256, "pinned")
    B = 1000 + 13
    s = w.random_state(tree, B, seed=17)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ee = list(tree.ee)
    ev = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    qdd_pin = api.aba(m, q, qd, tau)
    torch.cuda.synchronize()
    ref = _oracle_all(tree, s, ee)
    _assert_close({k: from_soa(v) for k, v in ev.items()}, ref, f"pinned/{name}/{table}")
    m.set_launch(["aba"], 256, "level")
    assert torch.equal(qdd_pin, api.aba(m, q, qd, tau))     # same level-parallel bodies


def test_pinned_step_in_a_graph(torch_cuda):
    """The step plan's pinned mode: the five operators in one SM-pinned
    launch, replayed from a CUDA graph, equal to the plain per-operator
    calls."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autotune
    tree = TREES["quadruped11"]()
    B = 4096
    m = api.Model(tree, specialize=True)
    plan = autotune.StepPlan(m, B, use_cache=False, modes=("fused",))
    plan._set_eval("pinned/256|level/256@64-32-24-32")
    plan.mode = "pinned"
    s = w.random_state(tree, B, seed=5)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    out = {"poses": torch.empty(tree.n_bodies, 12, B, device="cuda"),
           "J": torch.empty(4, 6, tree.nv, B, device="cuda"), "tau": torch.empty(tree.nv, B, device="cuda"),
           "M": torch.empty(tree.nv, tree.nv, B, device="cuda"), "qdd": torch.empty(tree.nv, B, device="cuda")}
    plan(q, qd, qdd, tau, out)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan(q, qd, qdd, tau, out)
    for v in out.values():
        v.fill_(float("nan"))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    m.set_launch(["eval", "aba"], 0, "auto")
    ref = {"poses": api.fk(m, q), "J": api.jacobian(m, q, tree.ee), "tau": api.rnea(m, q, qd, qdd),
           "M": api.crba(m, q), "qdd": api.aba(m, q, qd, tau)}
    torch.cuda.synchronize()
    for k in ref:
        g_, r_ = out[k].cpu().numpy(), ref[k].cpu().numpy()
        assert np.all(np.isfinite(g_)), k
        np.testing.assert_allclose(g_, r_, rtol=2e-5, atol=2e-5 * np.abs(r_).max(), err_msg=k)


def test_set_sm_roles_rejects_bad_tables(torch_cuda):
    from paper_2605_31481_gb300 import api, _ffi
    m = api.Model(TREES["chain7"]())
    with pytest.raises(_ffi.FstError):
        m.set_sm_roles([5] * 10)
    with pytest.raises(_ffi.FstError):
        m.set_sm_roles(["aba"] * 300)
    with pytest.raises(_ffi.FstError):
        m.set_launch(["rnea"], 64, "pinned")                 # eval and ABA only


def test_sm_ids_lists_every_sm_once(torch_cuda):
    """fst_sm_ids: as many distinct hardware SM ids as the device has SMs,
    sorted; a role table over them gives each role its requested SM count."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autotune
    ids = api.sm_ids()
    n = torch.cuda.get_device_properties(0).multi_processor_count
    assert len(ids) == n and ids == sorted(set(ids))
    roles = autotune.StepPlan.pin_roles([n // 2, n // 4, n // 8, n - n // 2 - n // 4 - n // 8], ids=ids)
    assert sum(roles[i] == "aba" for i in ids if i < 256) == n // 2
