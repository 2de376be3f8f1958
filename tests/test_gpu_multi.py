"""One persistent launch over a mixed batch of five trees (7, 11, 12, 18 and
23 revolute DOF with 4096, 2048, 1024, 512 and 256 environments): the same
numbers as the per-tree calls, and the oracle's."""
import numpy as np
import pytest

from oracle import rbd
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import TOL, env_err, from_soa, oracle_poses, to_soa_cuda

pytestmark = pytest.mark.gpu

COUNTS = (4096, 2048, 1024, 512, 256)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


def _items(torch, trees, counts, extra=0):
    items, states = [], []
    for k, (t, B) in enumerate(zip(trees, counts)):
        s = w.random_state(t, B + extra, seed=10 + k)
        states.append(s)
        items.append({"q": to_soa_cuda(s["q"], torch), "qd": to_soa_cuda(s["qd"], torch),
                      "qdd": to_soa_cuda(s["qdd"], torch), "tau": to_soa_cuda(s["tau"], torch),
                      "fk": True, "rnea": True, "crba": True, "aba": True})
    return items, states


def test_mixed_batch_equals_per_tree_calls_and_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    trees = w.mixed_trees()
    models = [api.Model(t) for t in trees]
    counts = [c + 7 for c in COUNTS]          # ragged tails in every tree
    items, states = _items(torch, trees, counts)
    mb = api.MultiBatch(models)
    res = mb.eval(items)
    res2 = mb.eval(items)                      # the work counter resets between calls
    torch.cuda.synchronize()
    for m, t, it, r, r2, s in zip(models, trees, items, res, res2, states):
        per = {"poses": api.fk(m, it["q"]), "tau": api.rnea(m, it["q"], it["qd"], it["qdd"]),
               "M": api.crba(m, it["q"]), "qdd": api.aba(m, it["q"], it["qd"], it["tau"])}
        for k in per:
            assert torch.equal(r[k], per[k]), (t.name, k)
            assert torch.equal(r2[k], per[k]), (t.name, k)
        idx = np.arange(0, s["q"].shape[0], 37)
        ref = {"poses": oracle_poses(t, s["q"][idx]), "tau": rbd.rnea(t, s["q"][idx], s["qd"][idx], s["qdd"][idx]),
               "M": rbd.crba(t, s["q"][idx]), "qdd": rbd.aba(t, s["q"][idx], s["qd"][idx], s["tau"][idx])}
        for k in ref:
            assert env_err(from_soa(r[k])[idx], ref[k]).max() <= TOL[k], (t.name, k)


def test_mixed_batch_subsets_and_empty_members(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    trees = w.mixed_trees()[:3]
    models = [api.Model(t) for t in trees]
    items, _ = _items(torch, trees, (100, 0, 33))
    items[0] = {**items[0], "fk": False, "crba": False, "aba": False}
    res = api.MultiBatch(models).eval(items)
    torch.cuda.synchronize()
    assert set(res[0]) == {"tau"} and res[1]["tau"].shape[-1] == 0
    assert torch.equal(res[0]["tau"], api.rnea(models[0], items[0]["q"], items[0]["qd"], items[0]["qdd"]))
    assert torch.equal(res[2]["qdd"], api.aba(models[2], items[2]["q"], items[2]["qd"], items[2]["tau"]))


def test_mixed_batch_replays_from_a_cuda_graph(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    trees = w.mixed_trees()
    models = [api.Model(t) for t in trees]
    items, _ = _items(torch, trees, COUNTS)
    for it in items:
        it["out"] = {"poses": torch.empty(0), "tau": None}
    outs = [{"poses": torch.empty(t.n_bodies, 12, B, device="cuda"), "tau": torch.empty(t.nv, B, device="cuda"),
             "M": torch.empty(t.nv, t.nv, B, device="cuda"), "qdd": torch.empty(t.nv, B, device="cuda")}
            for t, B in zip(trees, COUNTS)]
    for it, o in zip(items, outs):
        it["out"] = o
    mb = api.MultiBatch(models)
    eager = [{k: v.clone() for k, v in r.items()} for r in mb.eval(items)]
    for o in outs:
        for v in o.values():
            v.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mb.eval(items)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for e, o in zip(eager, outs):
        for k in e:
            assert torch.equal(e[k], o[k]), k


@pytest.mark.parametrize("block", [64, 256])
def test_mixed_batch_level_parallel_form(torch_cuda, block):
    """fst_multi_set_launch(FST_VARIANT_LEVEL): items of 32 environments run
    with the level-parallel bodies (ABA in its lean form); bit-identical to
    the per-tree level-parallel calls at the same block (lean ABA), and the
    oracle's numbers."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    trees = w.mixed_trees()
    models = [api.Model(t) for t in trees]
    counts = [c + 5 for c in COUNTS]
    items, states = _items(torch, trees, counts)
    mb = api.MultiBatch(models)
    mb.set_launch(block, "level")
    res = mb.eval(items)
    res2 = mb.eval(items)
    torch.cuda.synchronize()
    for m, t, it, r, r2, s in zip(models, trees, items, res, res2, states):
        m.set_launch(["fk", "rnea", "crba"], block, "level")
        m.set_launch(["aba"], block, "levellean")
        per = {"poses": api.fk(m, it["q"]), "tau": api.rnea(m, it["q"], it["qd"], it["qdd"]),
               "M": api.crba(m, it["q"]), "qdd": api.aba(m, it["q"], it["qd"], it["tau"])}
        for k in per:
            assert torch.equal(r[k], per[k]), (t.name, k)
            assert torch.equal(r2[k], per[k]), (t.name, k)
        idx = np.r_[np.arange(0, s["q"].shape[0], 41), s["q"].shape[0] - 1]
        ref = {"poses": oracle_poses(t, s["q"][idx]), "tau": rbd.rnea(t, s["q"][idx], s["qd"][idx], s["qdd"][idx]),
               "M": rbd.crba(t, s["q"][idx]), "qdd": rbd.aba(t, s["q"][idx], s["qd"][idx], s["tau"][idx])}
        for k in ref:
            assert env_err(from_soa(r[k])[idx], ref[k]).max() <= TOL[k], (t.name, k)


def test_multi_set_launch_rejects_bad_arguments(torch_cuda):
    from paper_2605_31481_gb300 import api, _ffi
    mb = api.MultiBatch([api.Model(w.chain(7, seed=0))])
    with pytest.raises(_ffi.FstError):
        mb.set_launch(96, "level")
    with pytest.raises(_ffi.FstError):
        mb.set_launch(64, "specialized")
