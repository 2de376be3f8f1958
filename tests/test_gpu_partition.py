"""SM partitions (green contexts) and the partitioned step plan: ABA, the
kinematics, RNEA and CRBA as four launches on four disjoint SM sets give the
same numbers as the same kernels without partitions, eagerly and replayed
from a CUDA graph, and the oracle's."""
import numpy as np
import pytest

from oracle import rbd
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import TOL, env_err, from_soa, oracle_poses, to_soa_cuda

pytestmark = pytest.mark.gpu

PLAN = "specialized/128|level/256"


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


def _outs(torch, tree, B, nl):
    return {"poses": torch.empty(tree.n_bodies, 12, B, device="cuda"),
            "J": torch.empty(nl, 6, tree.nv, B, device="cuda"), "tau": torch.empty(tree.nv, B, device="cuda"),
            "M": torch.empty(tree.nv, tree.nv, B, device="cuda"), "qdd": torch.empty(tree.nv, B, device="cuda")}


def test_partition_streams_and_counts(torch_cuda):
    from paper_2605_31481_gb300 import api
    p = api.SmPartition([64, 32, 30, 20])
    assert p.sm_counts == [64, 32, 32, 24]           # whole groups of 8 SMs
    assert len(p.streams) == 4 and len({s.cuda_stream for s in p.streams}) == 4
    assert api.sm_partition([64, 32, 32, 24]) is api.sm_partition([64, 32, 32, 24])
    p.close()


def test_partition_rejects_bad_counts(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, _ffi
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    for counts in ([n_sm, 8], [0, 8], [-8], [8] * 9, []):
        with pytest.raises(_ffi.FstError):
            api.SmPartition(counts)


@pytest.mark.parametrize("B", [4096, 1000])
def test_partitioned_step_matches_unpartitioned_and_oracle(torch_cuda, B):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autotune
    tree = w.spined_quadruped(seed=0)
    ee = list(tree.ee)
    s = w.random_state(tree, B, seed=31)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    m = api.Model(tree, specialize=True)
    hyb = autotune.StepPlan(m, B, links=ee, fixed=f"hybrid[{PLAN}]")
    ref = _outs(torch, tree, B, len(ee))
    hyb(q, qd, qdd, tau, ref)
    part = autotune.StepPlan(m, B, links=ee, fixed=f"partitioned[{PLAN}@64-32-32-24]")
    eager = _outs(torch, tree, B, len(ee))
    part(q, qd, qdd, tau, eager)
    graphed = _outs(torch, tree, B, len(ee))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        part(q, qd, qdd, tau, graphed)
    for v in graphed.values():
        v.fill_(float("nan"))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(eager[k], ref[k]), k      # the same kernels, so the same bits
        assert torch.equal(graphed[k], ref[k]), k
    idx = np.unique(np.r_[np.arange(0, B, 61), B - 1])
    orc = {"poses": oracle_poses(tree, s["q"][idx]),
           "J": np.stack([rbd.jacobian(tree, s["q"][idx], e) for e in ee], 1),
           "tau": rbd.rnea(tree, s["q"][idx], s["qd"][idx], s["qdd"][idx]), "M": rbd.crba(tree, s["q"][idx]),
           "qdd": rbd.aba(tree, s["q"][idx], s["qd"][idx], s["tau"][idx])}
    for k, tol in TOL.items():
        err = env_err(from_soa(eager[k])[idx], orc[k])
        assert np.all(np.isfinite(err)) and err.max() <= tol, (k, err.max())


def test_partitioned_step_packed_layout(torch_cuda):
    """The partitioned plan writes the packed layouts of eval(packed=True)
    like the hybrid plan."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autotune
    tree = w.spined_quadruped(seed=0)
    ee = list(tree.ee)
    B = 512
    s = w.random_state(tree, B, seed=32)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    m = api.Model(tree, specialize=True)
    _, j_rows, m_rows = api.packed_layout(m, ee)

    def outs():
        o = _outs(torch, tree, B, len(ee))
        o["J"] = torch.empty(j_rows, B, device="cuda")
        o["M"] = torch.empty(m_rows, B, device="cuda")
        return o
    hyb, part = outs(), outs()
    autotune.StepPlan(m, B, links=ee, fixed=f"hybrid[{PLAN}]")(q, qd, qdd, tau, hyb, packed=True)
    autotune.StepPlan(m, B, links=ee, fixed=f"partitioned[{PLAN}@64-32-32-24]")(q, qd, qdd, tau, part, packed=True)
    torch.cuda.synchronize()
    for k in hyb:
        assert torch.equal(hyb[k], part[k]), k
