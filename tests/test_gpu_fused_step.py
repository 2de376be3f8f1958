"""The fused controller step of fst_eval: one forward RNEA sweep feeding the
world poses, the Jacobians, tau and the RNEA adjoint's reverse sweeps (the
per-step sequence of the paper's RL experiment, Sec. 4.4, with the gradient
of RNEA). Every output must be bit-identical to the separate operator calls
of the same kernel variant and match the FP64 oracle at the parity bars."""
import numpy as np
import pytest

from oracle import derivs, rbd
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import TOL, env_err, from_soa, oracle_poses, to_soa_cuda
from tests.test_gpu_parity import TREES

pytestmark = pytest.mark.gpu

GTOL = 2e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


@pytest.mark.parametrize("specialize", [False, True])
@pytest.mark.parametrize("name", list(TREES))
def test_fused_step_matches_separate_calls_and_oracle(torch_cuda, name, specialize):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 333                                         # 10 tiles of 32 and a tail of 13
    s = w.random_state(tree, B, seed=61)
    rng = np.random.default_rng(62)
    tbn = rng.standard_normal((B, tree.nv))
    m = api.Model(tree, specialize=["eval", "fk", "jacobian", "rnea", "rnea_vjp"] if specialize else None)
    if not specialize:
        m.set_launch(None, 0, "generic")
    ee = list(tree.ee) if tree.ee else [tree.n_bodies - 1]
    q, qd, qdd, tb = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], tbn))
    sep = {"poses": api.fk(m, q), "J": api.jacobian(m, q, ee), "tau": api.rnea(m, q, qd, qdd)}
    vjp = api.rnea_vjp(m, q, qd, qdd, tb, theta_bar=False)
    vjp_tau = api.rnea_vjp(m, q, qd, qdd, sep["tau"], theta_bar=False)
    ref = {"poses": oracle_poses(tree, s["q"]), "J": np.stack([rbd.jacobian(tree, s["q"], l) for l in ee], 1),
           "tau": rbd.rnea(tree, s["q"], s["qd"], s["qdd"])}
    rq, rqd, rqdd, _ = derivs.rnea_vjp(tree, s["q"], s["qd"], s["qdd"], tbn)
    for one_sweep in (False, True):
        for given in (True, False):
            res = api.eval(m, q, qd, qdd, fk=True, links=ee, rnea=True, q_bar=True, qd_bar=True, qdd_bar=True,
                           tau_bar=tb if given else "tau", one_sweep=one_sweep)
            torch.cuda.synchronize()
            label = f"{name} spec={specialize} one_sweep={one_sweep} tau_bar={'given' if given else 'tau'}"
            for k in ("poses", "J", "tau"):
                assert torch.equal(res[k], sep[k]), f"{label}: {k} differs from the separate call"
                err = env_err(from_soa(res[k]), ref[k])
                assert err.max() <= TOL[k], f"{label}: {k} {err.max():.3e}"
            want = vjp if given else vjp_tau
            for k in ("q", "qd", "qdd"):
                assert torch.equal(res[k + "_bar"], want[k]), f"{label}: {k}_bar differs from fst_rnea_vjp"
            if given:
                for k, r in (("q", rq), ("qd", rqd), ("qdd", rqdd)):
                    err = env_err(from_soa(res[k + "_bar"]), r)
                    assert err.max() <= GTOL, f"{label}: {k}_bar {err.max():.3e}"


def test_fused_step_subsets_and_errors(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, _ffi
    tree = TREES["quadruped11"]()
    m = api.Model(tree)
    B = 100
    s = w.random_state(tree, B, seed=63)
    q, qd, qdd, tb = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    ref = api.rnea_vjp(m, q, qd, qdd, tb, theta_bar=False)
    # the adjoint alone (no tau output), and only one cotangent
    only = api.eval(m, q, qd, qdd, qd_bar=True, tau_bar=tb)
    assert set(only) == {"qd_bar"} and torch.equal(only["qd_bar"], ref["qd"])
    # one_sweep without the RNEA operator: kinematics keep their own blocks
    kin = api.eval(m, q, fk=True, links=list(tree.ee), one_sweep=True)
    assert torch.equal(kin["poses"], api.fk(m, q)) and torch.equal(kin["J"], api.jacobian(m, q, list(tree.ee)))
    # B = 0 and B = 1
    z = torch.empty(tree.nq, 0, device="cuda")
    zv = torch.empty(tree.nv, 0, device="cuda")
    assert api.eval(m, z, zv, zv, rnea=True, q_bar=True, tau_bar="tau")["q_bar"].shape == (tree.nq, 0)
    one = api.eval(m, q[:, :1].contiguous(), qd[:, :1].contiguous(), qdd[:, :1].contiguous(), q_bar=True,
                   tau_bar=tb[:, :1].contiguous())
    torch.cuda.synchronize()
    rq, _, _, _ = derivs.rnea_vjp(tree, s["q"][:1], s["qd"][:1], s["qdd"][:1], s["tau"][:1])
    assert env_err(from_soa(one["q_bar"]), rq).max() <= GTOL
    # a cotangent output without tau_bar, and unknown flags, are refused
    io = _ffi.EvalIO()
    io.q, io.qd, io.qdd = q.data_ptr(), qd.data_ptr(), qdd.data_ptr()
    qb = torch.empty_like(q)
    io.q_bar = qb.data_ptr()
    import ctypes
    L = _ffi.lib()
    assert L.fst_eval(m.handle, B, ctypes.byref(io), None, None) == -1
    assert "tau_bar" in L.fst_last_error().decode()
    io.tau_bar = tb.data_ptr()
    io.flags = 8
    assert L.fst_eval(m.handle, B, ctypes.byref(io), None, None) == -1


def _support_dofs(tree, link):
    """DOF indices on link's support path, in DOF order (from the tree table)."""
    path, i = [], link
    while i >= 0:
        path.append(i)
        i = int(tree.parent[i])
    nvs = [{0: 0, 1: 1, 2: 1, 3: 6}[int(t)] for t in tree.jtype]
    vi = np.concatenate([[0], np.cumsum(nvs)])[:-1]
    return [int(vi[b]) + j for b in sorted(path) for j in range(nvs[b])]


@pytest.mark.parametrize("specialize", [False, True])
@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8"])
def test_packed_layout_holds_the_full_layouts_entries(torch_cuda, name, specialize):
    """FST_EVAL_PACKED: M's upper triangle row by row and each link's
    support-path Jacobian columns, bit-identical to those entries of the full
    layouts; every dropped entry of the full J is a structural zero."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 150
    s = w.random_state(tree, B, seed=64)
    m = api.Model(tree, specialize=["eval"] if specialize else None)
    ee = list(tree.ee) if tree.ee else [tree.n_bodies - 1]
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    full = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True)
    cols, j_rows, m_rows = api.packed_layout(m, ee)
    dofs = [_support_dofs(tree, l) for l in ee]
    assert cols == [len(d) for d in dofs] and j_rows == 6 * sum(cols) and m_rows == tree.nv * (tree.nv + 1) // 2
    nv = tree.nv
    iu = np.triu_indices(nv)
    for one_sweep in (False, True):
        pk = api.eval(m, q, qd, qdd, tau, fk=True, links=ee, rnea=True, crba=True, aba=True, packed=True,
                      one_sweep=one_sweep)
        torch.cuda.synchronize()
        for k in ("poses", "tau", "qdd"):
            assert torch.equal(pk[k], full[k]), k
        Mf = full["M"].cpu().numpy()
        assert pk["M"].shape == (m_rows, B)
        assert np.array_equal(pk["M"].cpu().numpy(), Mf[iu[0], iu[1]])
        Jf = full["J"].cpu().numpy()
        Jp = pk["J"].cpu().numpy()
        off = 0
        for l, d in enumerate(dofs):
            blk = Jp[off:off + 6 * len(d)].reshape(6, len(d), B)
            assert np.array_equal(blk, Jf[l][:, d]), (name, l)
            rest = np.setdiff1d(np.arange(nv), d)
            assert not np.any(Jf[l][:, rest]), (name, l)
            off += 6 * len(d)
        assert off == j_rows
