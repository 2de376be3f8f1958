"""Hand-written adjoint kernels (through the C ABI) against the oracle's
reference gradients (complex-step derivatives and the regressor), plus the
determinism of the thetabar reduction and the autograd wrappers."""
import numpy as np
import pytest

from oracle import rbd, derivs
from paper_2605_31481_gb300 import workloads as w
from tests._helpers import env_err, from_soa, to_soa_cuda, oracle_poses, solve_backward_err
from tests.test_gpu_parity import TREES

pytestmark = pytest.mark.gpu

GTOL = 2e-4          # per-environment normwise relative error of q/qd/qdd/tau cotangents
THTOL = 2e-4         # thetabar relative to its largest entry
BWD_BAR = 1e-5       # normwise backward error of an M^-1 product (lambda = M^-1 qdd_bar): ~150 FP32 roundings
COND_MAX = 1e3       # forward-error checks of M^-1 products only where cond(M) is below this
FWD_BAR = 2e-3       # = COND_MAX x 2e-6, a backward error of about 30 FP32 roundings


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_31481_gb300 import build
    build.build(quiet=True)
    return torch


def _th_err(g, r):
    return np.abs(np.asarray(g, np.float64) - r).max() / max(np.abs(r).max(), 1e-30)


@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8"])
def test_rnea_vjp_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 161                                    # 5 tiles of 32 plus a tail of 1
    s = w.random_state(tree, B, seed=3)
    rng = np.random.default_rng(1)
    tb = rng.standard_normal((B, tree.nv))
    m = api.Model(tree)
    q, qd, qdd, tbar = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], tb))
    res = api.rnea_vjp(m, q, qd, qdd, tbar)
    torch.cuda.synchronize()
    rq, rqd, rqdd, rth = derivs.rnea_vjp(tree, s["q"], s["qd"], s["qdd"], tb)
    for k, ref in (("q", rq), ("qd", rqd), ("qdd", rqdd)):
        err = env_err(from_soa(res[k]), ref)
        assert err.max() <= GTOL, f"{name} {k}: {err.max():.3e}"
    assert _th_err(res["theta"].cpu().numpy(), rth) <= THTOL


def _check_aba_vjp(tree, s, qdd_gpu, qb, res, label, theta=None, full_theta=True):
    """The ABA adjoint, checked without a bar that grows with cond(M).

    The adjoint is lambda = M^-1 qdd_bar (returned as tau_bar), then
    {q_bar, qd_bar, theta_bar} = -RNEA-adjoint(q, qd, qdd; lambda) at the
    forward result qdd (the implicit-function identity that the oracle's
    pins hold exactly). So:
      * lambda: its backward error as a solution of M lambda = qdd_bar, with
        the oracle's FP64 M, is held to BWD_BAR (unscaled);
      * q_bar, qd_bar, theta_bar: held to the RNEA-adjoint bar against the
        oracle's FP64 RNEA adjoint evaluated at the kernel's own qdd and
        lambda, which isolates the FP32 rounding of that second stage;
      * the forward error against the oracle's complex-step ABA cotangents
        is held to FWD_BAR only where cond(M) < COND_MAX.
    Returns the measured maxima for the log."""
    M = rbd.crba(tree, s["q"], theta=theta)
    lam = from_soa(res["tau"])
    bwd = solve_backward_err(M, lam, qb)
    assert bwd.max() <= BWD_BAR, f"{label} tau_bar backward error {bwd.max():.3e}"
    rq, rqd, _, rth = derivs.rnea_vjp(tree, s["q"], s["qd"], qdd_gpu, lam, theta=theta)
    meas = {"tau_bar_backward": float(bwd.max())}
    for k, ref in (("q", -rq), ("qd", -rqd)):
        err = env_err(from_soa(res[k]), ref)
        meas[k + "_bar_at_kernel_lambda"] = float(err.max())
        assert err.max() <= GTOL, f"{label} {k}: {err.max():.3e}"
    if full_theta:
        e = _th_err(res["theta"].cpu().numpy(), -rth)
        meas["theta_bar_at_kernel_lambda"] = float(e)
        assert e <= THTOL, f"{label} theta: {e:.3e}"
    good = np.linalg.cond(M) < COND_MAX
    if good.any():
        idx = np.flatnonzero(good)
        fq, fqd, ftau, _ = derivs.aba_vjp(tree, s["q"][idx], s["qd"][idx], s["tau"][idx], qb[idx], theta=theta)
        for k, ref in (("q", fq), ("qd", fqd), ("tau", ftau)):
            err = env_err(from_soa(res[k])[idx], ref)
            meas[k + "_bar_forward_cond<1e3"] = float(err.max())
            assert err.max() <= FWD_BAR, f"{label} forward {k}: {err.max():.3e}"
    return meas


@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8"])
def test_aba_vjp_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 97
    s = w.random_state(tree, B, seed=4)
    rng = np.random.default_rng(2)
    qb = rng.standard_normal((B, tree.nv))
    m = api.Model(tree)
    q, qd, tau, qbar = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["tau"], qb))
    qdd = api.aba(m, q, qd, tau)
    res = api.aba_vjp(m, q, qd, qdd, qbar)
    torch.cuda.synchronize()
    meas = _check_aba_vjp(tree, s, from_soa(qdd), qb, res, name)
    print(f"aba_vjp {name} B={B}: " + ", ".join(f"{k} {v:.2e}" for k, v in meas.items()))


@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8"])
def test_fk_vjp_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 70
    s = w.random_state(tree, B, seed=5)
    rng = np.random.default_rng(3)
    pb = rng.standard_normal((B, tree.n_bodies, 12))
    m = api.Model(tree)
    q = to_soa_cuda(s["q"], torch)
    pbar = torch.from_numpy(np.ascontiguousarray(np.moveaxis(pb, 0, -1).astype(np.float32))).cuda()
    qbar = api.fk_vjp(m, q, pbar)
    torch.cuda.synchronize()
    ref = derivs.fk_vjp(tree, s["q"], pb)
    err = env_err(from_soa(qbar), ref)
    assert err.max() <= GTOL, f"{name}: {err.max():.3e}"


def test_loss_grad_matches_oracle_and_is_deterministic(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES["chain7"]()
    B = 8192 + 13
    s = w.random_state(tree, B, seed=6)
    rng = np.random.default_rng(4)
    tau_true = rbd.rnea(tree, s["q"], s["qd"], s["qdd"])
    tau_meas = tau_true * (1 + 0.05 * rng.standard_normal(tau_true.shape))
    m = api.Model(tree)
    q, qd, qdd, tm = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], tau_meas))
    th = rbd.Model(tree).theta() * (1 + rng.uniform(-0.3, 0.3, (tree.n_bodies, 10)))
    tht = torch.from_numpy(th.astype(np.float32)).cuda()
    L, thb, qb, qdb = api.rnea_loss_grad(m, q, qd, qdd, tm, theta=tht, q_bar=True, qd_bar=True)
    L2, thb2, _, _ = api.rnea_loss_grad(m, q, qd, qdd, tm, theta=tht)
    torch.cuda.synchronize()
    assert torch.equal(thb, thb2) and torch.equal(L, L2)          # bit-reproducible
    r = rbd.rnea(tree, s["q"], s["qd"], s["qdd"], theta=th) - tau_meas
    L_ref = np.sum(r * r)
    assert abs(float(L) - L_ref) / L_ref < 1e-4
    idx = np.arange(0, B, 97)
    rq, rqd, _, _ = derivs.rnea_vjp(tree, s["q"][idx], s["qd"][idx], s["qdd"][idx], 2 * r[idx], theta=th)
    assert env_err(from_soa(qb)[idx], rq).max() <= GTOL
    assert env_err(from_soa(qdb)[idx], rqd).max() <= GTOL
    Y = derivs.regressor(tree, s["q"], s["qd"], s["qdd"])
    th_ref = np.einsum("bi,bink->nk", 2 * r, Y)
    assert _th_err(thb.cpu().numpy(), th_ref) <= THTOL


def test_theta_bar_is_bit_reproducible(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES["quadruped11"]()
    B = 4096
    s = w.random_state(tree, B, seed=7)
    m = api.Model(tree)
    q, qd, qdd, tb = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd", "tau"))
    a = api.rnea_vjp(m, q, qd, qdd, tb)["theta"]
    b = api.rnea_vjp(m, q, qd, qdd, tb)["theta"]
    assert torch.equal(a, b)


def test_autograd_wrappers(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autograd
    tree = TREES["quadruped11"]()
    B = 300
    s = w.random_state(tree, B, seed=8)
    m = api.Model(tree)
    q, qd, qdd, tau = (to_soa_cuda(s[k], torch).requires_grad_() for k in ("q", "qd", "qdd", "tau"))
    th0 = torch.from_numpy(rbd.Model(tree).theta().astype(np.float32)).cuda().requires_grad_()
    out = autograd.rnea(m, q, qd, qdd, th0)
    g = torch.randn_like(out)
    out.backward(g)
    ref = api.rnea_vjp(m, q.detach(), qd.detach(), qdd.detach(), g, theta=th0.detach())
    for t, k in ((q, "q"), (qd, "qd"), (qdd, "qdd"), (th0, "theta")):
        assert torch.equal(t.grad, ref[k]), k
    # FK and ABA through autograd against the oracle
    q2 = to_soa_cuda(s["q"], torch).requires_grad_()
    poses = autograd.fk(m, q2)
    pb = torch.randn_like(poses)
    poses.backward(pb)
    ref = derivs.fk_vjp(tree, s["q"], np.moveaxis(pb.cpu().numpy().astype(np.float64), -1, 0))
    assert env_err(from_soa(q2.grad), ref).max() <= GTOL
    tau2 = to_soa_cuda(s["tau"], torch).requires_grad_()
    qdd2 = autograd.aba(m, to_soa_cuda(s["q"], torch), to_soa_cuda(s["qd"], torch), tau2)
    gq = torch.randn_like(qdd2)
    qdd2.backward(gq)
    M = rbd.crba(tree, s["q"])
    qbn = np.moveaxis(gq.cpu().numpy().astype(np.float64), -1, 0)
    assert solve_backward_err(M, from_soa(tau2.grad), qbn).max() <= BWD_BAR


@pytest.mark.parametrize("specialize", [False, True])
@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8"])
def test_rnea_store_variant_matches_oracle_and_recompute(torch_cuda, name, specialize):
    """Store variant: fst_rnea_store writes the forward tape, and
    fst_rnea_vjp_stored gives the oracle's cotangents (and the recompute
    variant's within FP32 rounding) without re-running the forward sweep."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 161
    s = w.random_state(tree, B, seed=13)
    rng = np.random.default_rng(11)
    tb = rng.standard_normal((B, tree.nv))
    m = api.Model(tree, specialize=["rnea_store", "rnea_vjp_stored", "rnea_vjp"] if specialize else None)
    th = rbd.Model(tree).theta() * (1 + rng.uniform(-0.2, 0.2, (tree.n_bodies, 10)))
    tht = torch.from_numpy(th.astype(np.float32)).cuda()
    q, qd, qdd, tbar = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], tb))
    tau, tape = api.rnea_store(m, q, qd, qdd, theta=tht)
    assert tape.numel() == 30 * tree.n_bodies * B
    tau_plain = api.rnea(m, q, qd, qdd, theta=tht)
    res = api.rnea_vjp_stored(m, q, qd, tape, tbar, theta=tht)
    rec = api.rnea_vjp(m, q, qd, qdd, tbar, theta=tht)
    torch.cuda.synchronize()
    assert env_err(from_soa(tau), rbd.rnea(tree, s["q"], s["qd"], s["qdd"], theta=th)).max() <= 1e-4
    assert env_err(from_soa(tau), from_soa(tau_plain)).max() <= 1e-6
    rq, rqd, rqdd, rth = derivs.rnea_vjp(tree, s["q"], s["qd"], s["qdd"], tb, theta=th)
    for k, ref in (("q", rq), ("qd", rqd), ("qdd", rqdd)):
        err = env_err(from_soa(res[k]), ref)
        assert err.max() <= GTOL, f"{name} {k}: {err.max():.3e}"
        assert env_err(from_soa(res[k]), from_soa(rec[k])).max() <= 1e-5, k
    assert _th_err(res["theta"].cpu().numpy(), rth) <= THTOL
    assert _th_err(res["theta"].cpu().numpy(), rec["theta"].cpu().numpy().astype(np.float64)) <= 1e-5
    # the tape of the first environment holds X, v, a and the accumulated force of body 0
    X0 = tape.view(tree.n_bodies, 30, B)[0, :, 0].cpu().numpy()
    R = X0[:9].reshape(3, 3)
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-5


def test_rnea_store_rejects_small_tape(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, _ffi
    tree = TREES["chain7"]()
    m = api.Model(tree)
    B = 64
    s = w.random_state(tree, B, seed=1)
    q, qd, qdd = (to_soa_cuda(s[k], torch) for k in ("q", "qd", "qdd"))
    small = torch.empty(30 * tree.n_bodies * B - 1, device="cuda")
    with pytest.raises(_ffi.FstError):
        api.rnea_store(m, q, qd, qdd, tape=small)
    with pytest.raises(_ffi.FstError):
        api.rnea_vjp_stored(m, q, qd, small, qd)


def test_autograd_store_variant(torch_cuda):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api, autograd
    tree = TREES["quadruped11"]()
    B = 100
    s = w.random_state(tree, B, seed=21)
    m = api.Model(tree)
    th0 = torch.from_numpy(rbd.Model(tree).theta().astype(np.float32)).cuda()
    grads = []
    for store in (False, True):
        q, qd, qdd = (to_soa_cuda(s[k], torch).requires_grad_() for k in ("q", "qd", "qdd"))
        th = th0.clone().requires_grad_()
        tau = autograd.rnea(m, q, qd, qdd, theta=th, store=store)
        (tau * tau).sum().backward()
        grads.append([x.grad for x in (q, qd, qdd, th)])
    for a, b in zip(*grads):
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-5 * float(b.abs().max()))


@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8", "urdf_arm6_tool"])
def test_jacobian_vjp_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 75
    s = w.random_state(tree, B, seed=41)
    links = list(tree.ee)[:4] or [tree.n_bodies - 1]
    rng = np.random.default_rng(5)
    Jb = rng.standard_normal((B, len(links), 6, tree.nv))
    m = api.Model(tree)
    q = to_soa_cuda(s["q"], torch)
    Jbar = torch.from_numpy(np.ascontiguousarray(np.moveaxis(Jb, 0, -1).astype(np.float32))).cuda()
    qbar = api.jacobian_vjp(m, q, links, Jbar)
    torch.cuda.synchronize()
    ref = derivs.jacobian_vjp(tree, s["q"], links, Jb)
    err = env_err(from_soa(qbar), ref)
    assert err.max() <= GTOL, f"{name}: {err.max():.3e}"


@pytest.mark.parametrize("name", ["chain7", "quadruped11", "humanoid29", "general8"])
def test_crba_vjp_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    B = 67
    s = w.random_state(tree, B, seed=42)
    rng = np.random.default_rng(6)
    Mb = rng.standard_normal((B, tree.nv, tree.nv))
    th = rbd.Model(tree).theta() * (1 + rng.uniform(-0.2, 0.2, (tree.n_bodies, 10)))
    m = api.Model(tree)
    q = to_soa_cuda(s["q"], torch)
    Mbar = torch.from_numpy(np.ascontiguousarray(np.moveaxis(Mb, 0, -1).astype(np.float32))).cuda()
    tht = torch.from_numpy(th.astype(np.float32)).cuda()
    res = api.crba_vjp(m, q, Mbar, theta=tht)
    again = api.crba_vjp(m, q, Mbar, theta=tht)
    torch.cuda.synchronize()
    rq, rth = derivs.crba_vjp(tree, s["q"], Mb, theta=th)
    err = env_err(from_soa(res["q"]), rq)
    assert err.max() <= GTOL, f"{name} q: {err.max():.3e}"
    assert _th_err(res["theta"].cpu().numpy(), rth) <= THTOL
    assert torch.equal(res["theta"], again["theta"]) and torch.equal(res["q"], again["q"])


FULL_SIZES = [("chain7", 8192), ("quadruped11", 8192), ("humanoid29", 65536), ("chain7", 65536)]


@pytest.mark.parametrize("specialize", [False, True])
@pytest.mark.parametrize("name,B", FULL_SIZES)
def test_adjoints_full_size_sampled(torch_cuda, name, B, specialize):
    """Every adjoint at the batch sizes of the workloads, where the launchers
    pick 64- and 128-thread blocks and hundreds of theta_bar partial sums:
    per-environment cotangents on sampled environments against the oracle,
    and theta_bar over the whole batch (through the regressor, exact because
    tau and M are linear in theta) where the batch is the 7-DOF chain's."""
    torch = torch_cuda
    from paper_2605_31481_gb300 import api
    tree = TREES[name]()
    s = w.random_state(tree, B, seed=50)
    rng = np.random.default_rng(51)
    kinds = ["fk_vjp", "rnea_vjp", "aba_vjp", "aba"]         # the adjoints that have specialised kernels
    m = api.Model(tree, specialize=kinds if specialize else None)
    tb = rng.standard_normal((B, tree.nv)).astype(np.float32)
    qb = rng.standard_normal((B, tree.nv)).astype(np.float32)
    q, qd, qdd, tau, tbar, qbar = (to_soa_cuda(x, torch) for x in (s["q"], s["qd"], s["qdd"], s["tau"], tb, qb))
    links = list(tree.ee)[:4] or [tree.n_bodies - 1]
    Jb = torch.randn(len(links), 6, tree.nv, B, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    Mb = torch.randn(tree.nv, tree.nv, B, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    pb = torch.randn(tree.n_bodies, 12, B, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    r_rnea = api.rnea_vjp(m, q, qd, qdd, tbar)
    qdd_f = api.aba(m, q, qd, tau)
    r_aba = api.aba_vjp(m, q, qd, qdd_f, qbar)
    r_crba = api.crba_vjp(m, q, Mb)
    r_jac = api.jacobian_vjp(m, q, links, Jb)
    r_fk = api.fk_vjp(m, q, pb)
    torch.cuda.synchronize()
    idx = np.unique(np.r_[np.random.default_rng(0).choice(B, 48, replace=False), 0, B - 1])
    sub = {k: v[idx] for k, v in s.items()}
    tbn, qbn = tb[idx].astype(np.float64), qb[idx].astype(np.float64)
    label = f"{name}@{B}/{'spec' if specialize else 'generic'}"
    meas = {}
    rq, rqd, rqdd, _ = derivs.rnea_vjp(tree, sub["q"], sub["qd"], sub["qdd"], tbn)
    for k, ref in (("q", rq), ("qd", rqd), ("qdd", rqdd)):
        err = env_err(from_soa(r_rnea[k])[idx], ref)
        meas["rnea_vjp " + k] = float(err.max())
        assert err.max() <= GTOL, f"{label} rnea_vjp {k}: {err.max():.3e}"
    sub_res = {k: v[..., idx] for k, v in r_aba.items() if k != "theta"}
    meas.update({"aba_vjp " + k: v for k, v in
                 _check_aba_vjp(tree, sub, from_soa(qdd_f)[idx], qbn, sub_res, label, full_theta=False).items()})
    Mbn = np.moveaxis(Mb.cpu().numpy().astype(np.float64), -1, 0)
    rcq, _ = derivs.crba_vjp(tree, sub["q"], Mbn[idx])
    err = env_err(from_soa(r_crba["q"])[idx], rcq)
    meas["crba_vjp q"] = float(err.max())
    assert err.max() <= GTOL, f"{label} crba_vjp q: {err.max():.3e}"
    Jbn = np.moveaxis(Jb.cpu().numpy().astype(np.float64), -1, 0)
    err = env_err(from_soa(r_jac)[idx], derivs.jacobian_vjp(tree, sub["q"], links, Jbn[idx]))
    meas["jacobian_vjp q"] = float(err.max())
    assert err.max() <= GTOL, f"{label} jacobian_vjp q: {err.max():.3e}"
    pbn = np.moveaxis(pb.cpu().numpy().astype(np.float64), -1, 0)
    err = env_err(from_soa(r_fk)[idx], derivs.fk_vjp(tree, sub["q"], pbn[idx]))
    meas["fk_vjp q"] = float(err.max())
    assert err.max() <= GTOL, f"{label} fk_vjp q: {err.max():.3e}"
    if name == "chain7" and B == 8192:
        # theta_bar over all 8192 environments: RNEA and ABA adjoints through
        # the regressor Y (tau = Y theta), CRBA's through M's linearity
        Y = derivs.regressor(tree, s["q"], s["qd"], s["qdd"])
        e = _th_err(r_rnea["theta"].cpu().numpy(), np.einsum("bi,bink->nk", tb.astype(np.float64), Y))
        meas["rnea_vjp theta"] = float(e)
        assert e <= THTOL, f"{label} rnea theta {e:.3e}"
        lam = from_soa(r_aba["tau"])
        Ya = derivs.regressor(tree, s["q"], s["qd"], from_soa(qdd_f))
        e = _th_err(r_aba["theta"].cpu().numpy(), -np.einsum("bi,bink->nk", lam, Ya))
        meas["aba_vjp theta (at kernel lambda)"] = float(e)
        assert e <= THTOL, f"{label} aba theta {e:.3e}"
        th_ref = np.zeros((tree.n_bodies, 10))
        for b in range(tree.n_bodies):
            for k in range(10):
                u = np.zeros((tree.n_bodies, 10))
                u[b, k] = 1.0
                th_ref[b, k] = np.sum(Mbn * rbd.crba(tree, s["q"], theta=u))
        e = _th_err(r_crba["theta"].cpu().numpy(), th_ref)
        meas["crba_vjp theta"] = float(e)
        assert e <= THTOL, f"{label} crba theta {e:.3e}"
    print(f"{label}: " + ", ".join(f"{k} {v:.2e}" for k, v in meas.items()))
