"""Host-side parts of bench.py and the step planner that need no GPU: the
reference arm's JSON line (the FP64 oracle, sampled so the run stays short)
and the SM role table of the pinned mode."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "10",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "env-evals/s" and d["higher_is_better"] is True
    assert d["steps"] == 10 and d["warmup"] == 3 and d["value"] > 0 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "env-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert 1 <= d["config"]["sample_envs_per_step"] <= 256


def test_bench_refuses_too_few_warmup_steps():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", "2"], capture_output=True,
                       text=True, timeout=120, cwd=ROOT)
    assert r.returncode != 0 and "warmup" in r.stderr


def test_pin_roles_counts_and_spread():
    """The pinned step's SM table: exactly the requested SM count per role
    over the first sum(counts) ids, every role spread along the ids (each
    half of the ids holds about half of each role's SMs), no role past them."""
    sys.path.insert(0, ROOT)
    from paper_2605_31481_gb300.autotune import StepPlan
    for counts in ((64, 32, 24, 32), (56, 40, 16, 40), (76, 25, 25, 26)):
        roles = StepPlan.pin_roles(list(counts))
        n = sum(counts)
        assert len(roles) == 256 and set(roles[n:]) <= {"none"}
        for name, c in zip(("aba", "kin", "rnea", "crba"), counts):
            assert roles[:n].count(name) == c
            assert abs(roles[:n // 2].count(name) - c / 2) <= 1.5
    # over hardware ids with gaps: the roles land on the given ids only
    ids = [i for i in range(200) if i % 9 != 4][:152]
    roles = StepPlan.pin_roles([64, 32, 24, 32], ids=ids)
    assert [roles[i] for i in range(256) if i not in ids] == ["none"] * (256 - 152)
    assert sorted(roles[i] for i in ids).count("aba") == 64


def test_algorithmic_bytes_per_environment():
    """FP32 inputs and outputs per environment of each operator: FK
    4(nq + 12 n_b), Jacobian 4(nq + 6 nv k), RNEA and ABA 4(nq + 3 nv), CRBA
    4(nq + nv^2), at the three benchmark trees (7-DOF chain with one
    end-effector, 11-DOF quadruped with four feet, floating humanoid with
    nq = 30, nv = 29 and 24 bodies)."""
    from paper_2605_31481_gb300 import costs, workloads as w
    chain, quad, hum = w.chain(7), w.spined_quadruped(), w.humanoid()
    assert (hum.nq, hum.nv, hum.n_bodies) == (30, 29, 24)
    expect = {"fk": (364, 572, 1272), "rnea": (112, 176, 468), "aba": (112, 176, 468), "crba": (224, 528, 3484)}
    for op, values in expect.items():
        assert tuple(costs.io_bytes(t, op) for t in (chain, quad, hum)) == values, op
    assert costs.io_bytes(chain, "jacobian", 1) == 196 and costs.io_bytes(quad, "jacobian", 4) == 1100
    # the timed step (FK + 4 foot Jacobians + RNEA + CRBA + ABA on the
    # quadruped) reads q, qd, qdd and tau once: the operators' sum less the
    # four extra reads of q and the second read of qd, 2332 B
    ops = sum(costs.io_bytes(quad, op, 4) for op in ("fk", "jacobian", "rnea", "crba", "aba"))
    assert ops - 4 * (4 * quad.nq + quad.nv) == 2332


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 times the reference arm and prints; the
    other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "10", "--warmup", "3"], capture_output=True, text=True, timeout=120, cwd=ROOT,
                       env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_cpu_baseline_parity_report():
    """The CPU-baseline leg's parity report on stand-in GPU outputs (the
    oracle's own results rounded to FP32, in the step's [field][B] layout):
    the largest and the 99.9th-percentile normwise error per output, the
    backward error of the accelerations and the conditioning of M; and a
    wrong output fails the check."""
    import numpy as np
    import pytest
    sys.path.insert(0, ROOT)
    import bench
    from oracle import rbd
    from paper_2605_31481_gb300 import workloads as w
    tree = w.spined_quadruped(seed=0)
    links = list(tree.ee)
    Bs = 24
    s = w.random_state(tree, Bs, seed=1)
    T = rbd.fk(tree, s["q"])
    out = {"poses": np.concatenate([T[..., :3, :3].reshape(Bs, -1, 9), T[..., :3, 3]], -1),
           "J": np.stack([rbd.jacobian(tree, s["q"], l) for l in links], 1),
           "tau": rbd.rnea(tree, s["q"], s["qd"], s["qdd"]), "M": rbd.crba(tree, s["q"]),
           "qdd": rbd.aba(tree, s["q"], s["qd"], s["tau"])}
    first = {k: np.moveaxis(v.astype(np.float32).astype(np.float64), 0, -1) for k, v in out.items()}
    cpu, parity, detail = bench.cpu_baseline(tree, links, None, s, first, budget_s=0.05, Bs=Bs)
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["value"] > 0
    assert set(parity) == {"poses", "J", "tau", "M", "qdd"} and max(parity.values()) < 1e-6
    assert detail["envs"] == Bs and set(detail["p99_9"]) == set(parity)
    assert all(detail["p99_9"][k] <= parity[k] for k in parity)
    assert 0 < detail["qdd_backward_error"]["max"] < 1e-5
    assert detail["cond2_M"]["max"] >= detail["cond2_M"]["median"] >= 1.0
    first["tau"][3] += 1e-2                        # a wrong torque row fails the check
    with pytest.raises(RuntimeError):
        bench.cpu_baseline(tree, links, None, s, first, budget_s=0.05, Bs=Bs)
