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


def test_pin_roles_proportions():
    sys.path.insert(0, ROOT)
    from paper_2605_31481_gb300.autotune import StepPlan
    for share in (0.45, 0.55, 0.65):
        roles = StepPlan.pin_roles(share)
        assert len(roles) == 256 and set(roles) <= {"aba", "kin", "rnea", "crba"}
        frac = roles.count("aba") / 256
        assert abs(frac - share) <= 0.05
        others = [roles.count(r) for r in ("kin", "rnea", "crba")]
        assert max(others) - min(others) <= 256 // 20 + 1       # the three roles evenly
