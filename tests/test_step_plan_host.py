"""The step planner's selection and cache logic on the host, with the
measurements, the tuner, the kernels and the CUDA streams replaced by fakes
(no GPU): it keeps the fastest measured combination, applies its launch
settings and carveout, and a second planner reads the same decision back
from the cache without measuring."""
import json

import pytest

from paper_2605_31481_gb300 import autotune


class FakeModel:
    device = "cpu"
    ee = (1, 2)
    fingerprint = "fake"
    nq = nv = 3
    n_bodies = 3

    def __init__(self):
        self.launch = {}
        self.roles = None

    def set_launch(self, kinds, block, variant):
        for k in kinds:
            self.launch[k] = (variant, block)

    def set_sm_roles(self, roles):
        self.roles = list(roles)


@pytest.fixture
def fakes(monkeypatch, tmp_path):
    monkeypatch.setenv("FST_TUNE_CACHE", str(tmp_path / "tune.json"))
    carve = []
    monkeypatch.setattr(autotune.api, "set_smem_carveout", lambda c: carve.append(c))
    cands = {"specialized/128": 17.0, "specialized/256": 21.0, "level/256": 17.1, "generic/64": 22.0}
    aba = {"level/256": 10.2, "level/128": 10.4, "specialized/64": 14.3}
    tuned = {k: {"variant": "specialized", "block": 64, "us": 5.0, "candidates": {"specialized/64": 5.0}}
             for k in autotune.FORWARD_KINDS}
    tuned["aba"] = {"variant": "level", "block": 256, "us": 10.2, "candidates": aba}
    tuned["eval"] = {"variant": "specialized", "block": 128, "us": 17.0, "candidates": cands}
    monkeypatch.setattr(autotune, "tune", lambda *a, **k: tuned)
    monkeypatch.setattr(autotune.torch.cuda, "Stream", lambda *a, **k: object())
    monkeypatch.setattr(autotune, "ColdSets", lambda *a, **k: type("C", (), {"R": 1, "sets": [{}]})())
    monkeypatch.setattr(autotune, "sm_count", lambda device: 152)
    monkeypatch.setattr(autotune, "sm_ids", lambda device: list(range(152)))
    monkeypatch.setattr(autotune, "_key", lambda model, kind, B: f"{model.fingerprint}|{kind}|{B}")
    calls = []

    def fake_time(fn):
        m = current["plan"]
        t = {"fused": 17.0, "hybrid": 16.0, "split": 16.5, "pinned": 27.0, "concurrent": 25.0,
             "sequential": 33.0}[m.mode]
        ev = m.model.launch.get("eval")
        if m.mode == "hybrid" and ev == ("specialized", 128) and m.alt and carve[-1] == 100:
            t = 14.5                                   # the one combination that wins
        calls.append((m.mode, carve[-1], m.alt, ev))
        return t

    current = {}
    monkeypatch.setattr(autotune.StepPlan, "_time", lambda self, cold: fake_time(None))
    monkeypatch.setattr(autotune.StepPlan, "__call__", lambda self, *a: None)
    return {"current": current, "calls": calls, "carve": carve, "tmp": tmp_path}


def test_plan_keeps_the_fastest_combination_and_caches_it(fakes):
    model = FakeModel()
    orig_init = autotune.StepPlan.__init__

    def init(self, *a, **k):
        fakes["current"]["plan"] = self
        orig_init(self, *a, **k)

    autotune.StepPlan.__init__ = init
    try:
        plan = autotune.StepPlan(model, 4096)
        assert (plan.mode, plan.carveout, plan.alt) == ("hybrid", 100, True)
        assert plan.eval_config.startswith("specialized/128|") and plan.expected_us == 14.5
        assert model.launch["eval"] == ("specialized", 128) and fakes["carve"][-1] == 100
        d = plan.describe()
        assert d["fused_forked_first"] is True and d["priorities"] is False
        assert min(d["us"].values()) == 14.5
        n_measured = len(fakes["calls"])
        assert n_measured > 20
        cache = json.load(open(fakes["tmp"] / "tune.json"))
        assert any(k.endswith("|plan11|4096") for k in cache)
        # a second planner reads the decision back without measuring
        model2 = FakeModel()
        plan2 = autotune.StepPlan(model2, 4096)
        assert len(fakes["calls"]) == n_measured
        assert (plan2.mode, plan2.carveout, plan2.alt, plan2.eval_config) == \
               (plan.mode, plan.carveout, plan.alt, plan.eval_config)
        assert model2.launch["eval"] == ("specialized", 128)
    finally:
        autotune.StepPlan.__init__ = orig_init


def test_fork_order_and_priority_options(fakes):
    plan = autotune.StepPlan.__new__(autotune.StepPlan)
    plan._plain, plan._ranked = ["p"], ["r"]
    plan._set_alt("concurrent", True)
    assert plan.prio and plan.streams == ["r"]
    plan._set_alt("hybrid", True)
    assert plan.alt and not plan.prio and plan.streams == ["p"]
    plan._set_alt("fused", False)
    assert not plan.alt and not plan.prio


def test_every_described_plan_parses_back_to_its_measurement(fakes):
    model = FakeModel()
    orig_init = autotune.StepPlan.__init__

    def init(self, *a, **k):
        fakes["current"]["plan"] = self
        orig_init(self, *a, **k)

    autotune.StepPlan.__init__ = init
    try:
        plan = autotune.StepPlan(model, 4096, use_cache=False)
        names = plan.describe()["us"]
        assert len(names) == len(plan.times)
        for name, us in names.items():
            mode, carveout, alt, ev = autotune.StepPlan.parse_key(name)
            if ev is None:                       # modes whose launches the per-kind tuning sets
                ev = next(e for (m, c, a, e) in plan.times if (m, c, a) == (mode, carveout, alt))
            assert round(plan.times[(mode, carveout, alt, ev)], 3) == us
    finally:
        autotune.StepPlan.__init__ = orig_init


def test_fixed_plan_runs_without_tuning_or_search(fakes, monkeypatch):
    def no_tune(*a, **k):
        raise AssertionError("a fixed plan with its launch configurations tunes nothing")

    monkeypatch.setattr(autotune, "tune", no_tune)
    model = FakeModel()
    orig_init = autotune.StepPlan.__init__

    def init(self, *a, **k):
        fakes["current"]["plan"] = self
        orig_init(self, *a, **k)

    autotune.StepPlan.__init__ = init
    try:
        plan = autotune.StepPlan(model, 4096, fixed="hybrid[specialized/128|level/128]@100%+fusedfirst")
        assert len(fakes["calls"]) == 1
        assert (plan.mode, plan.carveout, plan.alt) == ("hybrid", 100, True)
        assert model.launch == {"eval": ("specialized", 128), "aba": ("level", 128)}
        assert fakes["carve"][-1] == 100 and plan.expected_us == 14.5
        d = plan.describe()
        assert d["kinds"] == {"eval": "specialized/128", "aba": "level/128"} and d["eval_candidates_us"] == {}
        assert list(d["us"]) == ["hybrid[specialized/128|level/128]@100%+fusedfirst"]
    finally:
        autotune.StepPlan.__init__ = orig_init


@pytest.mark.parametrize("bad", ["hybrid+prio", "fused+fusedfirst", "hybrid[specialized/128]", "warp",
                                 "concurrent@101%"])
def test_fixed_plan_names_are_checked(bad):
    with pytest.raises(ValueError):
        autotune.StepPlan.parse_key(bad)


@pytest.mark.parametrize("name", ["hybrid[specialized/128|level/128]@100%+fusedfirst", "fused[specialized/128|level/256]",
                                  "split[specialized/128|level/256]+fusedfirst", "concurrent@100%+prio", "sequential",
                                  "pinned[pinned/256|level/256@64-32-24-32]", "fused[mixed/128|levellean/128]"])
def test_bench_describes_a_fixed_plan(fakes, name):
    """bench.py's report of the timed step works from a named plan's
    describe(), with or without the per-kind tuning."""
    import bench
    model = FakeModel()
    orig_init = autotune.StepPlan.__init__

    def init(self, *a, **k):
        fakes["current"]["plan"] = self
        orig_init(self, *a, **k)

    autotune.StepPlan.__init__ = init
    try:
        plan = autotune.StepPlan(model, 4096, fixed=name)
        desc = plan.describe()
        text = bench.plan_kernel_name(plan.mode, desc)
        assert text and (plan.mode in ("concurrent", "sequential") or desc["kinds"]["eval"] in text)
        assert plan.mode in ("fused", "concurrent", "sequential") or desc["kinds"]["aba"] in text
        if desc["kinds"]["eval"].startswith("mixed"):
            assert "aba" in text.split(":")[1].split("level-parallel")[0]   # any level form of ABA is named
        key = (plan.mode, desc["kinds"]["aba"], desc["kinds"]["eval"], bench.kernel_source_hash())
        assert bench.NCU_TRAFFIC.get(key) is None or plan.mode == "hybrid"
        json.dumps(desc)
    finally:
        autotune.StepPlan.__init__ = orig_init


def test_autotune_off_measures_nothing(monkeypatch, tmp_path):
    """FST_AUTOTUNE=0: tune() sets every kind to the built-in heuristics
    (variant auto, block 0) without timing anything, and the step planner
    runs one fused launch, also without timing."""
    monkeypatch.setenv("FST_AUTOTUNE", "0")
    monkeypatch.setenv("FST_TUNE_CACHE", str(tmp_path / "tune.json"))

    def no_timing(*a, **k):
        raise AssertionError("nothing may be timed with FST_AUTOTUNE=0")

    monkeypatch.setattr(autotune, "graph_time_us", no_timing)
    monkeypatch.setattr(autotune, "cold_time_us", no_timing)
    monkeypatch.setattr(autotune, "Buffers", no_timing)
    monkeypatch.setattr(autotune, "ColdSets", no_timing)
    monkeypatch.setattr(autotune.StepPlan, "_time", no_timing)
    monkeypatch.setattr(autotune.api, "set_smem_carveout", lambda c: None)
    monkeypatch.setattr(autotune.torch.cuda, "Stream", lambda *a, **k: object())
    model = FakeModel()
    res = autotune.tune(model, 4096)
    assert set(res) == set(autotune.FORWARD_KINDS + ("eval",))
    assert all(v == {"variant": "auto", "block": 0, "us": None, "candidates": {}} for v in res.values())
    assert all(model.launch[k] == ("auto", 0) for k in res)
    plan = autotune.StepPlan(model, 4096)
    assert plan.mode == "fused" and plan.expected_us is None and plan.eval_config == "auto/0|auto/0"
    desc = plan.describe()
    assert desc["us"] == {"fused": None} and desc["kinds"]["eval"] == "auto/0"
    json.dumps(desc)
    assert not (tmp_path / "tune.json").exists()     # nothing measured, nothing cached
