"""Autotuner for the launch configuration of the kernels, and the step planner.

`tune(model, B)` measures, on the current GPU, every candidate configuration
of each kernel kind and keeps the fastest via fst_model_set_launch. A
candidate is an environment-to-thread mapping with a block size (32 to 256
threads):
  generic      one environment per thread, the tree from shared memory;
  specialized  one environment per thread, a kernel compiled for the tree;
  level        32 environments per block, the block's warps splitting each
               tree level;
  level2       the same with two such tiles per block (half the blocks);
  levellean    (CRBA, ABA) the level-parallel kernel with less state per
               body and a two-level ring of contributions to the parent, so
               that more tiles of a large tree fit on one SM;
  mixed        (eval) the specialised fused kernel with each role mapped as
               its own operator is set;
  path         a lane per root-to-leaf path (trees with at most 8 leaves);
  pathwarp     a warp per root-to-leaf path (block size fixed by the tree).

`StepPlan(model, B)` then decides how a step of the five forward operators
runs: one fused launch, ABA beside a fused launch of the other four (the
fused part whole or split in two, or both pinned to disjoint SM sets), every
operator on its own stream, or one after another; each at two
shared-memory carveouts and with its fork-order or stream-priority option.

Timings replay a CUDA graph of repeated launches, so host launch overhead is
excluded. Choices are cached in a JSON file (FST_TUNE_CACHE, default
~/.cache/fst_tune.json) keyed by the tree's fingerprint, the kind, B, the
GPU name and the library version. FST_AUTOTUNE=0 turns all measurement off
(autotune_enabled()): built-in launch heuristics and one fused launch.
"""
from __future__ import annotations

import json
import os
import re
import threading

import torch

from . import api
from . import _ffi

CANDIDATE_BLOCKS = (32, 64, 128, 256)
FORWARD_KINDS = ("fk", "jacobian", "rnea", "crba", "aba")
LEVEL_KINDS = FORWARD_KINDS + ("eval",)   # kinds with a level-parallel variant
_lock = threading.Lock()


def _cache_path():
    return os.environ.get("FST_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "fst_tune.json"))


def _load_cache():
    try:
        with open(_cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(entries):
    path = _cache_path()
    with _lock:
        data = _load_cache()
        data.update(entries)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def graph_time_us(fn, n=20, reps=10, trials=3):
    """Device time of fn() in microseconds, from a CUDA graph of n calls
    replayed reps times (fn must only enqueue work); the best of `trials`
    such measurements, so that one disturbed measurement does not decide."""
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(n):
            fn()
    g.replay()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(trials):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) * 1e3 / (n * reps))
    return best


L2_BYTES = 129 * 2 ** 20    # GB300's L2 cache


def sm_count(device):
    """Streaming multiprocessors of the device."""
    return torch.cuda.get_device_properties(device).multi_processor_count


def sm_ids(device):
    """The hardware ids of the device's SMs (api.sm_ids)."""
    return api.sm_ids(device)


def cold_time_us(fn, R, reps=5, trials=3):
    """Device time per call of fn(k) in microseconds, from a CUDA graph of the
    R calls fn(0) .. fn(R - 1) replayed reps times: with fn(k) working on the
    k-th of R rotating data sets larger than L2 together, every call reads and
    writes HBM. The best of `trials` measurements."""
    for k in range(min(R, 2)):
        fn(k)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for k in range(R):
            fn(k)
    g.replay()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(trials):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) * 1e3 / (R * reps))
    return best


class ColdSets:
    """R rotating copies of a five-operator step's inputs and outputs, more
    than twice the L2 cache together, for timing step plans the way the
    benchmark runs them (cold inputs every step). At most MAX_SETS copies:
    a batch so small that even that many sets fit in L2 is L2-resident in
    use as well."""

    MAX_SETS = 32

    def __init__(self, model, B, links):
        dev = model.device
        nq, nv, nb, nl = model.nq, model.nv, model.n_bodies, len(links)
        per = 4 * B * (nq + 3 * nv + 12 * nb + 6 * nv * nl + nv + nv * nv + nv)
        self.R = min(self.MAX_SETS, max(2, -(-2 * L2_BYTES // per) + 1))
        gen = torch.Generator(device=dev).manual_seed(1)
        r = lambda *sh: torch.randn(*sh, device=dev, generator=gen)
        self.sets = []
        for _ in range(self.R):
            self.sets.append({"q": r(nq, B), "qd": r(nv, B), "qdd": r(nv, B), "tau": r(nv, B),
                              "out": {"poses": torch.empty(nb, 12, B, device=dev),
                                      "J": torch.empty(nl, 6, nv, B, device=dev),
                                      "tau": torch.empty(nv, B, device=dev),
                                      "M": torch.empty(nv, nv, B, device=dev),
                                      "qdd": torch.empty(nv, B, device=dev)}})


class Buffers:
    """Synthetic device inputs and outputs for timing one model at batch B."""

    def __init__(self, model, B, links):
        dev = model.device
        gen = torch.Generator(device=dev).manual_seed(0)
        r = lambda *s: torch.randn(*s, device=dev, generator=gen)
        self.q = r(model.nq, B)   # a free base's quaternion rows are normalised in the kernels
        self.qd, self.qdd, self.tau = r(model.nv, B), r(model.nv, B), r(model.nv, B)
        self.links = list(links)
        self.out = {"poses": torch.empty(model.n_bodies, 12, B, device=dev),
                    "J": torch.empty(len(self.links), 6, model.nv, B, device=dev),
                    "tau": torch.empty(model.nv, B, device=dev), "M": torch.empty(model.nv, model.nv, B, device=dev),
                    "qdd": torch.empty(model.nv, B, device=dev)}
        self.tbar = r(model.nv, B)
        self.pbar = r(model.n_bodies, 12, B)
        self.scratch = api.adjoint_scratch(model, B)
        self.qdd_fwd = torch.empty(model.nv, B, device=dev)
        self.tape = api.rnea_tape(model, B)


def _op(model, kind, buf):
    m, b = model, buf
    if kind == "fk":
        return lambda: api.fk(m, b.q, out=b.out["poses"])
    if kind == "jacobian":
        return lambda: api.jacobian(m, b.q, b.links, out=b.out["J"])
    if kind == "rnea":
        return lambda: api.rnea(m, b.q, b.qd, b.qdd, out=b.out["tau"])
    if kind == "crba":
        return lambda: api.crba(m, b.q, out=b.out["M"])
    if kind == "aba":
        return lambda: api.aba(m, b.q, b.qd, b.tau, out=b.out["qdd"])
    if kind == "eval":
        return lambda: api.eval(m, b.q, b.qd, b.qdd, b.tau, fk=True, links=b.links, rnea=True, crba=True, aba=True,
                                out=b.out)
    if kind == "rnea_vjp":
        return lambda: api.rnea_vjp(m, b.q, b.qd, b.qdd, b.tbar, scratch=b.scratch)
    if kind == "rnea_store":
        return lambda: api.rnea_store(m, b.q, b.qd, b.qdd, tape=b.tape, out=b.out["tau"])
    if kind == "rnea_vjp_stored":
        return lambda: api.rnea_vjp_stored(m, b.q, b.qd, b.tape, b.tbar, scratch=b.scratch)
    if kind == "fk_vjp":
        return lambda: api.fk_vjp(m, b.q, b.pbar)
    if kind == "aba_vjp":
        return lambda: api.aba_vjp(m, b.q, b.qd, b.qdd_fwd, b.tbar, scratch=b.scratch)
    if kind == "loss_grad":
        return lambda: api.rnea_loss_grad(m, b.q, b.qd, b.qdd, b.tau, scratch=b.scratch)
    raise ValueError(kind)


def _key(model, kind, B):
    return f"{model.fingerprint}|{kind}|{B}|{torch.cuda.get_device_name(model.device)}|{_ffi.lib().fst_version().decode()}"


def autotune_enabled():
    """False when FST_AUTOTUNE=0: then nothing is measured. tune() keeps the
    library's built-in launch heuristics (variant auto: the specialised
    kernel where compiled, else the generic one; block 0) and StepPlan runs
    the step as one fused launch."""
    return os.environ.get("FST_AUTOTUNE", "1").strip() != "0"


def tune(model, B, kinds=FORWARD_KINDS + ("eval",), links=None, use_cache=True, verbose=False):
    """Pick and set the fastest (variant, block) for each kind at batch B.
    Returns {kind: {"variant", "block", "us", "candidates"}} ("us" None and
    no candidates when FST_AUTOTUNE=0)."""
    if not autotune_enabled():
        out = {}
        for kind in kinds:
            model.set_launch([kind], 0, "auto")
            out[kind] = {"variant": "auto", "block": 0, "us": None, "candidates": {}}
        return out
    links = list(links if links is not None else (model.ee or (model.n_bodies - 1,)))
    cache = _load_cache() if use_cache else {}
    spec = set(model.specialized())
    buf = None
    result, new = {}, {}
    for kind in kinds:
        key = _key(model, kind, B)
        hit = cache.get(key)
        if hit and (hit["variant"] != "specialized" or kind in spec):
            model.set_launch([kind], hit["block"], hit["variant"])
            result[kind] = hit
            continue
        if buf is None:
            buf = Buffers(model, B, links)
            if "aba_vjp" in kinds:
                api.aba(model, buf.q, buf.qd, buf.tau, out=buf.qdd_fwd)
            if "rnea_vjp_stored" in kinds:
                api.rnea_store(model, buf.q, buf.qd, buf.qdd, tape=buf.tape, tau=False)
        fn = _op(model, kind, buf)
        cands = {}
        variants = ["generic"] + (["specialized"] if kind in spec else []) + \
            (["level", "level2"] if kind in LEVEL_KINDS else []) + (["levellean"] if kind in ("aba", "crba") else [])
        if kind == "eval" and "eval_mixed" in spec:
            variants.append("mixed")       # specialised fused kernel, roles mapped as their operators
        if kind in spec and kind in LEVEL_KINDS:
            variants += ["path", "pathwarp"]   # path-parallel, where the tree has at most 8 leaves
        for variant in variants:
            blocks = (0,) if variant == "pathwarp" else CANDIDATE_BLOCKS[1:] if variant == "level2" else \
                CANDIDATE_BLOCKS[2:] if variant == "levellean" else CANDIDATE_BLOCKS
            for block in blocks:
                try:
                    model.set_launch([kind], block, variant)
                except _ffi.FstError:
                    break                      # no such kernel for this tree
                cands[f"{variant}/{block}"] = graph_time_us(fn)
        best = min(cands, key=cands.get)
        variant, block = best.split("/")
        model.set_launch([kind], int(block), variant)
        entry = {"variant": variant, "block": int(block), "us": round(cands[best], 3),
                 "candidates": {k: round(v, 3) for k, v in cands.items()}}
        result[kind] = new[key] = entry
        if verbose:
            print(f"[autotune] {model.name} B={B} {kind}: {best} {cands[best]:.2f} us")
    if new and use_cache:
        _store_cache(new)
    return result


class StepPlan:
    """How to run the five forward operators on one batch, whichever the
    tuner measured fastest (each operator already at its tuned
    configuration):
      fused       one launch (fst_eval), operators side by side in one kernel
                  with one variant for all of them;
      hybrid      ABA's own kernel (at its best variant) on a side stream,
                  overlapping one fused launch of the four other operators;
      split       the same, with that fused launch split in two (FK with the
                  Jacobians; RNEA with CRBA) on two more branches;
      pinned      one launch of one block per SM, each SM serving one operator
                  (fst_eval with FST_VARIANT_PINNED; SM counts tuned);
      partitioned ABA, the kinematics (FK with the Jacobians), RNEA and CRBA
                  as four launches on four disjoint SM partitions (green
                  contexts, fst_sm_partition_create; SM counts tuned), so no
                  SM runs two operators' code;
      concurrent  each operator's own kernel on its own stream;
      sequential  the per-operator kernels one after another.
    Side streams are forked from and joined back into the caller's stream,
    so in a captured CUDA graph they become parallel branches. Kernels only
    share an SM when they request the same shared-memory carveout, so the
    overlapping modes are also tried with one common carveout (100 %); the
    chosen carveout is applied with fst_set_smem_carveout. They are also
    tried with the operator measured slowest on a high-priority stream
    (concurrent mode) or with the fused launch forked before the ABA branch
    (the block scheduler places the first-forked kernel's blocks first, and
    on GB300 the order moves a hybrid step between 14.5 and 22 us)."""

    MODES = ("fused", "hybrid", "split", "pinned", "partitioned", "concurrent", "sequential")

    def __init__(self, model, B, links=None, use_cache=True, verbose=False, modes=MODES, fixed=None):
        """fixed: run this one plan instead of searching, named as the keys of
        describe()["us"] name plans (see parse_key); with the launch
        configurations in brackets, nothing else is tuned either."""
        self.model = model
        self.links = list(links if links is not None else model.ee)
        api.set_smem_carveout(-1)
        fixed = self.parse_key(fixed) if fixed else None
        if fixed and fixed[3] and fixed[0] not in ("concurrent", "sequential"):
            self.tuned = {}                      # the plan names every launch it makes
        else:
            self.tuned = tune(model, B, FORWARD_KINDS + ("eval",), links=self.links, use_cache=use_cache,
                              verbose=verbose)
        self._plain = [torch.cuda.Stream(device=model.device) for _ in FORWARD_KINDS]
        # the first stream forked (the longest operator) at the device's highest
        # priority (out-of-range values clamp to it), the others at the default
        self._ranked = [torch.cuda.Stream(device=model.device, priority=-1000 if k == 0 else 0)
                        for k in range(len(FORWARD_KINDS))]
        if fixed:
            mode, carveout, alt, ev = fixed
            if ev is None:
                ev = "|".join(f"{self.tuned[k]['variant']}/{self.tuned[k]['block']}" for k in ("eval", "aba"))
            cold = ColdSets(model, B, self.links)
            api.set_smem_carveout(carveout)
            self._set_eval(ev)
            self._set_alt(mode, alt)
            self.times = {(mode, carveout, alt, ev): self._time(cold)}
            self._apply(mode, carveout, alt, ev)
            return
        if not autotune_enabled():          # FST_AUTOTUNE=0: one fused launch, nothing timed
            ev = "|".join(f"{self.tuned[k]['variant']}/{self.tuned[k]['block']}" for k in ("eval", "aba"))
            self.times = {("fused", -1, False, ev): None}
            self._apply("fused", -1, False, ev)
            return
        key = _key(model, "plan11", B)      # plans timed on cold, rotating inputs
        hit = _load_cache().get(key) if use_cache else None
        if hit:
            self.times = {(k, c, a, ev): v for k, c, a, ev, v in hit["times"]}
            self._apply(hit["mode"], hit["carveout"], hit["alt"], hit["eval"])
            return
        cold = ColdSets(model, B, self.links)
        # the hybrid's fused kernel carries three roles, not the four the
        # eval tuning measured: try the best few fused configurations there
        ranked = sorted(self.tuned["eval"]["candidates"].items(), key=lambda kv: kv[1])
        best_eval = f"{self.tuned['eval']['variant']}/{self.tuned['eval']['block']}"
        hybrid_evals = [name for name, _ in ranked[:5]]
        # beside the ABA branch, fewer and larger fused blocks can win: every
        # block size of the specialised fused kernel is tried as well
        hybrid_evals += [n for n in (f"specialized/{b}" for b in CANDIDATE_BLOCKS)
                         if n in self.tuned["eval"]["candidates"] and n not in hybrid_evals]
        # and the ABA branch at its three best configurations
        best_aba = f"{self.tuned['aba']['variant']}/{self.tuned['aba']['block']}"
        abas = [n for n, _ in sorted(self.tuned["aba"]["candidates"].items(), key=lambda kv: kv[1])[:3]]
        hybrid_cfgs = [f"{ev}|{ab}" for ev in hybrid_evals for ab in abas]
        # SM-pinned: the whole step in one launch of one block per SM, every SM
        # serving one operator (ABA level-parallel, the others one environment
        # per thread) with the SM counts of the candidates below
        pinned_cfgs = []
        if "specialized" in {c.split("/")[0] for c in self.tuned["eval"]["candidates"]}:
            pinned_cfgs = [f"pinned/256|level/256@{c}" for c in self.pin_count_candidates(B)]
        # SM partitions: the best two fused configurations for the single-role
        # launches, the best ABA configuration, the SM splits below
        part_cfgs = []
        if B <= 16384:
            part_evals = [n for n in hybrid_evals if n.split("/")[0] in ("specialized", "level")][:2]
            part_cfgs = [f"{ev}|{abas[0]}@{c}" for ev in part_evals for c in self.partition_count_candidates(B)]
        times = {}
        for carveout in (-1, 100):
            api.set_smem_carveout(carveout)
            for mode in modes:
                cfgs = {"hybrid": hybrid_cfgs, "split": hybrid_cfgs, "pinned": pinned_cfgs,
                        "partitioned": part_cfgs}.get(
                    mode, [f"{best_eval}|{best_aba}"])
                for ev in cfgs:
                    try:
                        self._set_eval(ev)
                    except _ffi.FstError:
                        continue                 # not available for this model
                    for alt in (False, True):
                        if (carveout >= 0 or alt) and mode in ("fused", "sequential", "pinned", "partitioned"):
                            continue
                        self._set_alt(mode, alt)
                        times[(mode, carveout, alt, ev)] = self._time(cold)
        self.times = times
        self._apply(*min(times, key=times.get))
        if use_cache:
            _store_cache({key: {"mode": self.mode, "carveout": self.carveout, "alt": self.alt,
                                "eval": self.eval_config,
                                "times": [[k, c, p, ev, round(v, 3)] for (k, c, p, ev), v in times.items()]}})

    def _time(self, cold):
        """Microseconds per step of the current plan, each step on the next of
        the rotating cold data sets (as the benchmark's timed steps run)."""
        def step(k):
            d = cold.sets[k]
            self(d["q"], d["qd"], d["qdd"], d["tau"], d["out"])
        return cold_time_us(step, cold.R)

    @classmethod
    def parse_key(cls, key):
        """A plan named as the keys of describe()["us"] name them:
        "<mode>[<eval variant>/<block>|<aba variant>/<block>[@<ABA share>]]
        [@<carveout>%][+fusedfirst | +prio]", the bracketed launch
        configurations optional. Returns (mode, carveout or -1, the binary
        option, the bracketed configuration or None)."""
        m = re.fullmatch(r"([a-z]+)(?:\[([^\]]+)\])?(?:@(\d+)%)?(\+fusedfirst|\+prio)?", key)
        if not m or m.group(1) not in cls.MODES:
            raise ValueError(f"not a step plan: {key!r}")
        mode, ev, carveout, opt = m.groups()
        if opt and opt != ("+prio" if mode == "concurrent" else "+fusedfirst"):
            raise ValueError(f"{opt} is not an option of the {mode} mode")
        if opt and mode in ("fused", "sequential"):
            raise ValueError(f"the {mode} mode has no option")
        if ev is not None and (ev.count("|") != 1 or any(p.count("/") != 1 for p in ev.split("@")[0].split("|"))):
            raise ValueError(f"launch configurations must read <variant>/<block>|<variant>/<block>: {ev!r}")
        carveout = -1 if carveout is None else int(carveout)
        if carveout > 100:
            raise ValueError("carveout above 100 %")
        return mode, carveout, opt is not None, ev

    def _set_eval(self, config):
        """config: "<eval variant>/<block>|<aba variant>/<block>[@<SM counts>]";
        SM counts "a-k-r-c" (ABA, KIN, RNEA, CRBA) set the SM roles of the
        pinned step (eval variant "pinned"), or the SM partitions of the
        partitioned step (any other eval variant)."""
        config, _, counts = config.partition("@")
        for kind, part in zip(("eval", "aba"), config.split("|")):
            variant, block = part.split("/")
            self.model.set_launch([kind], int(block), variant)
        if counts and config.startswith("pinned/"):
            self.model.set_sm_roles(self.pin_roles([int(c) for c in counts.split("-")],
                                                   ids=sm_ids(self.model.device)))
        elif counts:
            self.partition = api.sm_partition([int(c) for c in counts.split("-")], self.model.device)

    def partition_count_candidates(self, B, n_sm=None):
        """SM counts (ABA, KIN, RNEA, CRBA), in groups of 8, for the
        partitioned step: ABA about one SM per two 32-environment tiles (two
        level-parallel tiles fit an SM for trees up to about 14 bodies),
        that less or more one group; the rest split between the other three
        evenly and in proportion to their measured times."""
        n_sm = n_sm or sm_count(self.model.device)
        groups = n_sm // 8
        tiles = -(-B // 32)
        a0 = min(max(1, -(-tiles // 16)), groups - 3)    # ceil(tiles / 2 per SM / 8 SMs per group)
        out = []
        for a in (a0, a0 - 1, a0 + 1):
            rest = groups - a
            if a < 1 or rest < 3:
                continue
            t = [self.tuned[k]["us"] for k in ("jacobian", "rnea", "crba")] if self.tuned else [1.0, 1.0, 1.0]
            for wts in (t, (1.0, 1.0, 1.0)):
                k = [max(1, int(rest * x / sum(wts))) for x in wts]
                while sum(k) < rest:     # the next group to the most loaded operator
                    i = max(range(3), key=lambda j: wts[j] / k[j])
                    k[i] += 1
                while sum(k) > rest:
                    i = min((j for j in range(3) if k[j] > 1), key=lambda j: wts[j] / k[j])
                    k[i] -= 1
                c = "-".join(str(8 * g) for g in [a] + k)
                if c not in out:
                    out.append(c)
        return out

    def pin_count_candidates(self, B, n_sm=None):
        """SM counts (ABA, KIN, RNEA, CRBA) to try for the pinned step: ABA
        gets one SM per 64-environment tile (at most all but 24 SMs); the rest
        is split between the other three in proportion to their measured
        times, evenly, and with KIN and CRBA favoured."""
        n_sm = n_sm or sm_count(self.model.device)
        n_aba = min(-(-B // 64), n_sm - 24)
        out = []
        for a in (n_aba, n_aba - 8):
            rest = n_sm - a
            t = [self.tuned[k]["us"] for k in ("jacobian", "rnea", "crba")]
            for w in (t, (1.0, 1.0, 1.0), (1.0, 0.5, 1.0)):
                k = [max(1, int(rest * x / sum(w))) for x in w]
                k[0] += rest - sum(k)
                out.append(f"{a}-{k[0]}-{k[1]}-{k[2]}")
        return list(dict.fromkeys(out))

    @staticmethod
    def pin_roles(counts, ids=None, n_ids=256):
        """Role names for the SM ids 0 .. n_ids - 1 from SM counts (ABA, KIN,
        RNEA, CRBA): the roles are interleaved along the given SM ids (the
        hardware's, api.sm_ids(); by default 0 .. sum(counts) - 1), each
        spread evenly over them (so over both dies of the GPU); every other
        id gets no role."""
        names = ("aba", "kin", "rnea", "crba")
        total = sum(counts)
        ids = list(range(total)) if ids is None else list(ids)[:total]
        out, acc = ["none"] * n_ids, [0.0] * 4
        for sid in ids:
            for r in range(4):
                acc[r] += counts[r] / total
            r = max(range(4), key=lambda j: acc[j])
            acc[r] -= 1.0
            if sid < n_ids:
                out[sid] = names[r]
        return out

    def _set_alt(self, mode, alt):
        """The plan's binary option: for the concurrent mode, the longest
        operator's stream at high priority; for the modes with an ABA branch,
        the fused launch(es) forked before ABA instead of after it (the block
        scheduler places the first-forked kernel's blocks first)."""
        self.mode, self.alt = mode, bool(alt)
        self.prio = self.alt and mode == "concurrent"
        self.streams = self._ranked if self.prio else self._plain

    def _apply(self, mode, carveout, alt, eval_config):
        self.carveout, self.eval_config = carveout, eval_config
        self._set_alt(mode, alt)
        self._set_eval(eval_config)
        api.set_smem_carveout(carveout)
        self.fused = mode == "fused"
        self.expected_us = self.times[(mode, carveout, self.alt, eval_config)]

    def _ops(self, q, qd, qdd, tau, out):
        m = self.model
        return (lambda: api.fk(m, q, out=out["poses"]),
                lambda: api.jacobian(m, q, self.links, out=out["J"]),
                lambda: api.rnea(m, q, qd, qdd, out=out["tau"]),
                lambda: api.crba(m, q, out=out["M"]),
                lambda: api.aba(m, q, qd, tau, out=out["qdd"]))

    def _fork(self, fns, streams=None):
        streams = self.streams if streams is None else streams
        cur = torch.cuda.current_stream(self.model.device)
        for st, fn in zip(streams, fns):
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                fn()
        for st in streams[:len(fns)]:
            cur.wait_stream(st)

    def __call__(self, q, qd, qdd, tau, out, packed=False):
        """One step into `out`. packed=True writes M and J in the packed
        layouts of eval(packed=True); only the modes that compute M and J in
        fused launches (fused, hybrid, split, pinned, partitioned) have them."""
        m = self.model
        if packed and self.mode in ("sequential", "concurrent"):
            raise ValueError(f"the {self.mode} step plan has no packed outputs")
        if self.mode == "fused":
            return api.eval(m, q, qd, qdd, tau, fk=True, links=self.links, rnea=True, crba=True, aba=True, out=out,
                            packed=packed)
        ops = self._ops(q, qd, qdd, tau, out)
        if self.mode == "sequential":
            for op in ops:
                op()
        elif self.mode == "pinned":
            # the SM-pinned step: all five operators in one launch
            api.eval(m, q, qd, qdd, tau, fk=True, links=self.links, rnea=True, crba=True, aba=True, out=out,
                     packed=packed)
        elif self.mode == "partitioned":
            # ABA, the kinematics, RNEA and CRBA each on its own SMs
            self._fork([ops[4],
                        lambda: api.eval(m, q, qd, qdd, tau, fk=True, links=self.links, out=out, packed=packed),
                        lambda: api.eval(m, q, qd, qdd, tau, fk=False, rnea=True, out=out, packed=packed),
                        lambda: api.eval(m, q, qd, qdd, tau, fk=False, crba=True, out=out, packed=packed)],
                       streams=self.partition.streams)
        elif self.mode == "hybrid":
            fused = [lambda: api.eval(m, q, qd, qdd, tau, fk=True, links=self.links, rnea=True, crba=True, aba=False,
                                      out=out, packed=packed)]
            self._fork(fused + [ops[4]] if self.alt else [ops[4]] + fused)
        elif self.mode == "split":
            # ABA beside the fused kernel twice: kinematics alone, RNEA with CRBA
            fused = [lambda: api.eval(m, q, qd, qdd, tau, fk=True, links=self.links, out=out, packed=packed),
                     lambda: api.eval(m, q, qd, qdd, tau, fk=False, rnea=True, crba=True, out=out, packed=packed)]
            self._fork(fused + [ops[4]] if self.alt else [ops[4]] + fused)
        else:
            # longest first, so its blocks are dispatched first
            order = sorted(range(len(ops)), key=lambda k: -(self.tuned[FORWARD_KINDS[k]]["us"] or 0.0))
            self._fork([ops[k] for k in order])
        return out

    def describe(self):
        kinds = {k: f"{v['variant']}/{v['block']}" for k, v in self.tuned.items()}
        kinds["eval"], kinds["aba"] = self.eval_config.split("|")
        return {"mode": self.mode, "carveout": self.carveout, "priorities": self.prio,
                "fused_forked_first": self.alt and self.mode != "concurrent",
                "us": {f"{k[0]}{'[' + k[3] + ']' if k[0] in ('hybrid', 'split', 'pinned', 'partitioned') else ''}"
                       f"{'' if k[1] < 0 else f'@{k[1]}%'}"
                       f"{('+prio' if k[0] == 'concurrent' else '+fusedfirst') if k[2] else ''}": None if v is None else round(v, 3)
                       for k, v in self.times.items()},
                "kinds": kinds,
                "eval_candidates_us": self.tuned.get("eval", {}).get("candidates", {})}
