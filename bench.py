#!/usr/bin/env python3
"""Throughput of the batched rigid-body dynamics hot path on GB300.

Workload: the branched 11-DOF spined-quadruped tree (3-joint spine on a
fixed base, rear leg pair off the first spine link, front pair off the last;
depth 5), seeded random inertias, B = 4096 environments. One step = one pass
of every operator over the batch: FK of all bodies, the four foot Jacobians,
RNEA, CRBA and ABA.

Metric: env-evals/s = environments x steps / device time (higher is
better). Inputs and outputs rotate over enough replica sets (> 2x the
129 MB L2) that every step reads and writes HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fst|reference]

Under torchrun every rank runs an independent replica of the workload on its
own GPU (environments are independent; there is no collective on the data
path); rank 0 prints one JSON line with the whole-job throughput.
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import ctypes
import json
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-evals/s for FK/Jac/RNEA/CRBA/ABA @4096 envs; RNEA fwd+bwd/s vs plain"
L2_BYTES = 129 * 2 ** 20
FP32_LANES_PER_SM, N_SM = 128, 152
OPS = ("fk", "jacobian", "rnea", "crba", "aba")


# DRAM bytes (read + write) per step of the timed kernels, from one ncu
# capture of each (the step's summary under profiles/), keyed by the step
# plan and a hash of the kernel sources at capture time: a source change
# since the capture makes the entry stale and the reported traffic null.
NCU_TRAFFIC = {
    ("hybrid", "levellean/128", "specialized/128", "15950e7be32c"): 782520 + 594817,
}


# The sources the two kernels of the hybrid step are built from (the
# specialised fused kernel: the JIT headers and their generator; the
# level-parallel ABA: level.cu and the headers it includes; the model
# constants both read). Host-only files of the C ABI are left out.
STEP_KERNEL_SOURCES = ("fst_layout.h", "fst_device.cuh", "ops.cuh", "adjoint.cuh", "derivs.cuh", "level.cuh",
                       "pathpar.cuh", "jit_kernels.cuh", "jit.cpp", "jit.h", "level.cu", "launch.h", "model.cpp",
                       "fst_internal.h")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2605_31481_gb300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "src": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "src": "fallback"}


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x clock
    return N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def roof_of(bytes_, flops_, seconds, p_alu_tflops, hbm_gbs):
    """Roofline position of one launch (or step): algorithmic bytes and
    flops, their rates and the fraction of each ceiling; `bound` is the
    ceiling the algorithmic cost hits first (the larger time), `frac` the
    fraction of that one."""
    t_hbm, t_alu = bytes_ / (hbm_gbs * 1e9), flops_ / (p_alu_tflops * 1e12)
    hf, af = t_hbm / seconds, t_alu / seconds
    return {"bytes": int(bytes_), "flops": int(flops_), "us": round(seconds * 1e6, 3),
            "gbs": round(bytes_ / seconds / 1e9, 1), "tflops": round(flops_ / seconds / 1e12, 3),
            "hbm_frac": round(hf, 4), "alu_frac": round(af, 4), "bound": "hbm" if t_hbm >= t_alu else "alu",
            "frac": round(max(hf, af), 4)}


def measure_fp32_peak(torch, gpu_index, launches=12, iters=1 << 19):
    """FP32 FMA throughput of this GPU, measured: the library's FMA probe
    (fst_fp32_probe: 4 blocks of 256 threads per SM, 16 independent chains
    per thread) launched back to back for about half a second, each launch
    timed with CUDA events on the launching stream, with nvidia-smi clocks
    sampled over the same interval. Returns the best launch's TFLOP/s (a
    burst figure, like the measured copy bandwidth), the median, and the
    clocks seen."""
    from paper_2605_31481_gb300 import api
    fl, buf = api.fp32_probe(4, 1 << 10)          # first launch: module load, not timed
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clk = ClockSampler(gpu_index)
    clk.start()
    time.sleep(0.15)
    clk.mark("soak")
    clk.mark("t0")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(launches + 1)]
    ev[0].record(stream)
    for k in range(launches):
        fl, buf = api.fp32_probe(4, iters, out=buf)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clk.mark("t1")
    clocks = clk.stop()
    tf = [fl / (ev[k].elapsed_time(ev[k + 1]) / 1e3) / 1e12 for k in range(launches)]
    return {"tflops": round(max(tf), 2), "tflops_median": round(statistics.median(tf), 2),
            "launch_ms": round(ev[0].elapsed_time(ev[-1]) / launches, 3), "clocks": clocks,
            "derived_at_max_clock": round(fp32_peak_tflops(2070.0), 2),
            "how": "fst_fp32_probe: SMs x 4 blocks x 256 threads x 16 FMA chains, best of "
                   f"{launches} launches of {iters} iterations (CUDA events)"}


def workload():
    from paper_2605_31481_gb300 import workloads as w
    tree = w.spined_quadruped(seed=0)
    return tree, 4096, list(tree.ee)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class NvmlPoller:
    """SM clock and clock-event reasons read through NVML (libnvidia-ml,
    through ctypes: read-only queries) from a host thread every ~0.2 ms, so
    that a timed region far shorter than nvidia-smi's sampling period still
    holds samples. The reason bits are NVML's public clock-event reason
    masks."""
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, torch_device_index):
        import ctypes
        import threading
        self.rows, self.ok, self._stop = [], False, threading.Event()
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            self.dev = ctypes.c_void_p()
            uuid = None
            try:
                import torch
                uuid = "GPU-" + str(torch.cuda.get_device_properties(torch_device_index).uuid)
            except Exception:
                uuid = None
            rc = 1
            if uuid:
                rc = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.dev))
            if rc != 0:
                rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(torch_device_index), ctypes.byref(self.dev))
            if rc != 0:
                return
            self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.ct = ctypes
            self.ok = True
        except (OSError, AttributeError):
            self.ok = False
        self.thread = threading.Thread(target=self._run, daemon=True) if self.ok else None

    def _read(self):
        ct = self.ct
        mhz, mx, rs = ct.c_uint(0), ct.c_uint(0), ct.c_ulonglong(0)
        if self.lib.nvmlDeviceGetClockInfo(self.dev, 1, ct.byref(mhz)) != 0:      # NVML_CLOCK_SM
            return None
        self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, ct.byref(mx))
        self.reasons_fn(self.dev, ct.byref(rs))
        return (time.time(), float(mhz.value), float(mx.value), None,
                [bool(rs.value & self.BITS[n]) for n in ClockSampler.NAMES])

    def _run(self):
        while not self._stop.is_set():
            r = self._read()
            if r is not None:
                self.rows.append(r)
            time.sleep(0.0002)

    def start(self):
        if self.thread is not None:
            self.thread.start()

    def stop(self):
        if self.thread is not None:
            self._stop.set()
            self.thread.join(timeout=5)
            self.lib.nvmlShutdown()
        return self.rows


class ClockSampler:
    """nvidia-smi samples (100 ms period) of SM clock and throttle reasons,
    plus NVML reads every ~0.2 ms (NvmlPoller); stats are taken over the
    samples whose timestamps fall in the timed region (or, if none does,
    over the samples of the loaded soak just before it, flagged
    in_region=false)."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.marks = {}
        self.nvml = NvmlPoller(gpu_index)

    def start(self):
        self.nvml.start()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def mark(self, name):
        self.marks[name] = time.time()

    def read_now(self):
        """One NVML read from the calling thread, stamped now: called while
        the timed work runs on the device (after it was enqueued, before the
        host waits for it) and right after it, so that a timed region shorter
        than the polling period still holds samples."""
        if self.nvml.ok:
            r = self.nvml._read()
            if r is not None:
                self.nvml.rows.append(r)

    def stop(self):
        nv_rows = self.nvml.stop()
        if self.proc is None and not nv_rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
        import datetime
        rows = list(nv_rows)
        for line in out.strip().splitlines():
            r = [x.strip() for x in line.split(",")]
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(r[1]), float(r[2]), float(r[3]), [v.lower() == "active" for v in r[4:8]]))
            except (ValueError, IndexError):
                continue

        def stats(lo, hi):
            sel = [x for x in rows if lo <= x[0] <= hi]
            if not sel:
                return None
            reasons = sorted({n for x in sel for n, a in zip(self.NAMES, x[4]) if a})
            pw = [x[3] for x in sel if x[3] is not None]
            return {"sm_mhz": statistics.median(x[1] for x in sel), "sm_max_mhz": max(x[2] for x in sel),
                    "power_w_median": statistics.median(pw) if pw else None, "reasons": reasons,
                    "samples": len(sel), "nvml_samples": sum(1 for x in sel if x[3] is None)}

        st = stats(self.marks.get("t0", 0), self.marks.get("t1", 0))
        if st is not None:
            st["in_region"] = True
            return st
        st = stats(self.marks.get("soak", 0), self.marks.get("t1", 0))
        if st is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "in_region": False}
        st["in_region"] = False
        return st


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def plan_kernel_name(mode, desc):
    """What the timed step launches under a step plan, from the plan's
    describe() (launch configurations of the kinds it sets)."""
    kinds, carveout = desc["kinds"], desc["carveout"]
    if mode == "fused":
        if kinds["eval"].startswith("mixed"):
            lv = [k for k in ("aba", "crba", "rnea")
                  if kinds.get(k, "").split("/")[0] in ("level", "level2", "levellean")]
            return (f"fused eval kernel ({kinds['eval']}: " + (", ".join(lv) + " level-parallel, " if lv else "") +
                    "the other roles one environment per thread)")
        return f"fused eval kernel ({kinds['eval']})"
    if mode == "hybrid":
        return (f"ABA kernel ({kinds['aba']}) on a parallel graph branch beside the fused kernel of the other four "
                f"({kinds['eval']}), carveout {carveout}" + (", fused kernel forked first" if desc["fused_forked_first"] else ""))
    if mode == "concurrent":
        return ("5 per-operator kernels on parallel graph branches (" +
                ", ".join(f"{k} {kinds.get(k, 'default')}" for k in OPS) + f"), carveout {carveout}" +
                (", longest operator on a high-priority stream" if desc["priorities"] else ""))
    if mode == "split":
        return (f"ABA kernel ({kinds['aba']}) beside two launches of the fused kernel ({kinds['eval']}: FK with the "
                f"Jacobians; RNEA with CRBA) on parallel graph branches, carveout {carveout}" +
                (", fused kernels forked first" if desc["fused_forked_first"] else ""))
    if mode == "partitioned":
        return (f"ABA kernel ({kinds['aba']}), and the fused kernel ({kinds['eval']}) once per operator group (FK with "
                f"the Jacobians; RNEA; CRBA), each on its own SM partition (green contexts; SM counts ABA-KIN-RNEA-CRBA "
                f"after the @), carveout {carveout}")
    if mode == "pinned":
        return (f"SM-pinned step ({kinds['eval']}): one launch of one block per SM, each SM serving one operator; "
                f"ABA level-parallel ({kinds['aba']}: SM counts ABA-KIN-RNEA-CRBA after the @), the others one "
                f"environment per thread")
    return "5 per-operator kernels in sequence"


def job_rate(ms, world, envs_per_rank, steps, device):
    """Whole-job throughput of `world` replicas: the slowest rank's time (the
    maximum over ranks of `ms`, in milliseconds, for `steps` steps of
    `envs_per_rank` environments each) and the env-evals/s of all ranks
    together over that time. Every rank must call it when world > 1."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return ms, world * envs_per_rank * steps / (ms / 1e3)


def run_fst(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2605_31481_gb300 import _ffi, costs
    from paper_2605_31481_gb300 import workloads as w
    import paper_2605_31481_gb300 as fst

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        # one rank builds the in-tree library, the others wait for it
        if rank == 0:
            __graft_entry__.build()
        dist.barrier()
        if rank != 0:
            __graft_entry__.build()          # up to date by now: only imports
    else:
        __graft_entry__.build()
    L = _ffi.lib()

    tree, B, links = workload()
    model = fst.Model(tree)
    if world > 1 and rank != 0:
        dist.barrier()                  # rank 0 compiles first and fills the on-disk cache
    try:
        model.specialize()
        kernels = "specialized available"
    except _ffi.FstError as exc:        # no NVRTC on this host: generic kernels only
        kernels = f"generic only ({exc})"
    if world > 1 and rank == 0:
        dist.barrier()
    from paper_2605_31481_gb300.autotune import StepPlan
    plan = StepPlan(model, B, links=links, fixed=args.plan)
    nq, nv, nb, nl = tree.nq, tree.nv, tree.n_bodies, len(links)
    out_floats = nb * 12 + nl * 6 * nv + nv + nv * nv + nv
    in_floats = nq + 3 * nv
    set_bytes = 4 * B * (in_floats + out_floats)
    R = max(2, int(np.ceil(2 * L2_BYTES / set_bytes)) + 1)
    st = w.random_state(tree, B * R, seed=1 + 1000 * rank)
    dev = torch.device("cuda", local)

    def soa(x, r):
        return torch.from_numpy(np.ascontiguousarray(x[r * B:(r + 1) * B].T.astype(np.float32))).to(dev)

    sets = []
    for r in range(R):
        d = {k: soa(st[k], r) for k in ("q", "qd", "qdd", "tau")}
        d["out"] = {"poses": torch.empty((nb, 12, B), device=dev), "J": torch.empty((nl, 6, nv, B), device=dev),
                    "tau": torch.empty((nv, B), device=dev), "M": torch.empty((nv, nv, B), device=dev),
                    "qdd": torch.empty((nv, B), device=dev)}
        sets.append(d)
    stream = torch.cuda.current_stream()

    def launch(op, d):
        """One operator alone (its own kernel), for the per-operator numbers."""
        o = d["out"]
        if op == "fk":
            fst.fk(model, d["q"], out=o["poses"])
        elif op == "jacobian":
            fst.jacobian(model, d["q"], links, out=o["J"])
        elif op == "rnea":
            fst.rnea(model, d["q"], d["qd"], d["qdd"], out=o["tau"])
        elif op == "crba":
            fst.crba(model, d["q"], out=o["M"])
        else:
            fst.aba(model, d["q"], d["qd"], d["tau"], out=o["qdd"])

    def step(k):
        """One pass of all five operators over the batch (fused or in
        sequence, as the autotuner measured faster)."""
        d = sets[k % R]
        plan(d["q"], d["qd"], d["qdd"], d["tau"], d["out"])

    # the step's outputs on the first input set, checked against the oracle
    # in the CPU-baseline leg below
    step(0)
    torch.cuda.synchronize()
    first = {k: v.detach().cpu().numpy().astype(np.float64) for k, v in sets[0]["out"].items()}

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    K = args.steps
    # The timed loop replays CUDA graphs: one graph of R steps (one per
    # rotating input/output set) K // R times, then one graph of the
    # remaining K mod R steps, so exactly K steps run back to back with no
    # host launch gap between them whatever K is.
    def capture(ks):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for k in ks:
                step(k)
        return g

    g_all = capture(range(R))
    g_rem = capture(range(K % R)) if K % R else None
    for _ in range(3):
        g_all.replay()
        if g_rem is not None:      # the first replay of a graph uploads it: keep that out of the timed region
            g_rem.replay()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.15)
    # loaded soak (untimed) so the clocks are at their loaded state
    clk.mark("soak")
    t_soak = time.time()
    while time.time() - t_soak < 0.5:
        for _ in range(20):
            g_all.replay()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.mark("t0")
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(K // R):
        g_all.replay()
    if g_rem is not None:
        g_rem.replay()
    t_end.record(stream)
    clk.read_now()             # the step graphs are running on the device
    torch.cuda.synchronize()
    clk.read_now()
    clk.mark("t1")
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = t_start.elapsed_time(t_end)
    kernel_ms = ms / K          # the step's kernel(s), back to back inside the graphs
    per_op_ms = per_op_times(torch, launch, sets, R, stream, K_op=min(K, 3000))
    per_op_hot_ms = per_op_times(torch, launch, sets, R, stream, K_op=min(K, 3000), hot=True)

    ms, value = job_rate(ms, world, B, K, dev)

    # end to end through the public binding, host buffers in and out
    # the packed layouts where the plan computes M and J in fused launches
    packed = plan.mode not in ("sequential", "concurrent")
    e2e = run_e2e(torch, fst, model, tree, B, links, st, dev, min(K, 5000), args.warmup, plan=plan,
                  slots=args.e2e_slots, split=args.e2e_split, packed=packed)
    e2e["ms"], e2e_value = job_rate(e2e["ms"], world, B, e2e["steps"], dev)
    link = link_bandwidth(torch, dev)
    # the end-to-end step against the link: its bytes in each direction per
    # second of step time, over the measured one-way copy bandwidths
    e2e_s = e2e["ms"] / e2e["steps"] / 1e3
    link["d2h_frac"] = round(e2e["d2h"] / e2e_s / 1e9 / link["d2h_gbs"], 4)
    link["h2d_frac"] = round(e2e["h2d"] / e2e_s / 1e9 / link["h2d_gbs"], 4)
    e2e_full = run_e2e(torch, fst, model, tree, B, links, st, dev, min(K, 5000), args.warmup, plan=plan,
                       slots=args.e2e_slots, split=args.e2e_split, packed=False)
    e2e_full["ms"], e2e_full_value = job_rate(e2e_full["ms"], world, B, e2e_full["steps"], dev)

    pk = peaks()
    fp32 = measure_fp32_peak(torch, local)
    p_alu = fp32["tflops"]
    fl = sum(costs.flops(tree, op, links=links if op == "jacobian" else ()) for op in OPS)
    by = 4 * (in_floats + out_floats)
    t_k = kernel_ms / 1e3
    bound = "alu" if fl / (p_alu * 1e12) > by / (pk["hbm_gbs"] * 1e9) else "hbm"
    desc = plan.describe()
    kname = plan_kernel_name(plan.mode, desc)
    traffic = args.traffic
    if traffic is None:
        traffic = NCU_TRAFFIC.get((plan.mode, desc["kinds"]["aba"], desc["kinds"]["eval"], kernel_source_hash()))
    common = {"kernel": kname, "traffic": traffic,
              "algorithmic_bytes_per_launch": by * B, "algorithmic_flops_per_launch": fl * B,
              "kernel_ms": round(kernel_ms, 5),
              "alu_frac": round(fl * B / t_k / 1e12 / p_alu, 5),
              "hbm_frac": round(by * B / t_k / 1e9 / pk["hbm_gbs"], 5),
              "alu_peak_src": f"measured: FP32 FMA probe {p_alu:.1f} TFLOP/s (burst) at SM clock "
                              f"{fp32['clocks'].get('sm_mhz')} MHz",
              "hbm_peak_src": f"{pk['src']} copy bandwidth {pk['hbm_gbs']} GB/s"}
    if bound == "alu":
        achieved = fl * B / t_k / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(p_alu, 2), "unit": "TFLOP/s",
                "frac": round(achieved / p_alu, 5), **common}
    else:
        achieved = by * B / t_k / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / pk["hbm_gbs"], 5), **common}

    extras = {}
    if rank == 0 and not args.no_extras:
        extras["rnea_fwd_bwd"] = rnea_fwd_bwd(torch, fst, w)
        extras["rl_step_graph"] = rl_step(torch, fst, w)
        extras["humanoid_sweep"] = humanoid_sweep(torch, fst, w, p_alu, pk["hbm_gbs"])
        extras["chain7_b1024"] = chain7_small(torch, fst, w, p_alu, pk["hbm_gbs"])
        extras["multi_tree"] = multi_tree(torch, fst, w)
        extras["sysid"] = sysid(torch, fst, w)
    if rank == 0:
        if args.no_cpu_baseline:
            cpu1 = parity = parity_detail = cpu = None
        else:
            cpu1, parity, parity_detail = cpu_baseline(tree, links, args, st, first)
            cpu = cpu_baseline_all_cores()
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "env-evals/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms / K, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{tree.name}: 11 revolute DOF branched tree, depth 5, B=4096 per GPU",
                       "B": B, "step": "+".join(OPS) + " (4 foot Jacobians)",
                       "l2": f"inputs/outputs rotate over {R} sets of {set_bytes / 2**20:.1f} MiB (> 2x L2)",
                       "parallelism": f"replicas x{world}",
                       "seeds": {"model": 0, "inputs": "1 + 1000 x rank"}},
            "per_op_ms": {k: round(v, 5) for k, v in per_op_ms.items()},
            "per_op_hot_ms": {k: round(v, 5) for k, v in per_op_hot_ms.items()},
            "per_op_env_evals_per_s": {k: round(B / (v / 1e3), 1) for k, v in per_op_ms.items()},
            "per_op_roofline": {k: roof_of(B * costs.io_bytes(tree, k, len(links)),
                                           B * costs.flops(tree, k, links=links if k == "jacobian" else ()),
                                           v / 1e3, p_alu, pk["hbm_gbs"]) for k, v in per_op_ms.items()},
            "fp32_peak": fp32,
            "roofline": roof,
            "e2e": {"value": round(e2e_value, 1), "unit": "env-evals/s", "h2d_bytes_per_step": e2e["h2d"],
                    "d2h_bytes_per_step": e2e["d2h"], "steps": e2e["steps"],
                    "pipelined_slots": e2e["slots"], "readback_chunks": e2e["readback_chunks"],
                    "output_layout": e2e["layout"], "link": link},
            "e2e_full_layout": {"value": round(e2e_full_value, 1), "unit": "env-evals/s",
                                "h2d_bytes_per_step": e2e_full["h2d"], "d2h_bytes_per_step": e2e_full["d2h"],
                                "steps": e2e_full["steps"]},
            "gpu_launches": K * {"fused": 1, "hybrid": 2, "split": 3, "pinned": 1, "partitioned": 4}.get(plan.mode,
                                                                                                  len(OPS)),
            "kernels": kernels,
            "plan": desc,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "cpu_baseline_1core": cpu1,
            "parity_vs_oracle": parity,
            "parity_detail": parity_detail,
            **extras,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def _graph_us(torch, fn, n=20, reps=10):
    from paper_2605_31481_gb300.autotune import graph_time_us
    return graph_time_us(fn, n=n, reps=reps)


def rnea_fwd_bwd(torch, fst, w):
    """RNEA forward + backward on the 7-DOF chain, B = 8192: the sysid loss
    sum (RNEA - tau_meas)^2 and its gradient in one fused kernel, against the
    plain sequence (RNEA kernel, the residual as a torch op, the RNEA adjoint
    kernel, which recomputes the forward sweep) and against the store
    variant of that sequence (the RNEA kernel writes its forward state to a
    tape that the adjoint kernel reads). All graph-replayed."""
    tree = w.chain(7, seed=0)
    B = 8192
    m = fst.Model(tree)
    try:
        m.specialize(["rnea", "rnea_vjp", "loss_grad", "rnea_store", "rnea_vjp_stored"])
    except Exception:
        pass
    s = w.random_state(tree, B, seed=1)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x.T.astype(np.float32))).cuda()
    q, qd, qdd, tm = cu(s["q"]), cu(s["qd"]), cu(s["qdd"]), cu(s["tau"])
    from paper_2605_31481_gb300 import autotune
    autotune.tune(m, B, kinds=("rnea", "rnea_vjp", "loss_grad", "rnea_store", "rnea_vjp_stored"), use_cache=False)
    tape = fst.api.rnea_tape(m, B)
    scratch = fst.api.adjoint_scratch(m, B)
    tau = torch.empty_like(tm)
    buf = torch.empty(tree.n_bodies * 10 + 1, device="cuda")

    def fused():
        fst.api.rnea_loss_grad(m, q, qd, qdd, tm, q_bar=False, scratch=scratch, out=buf)

    def plain():
        fst.rnea(m, q, qd, qdd, out=tau)
        tb = 2.0 * (tau - tm)
        fst.api.rnea_vjp(m, q, qd, qdd, tb, q_bar=False, qd_bar=False, qdd_bar=False, scratch=scratch)

    def stored():
        fst.api.rnea_store(m, q, qd, qdd, tape=tape, out=tau)
        tb = 2.0 * (tau - tm)
        fst.api.rnea_vjp_stored(m, q, qd, tape, tb, q_bar=False, qd_bar=False, qdd_bar=False, scratch=scratch)

    tf, tp, ts = _graph_us(torch, fused), _graph_us(torch, plain), _graph_us(torch, stored)
    return {"workload": "chain7, B=8192, loss sum (RNEA - tau_meas)^2 and d/dtheta",
            "fused_us": round(tf, 3), "plain_us": round(tp, 3), "plain_store_us": round(ts, 3),
            "fused_per_s": round(B / tf * 1e6, 1), "plain_per_s": round(B / tp * 1e6, 1),
            "plain_store_per_s": round(B / ts * 1e6, 1),
            "speedup": round(tp / tf, 3), "store_vs_recompute": round(tp / ts, 3),
            "tape_bytes": tape.numel() * 4, "unit": "RNEA fwd+bwd env-evals/s"}


def rl_step(torch, fst, w, steps=1000):
    """One RL-style controller step on the 11-DOF tree, B = 4096: FK, the four
    foot Jacobians, RNEA and the RNEA adjoint (cotangent tau), run eagerly
    through the binding as four launches and replayed from one captured CUDA
    graph; then the same step as ONE fused launch (fst_eval with the RNEA
    adjoint), with the kinematics in blocks of their own beside the
    RNEA+adjoint blocks, and with everything fed by one forward sweep."""
    tree = w.spined_quadruped(seed=0)
    B = 4096
    m = fst.Model(tree)
    try:
        m.specialize(["fk", "jacobian", "rnea", "rnea_vjp", "eval"])
    except Exception:
        pass
    from paper_2605_31481_gb300 import autotune
    autotune.tune(m, B, kinds=("fk", "jacobian", "rnea", "rnea_vjp"), use_cache=False)
    s = w.random_state(tree, B, seed=2)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x.T.astype(np.float32))).cuda()
    q, qd, qdd = cu(s["q"]), cu(s["qd"]), cu(s["qdd"])
    poses = torch.empty(tree.n_bodies, 12, B, device="cuda")
    J = torch.empty(4, 6, tree.nv, B, device="cuda")
    tau = torch.empty(tree.nv, B, device="cuda")
    scratch = fst.api.adjoint_scratch(m, B)

    def step():
        fst.fk(m, q, out=poses)
        fst.jacobian(m, q, tree.ee, out=J)
        fst.rnea(m, q, qd, qdd, out=tau)
        fst.api.rnea_vjp(m, q, qd, qdd, tau, qdd_bar=False, theta_bar=False, scratch=scratch)

    for _ in range(5):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step()
    b.record()
    torch.cuda.synchronize()
    eager = a.elapsed_time(b) * 1e3 / steps
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    g.replay()
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    graph = a.elapsed_time(b) * 1e3 / steps
    qb, qdb = torch.empty(tree.nq, B, device="cuda"), torch.empty(tree.nv, B, device="cuda")
    fused = {}
    for one_sweep in (False, True):
        fo = {"poses": poses, "J": J, "tau": tau, "q_bar": qb, "qd_bar": qdb}

        def fstep():
            fst.api.eval(m, q, qd, qdd, fk=True, links=tree.ee, rnea=True, q_bar=True, qd_bar=True, tau_bar="tau",
                         one_sweep=one_sweep, out=fo)

        best = {}
        for blk in (32, 64, 128, 256):          # the fused launch's block size, tuned here
            m.set_launch(["eval"], blk, "auto")
            best[blk] = _graph_us(torch, fstep, n=steps // 10, reps=10)
        blk = min(best, key=best.get)
        fused["one_sweep" if one_sweep else "kin_beside"] = {"graph_us_per_step": round(best[blk], 3), "block": blk,
                                                             "speedup_vs_4_launch_graph": round(graph / best[blk], 3)}
    return {"workload": "spined_quadruped11, B=4096: FK + 4 foot Jacobians + RNEA + RNEA adjoint", "steps": steps,
            "eager_us_per_step": round(eager, 3), "graph_us_per_step": round(graph, 3),
            "graph_steps_per_s": round(1e6 / graph, 1), "speedup": round(eager / graph, 3),
            "fused_one_launch": fused}


def chain7_small(torch, fst, w, p_alu, hbm_gbs, B=1024):
    """The plain method on the 7-DOF serial chain, B = 1024: FK of all links,
    the end-effector Jacobian, RNEA and CRBA in one fused launch (the tuned
    kernel configuration), graph-replayed over rotating input sets larger
    than L2. Env-evals/s and the roofline of the step."""
    from paper_2605_31481_gb300 import autotune, costs
    tree = w.chain(7, seed=0)
    m = fst.Model(tree)
    try:
        m.specialize(["fk", "jacobian", "rnea", "crba", "eval"])
    except Exception:
        pass
    autotune.tune(m, B, kinds=("eval",), links=[tree.n_bodies - 1], use_cache=False)
    links = [tree.n_bodies - 1]
    per_set = 4 * B * (tree.nq + 2 * tree.nv + 12 * tree.n_bodies + 6 * tree.nv + tree.nv + tree.nv ** 2)
    R = int(np.ceil(2 * L2_BYTES / per_set)) + 1
    st = w.random_state(tree, B * R, seed=1)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x.T.astype(np.float32))).cuda()
    sets = [{k: cu(st[k][r * B:(r + 1) * B]) for k in ("q", "qd", "qdd")} for r in range(R)]
    outs = [{"poses": torch.empty(tree.n_bodies, 12, B, device="cuda"), "J": torch.empty(1, 6, tree.nv, B, device="cuda"),
             "tau": torch.empty(tree.nv, B, device="cuda"), "M": torch.empty(tree.nv, tree.nv, B, device="cuda")}
            for _ in range(R)]
    k = [0]

    def step():
        d, o = sets[k[0] % R], outs[k[0] % R]
        k[0] += 1
        fst.eval(m, d["q"], d["qd"], d["qdd"], fk=True, links=links, rnea=True, crba=True, out=o)

    us = _graph_us(torch, step, n=R, reps=20)
    ops = ("fk", "jacobian", "rnea", "crba")
    by = B * sum(costs.io_bytes(tree, op, 1) for op in ops) - 3 * B * 4 * tree.nq   # q read once
    fl = B * sum(costs.flops(tree, op, links=links if op == "jacobian" else ()) for op in ops)
    return {"workload": "chain7 (7 revolute DOF serial chain), B=1024: FK + end-effector Jacobian + RNEA + CRBA, "
                        f"one fused launch, inputs rotating over {R} sets (> 2x L2)",
            "us": round(us, 3), "env_evals_per_s": round(B / us * 1e6, 1),
            "roofline": roof_of(by, fl, us / 1e6, p_alu, hbm_gbs)}


def humanoid_sweep(torch, fst, w, p_alu, hbm_gbs, Bs=(1, 64, 1024, 4096, 16384, 65536)):
    """The five operators on the floating-base 29-DOF humanoid across batch
    sizes (tuned plan per B), env-evals/s of the whole step and its roofline
    position (algorithmic bytes with q, qd, qdd and tau read once)."""
    from paper_2605_31481_gb300 import costs
    tree = w.humanoid(seed=0)
    m = fst.Model(tree)
    try:
        m.specialize(["fk", "jacobian", "rnea", "crba", "aba", "eval"])
    except Exception:
        pass
    from paper_2605_31481_gb300.autotune import StepPlan
    out = {}
    for B in Bs:
        s = w.random_state(tree, B, seed=1)
        cu = lambda x: torch.from_numpy(np.ascontiguousarray(x.T.astype(np.float32))).cuda()
        q, qd, qdd, tau = cu(s["q"]), cu(s["qd"]), cu(s["qdd"]), cu(s["tau"])
        plan = StepPlan(m, B, links=tree.ee)
        o = {"poses": torch.empty(tree.n_bodies, 12, B, device="cuda"),
             "J": torch.empty(len(tree.ee), 6, tree.nv, B, device="cuda"), "tau": torch.empty(tree.nv, B, device="cuda"),
             "M": torch.empty(tree.nv, tree.nv, B, device="cuda"), "qdd": torch.empty(tree.nv, B, device="cuda")}
        us = _graph_us(torch, lambda: plan(q, qd, qdd, tau, o))
        links = list(tree.ee)
        by = B * 4 * (tree.nq + 3 * tree.nv + 12 * tree.n_bodies + 6 * tree.nv * len(links) + tree.nv
                      + tree.nv ** 2 + tree.nv)
        fl = B * sum(costs.flops(tree, op, links=links if op == "jacobian" else ()) for op in OPS)
        tuned = getattr(plan, "tuned", None) or {}
        out[str(B)] = {"us": round(us, 3), "env_evals_per_s": round(B / us * 1e6, 1), "plan": plan.mode,
                       "roofline": roof_of(by, fl, us / 1e6, p_alu, hbm_gbs),
                       # each operator's tuned launch and its time alone (µs, graph replay)
                       "ops": {k: f"{v['variant']}/{v['block']} {v['us']}" for k, v in tuned.items()
                               if k in OPS}}
    return {"workload": "humanoid_float29 (free base + 23 revolute, depth 7): FK + 4 Jacobians + RNEA + CRBA + ABA",
            "per_B": out}


def multi_tree(torch, fst, w, counts=(4096, 2048, 1024, 512, 256)):
    """Mixed batch of five trees (7, 11, 12, 18, 23 revolute DOF; 7936
    environments): FK + RNEA + CRBA + ABA of every tree in one persistent
    launch, against one launch per tree and operator (generic kernels both
    ways). Graph-replayed."""
    trees = w.mixed_trees()
    models = [fst.Model(t) for t in trees]
    items, outs = [], []
    for k, (t, B) in enumerate(zip(trees, counts)):
        s = w.random_state(t, B, seed=20 + k)
        cu = lambda x: torch.from_numpy(np.ascontiguousarray(x.T.astype(np.float32))).cuda()
        o = {"poses": torch.empty(t.n_bodies, 12, B, device="cuda"), "tau": torch.empty(t.nv, B, device="cuda"),
             "M": torch.empty(t.nv, t.nv, B, device="cuda"), "qdd": torch.empty(t.nv, B, device="cuda")}
        items.append({"q": cu(s["q"]), "qd": cu(s["qd"]), "qdd": cu(s["qdd"]), "tau": cu(s["tau"]),
                      "fk": True, "rnea": True, "crba": True, "aba": True, "out": o})
    mb = fst.MultiBatch(models)

    def separate():
        for m, it in zip(models, items):
            o = it["out"]
            fst.fk(m, it["q"], out=o["poses"])
            fst.rnea(m, it["q"], it["qd"], it["qdd"], out=o["tau"])
            fst.crba(m, it["q"], out=o["M"])
            fst.aba(m, it["q"], it["qd"], it["tau"], out=o["qdd"])

    tp, ts = _graph_us(torch, lambda: mb.eval(items)), _graph_us(torch, separate)
    level = {}
    for block in (64, 128, 256):          # the level-parallel form of the same launch
        mb.set_launch(block, "level")
        level[f"level/{block}"] = round(_graph_us(torch, lambda: mb.eval(items)), 3)
    mb.set_launch(64, "generic")
    best = min(level, key=level.get)
    n = sum(counts)
    return {"workload": "5 trees (7/11/12/18/23 DOF) x (4096/2048/1024/512/256 envs): FK+RNEA+CRBA+ABA",
            "persistent_us": round(tp, 3), "separate_us": round(ts, 3),
            "persistent_level_us": level, "persistent_level_best": best,
            "persistent_env_evals_per_s": round(n / tp * 1e6, 1), "separate_env_evals_per_s": round(n / ts * 1e6, 1),
            "persistent_level_env_evals_per_s": round(n / level[best] * 1e6, 1),
            "speedup": round(ts / tp, 3), "level_speedup_vs_generic": round(tp / level[best], 3),
            "launches": {"persistent": 1, "separate": 4 * len(trees)}}


def sysid(torch, fst, w, steps=500):
    """Link-parameter identification on the 7-DOF chain (paper Sec. 4.3
    setting on a synthetic arm): B = 8192 samples, measured torques = true
    RNEA x (1 + 0.05 N(0,1)), all 70 parameters start perturbed by
    U(-30%, +30%), Adam (lr 1e-2) for `steps` steps, each step one fused
    loss-and-gradient kernel; and the exact least-squares minimiser from
    71 + 1 calls of the same kernel."""
    from paper_2605_31481_gb300 import sysid as sid
    tree = w.chain(7, seed=0)
    B = 8192
    m = fst.Model(tree)
    try:
        m.specialize(["rnea", "loss_grad"])
    except Exception:
        pass
    s = w.random_state(tree, B, seed=1)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(np.asarray(x).T.astype(np.float32))).cuda()
    q, qd, qdd = cu(s["q"]), cu(s["qd"]), cu(s["qdd"])
    true = m.theta()
    rng = np.random.default_rng(7)
    tau_true = fst.rnea(m, q, qd, qdd)
    tau_meas = (tau_true * torch.from_numpy((1 + 0.05 * rng.standard_normal(tuple(tau_true.shape))).astype(np.float32)).cuda()).contiguous()
    theta0 = (true * torch.from_numpy(rng.uniform(-0.3, 0.3, tuple(true.shape)).astype(np.float32) + 1).cuda()).contiguous()
    sid.identify(m, q, qd, qdd, tau_meas, theta0, steps=2)            # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    theta, _ = sid.identify(m, q, qd, qdd, tau_meas, theta0, steps=steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    err = sid.mass_errors(theta, true.cpu().numpy())
    err0 = sid.mass_errors(theta0, true.cpu().numpy())
    sid.identify_least_squares(m, q, qd, qdd, tau_meas, theta0)    # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    theta_ls, _ = sid.identify_least_squares(m, q, qd, qdd, tau_meas, theta0)
    torch.cuda.synchronize()
    dt_ls = time.perf_counter() - t0
    err_ls = sid.mass_errors(theta_ls, true.cpu().numpy())
    sid.identify_masses(m, q, qd, qdd, tau_meas, true)                # warm (first use of the solver)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    masses, _ = sid.identify_masses(m, q, qd, qdd, tau_meas, true)
    torch.cuda.synchronize()
    dt_m = time.perf_counter() - t0
    err_m = (masses - true[:, 0]).abs() / true[:, 0]
    return {"workload": "chain7, B=8192, 70 parameters, 5% torque noise, +-30% initial error",
            "adam": {"steps": steps, "seconds": round(dt, 3), "steps_per_s": round(steps / dt, 1),
                     "mass_error_pct_mean": round(100 * float(err.mean()), 2),
                     "mass_error_pct_per_link": [round(100 * float(x), 2) for x in err]},
            "least_squares": {"kernel_calls": int(true.numel()) + 2, "seconds": round(dt_ls, 4),
                              "mass_error_pct_mean": round(100 * float(err_ls.mean()), 2),
                              "mass_error_pct_per_link": [round(100 * float(x), 2) for x in err_ls]},
            "masses_only_least_squares": {
                "setting": "masses unknown, centres of mass and rotational inertias known (the paper's Sec. 4.3)",
                "kernel_calls": tree.n_bodies + 1, "seconds": round(dt_m, 4),
                "mass_error_pct_mean": round(100 * float(err_m.mean()), 2),
                "mass_error_pct_mean_links_2_to_7": round(100 * float(err_m[1:].mean()), 2),
                "mass_error_pct_per_link": [round(100 * float(x), 2) for x in err_m]},
            "mass_error_pct_initial_mean": round(100 * float(err0.mean()), 2)}


def per_op_times(torch, launch, sets, R, stream, K_op, hot=False):
    """Each operator alone, its own kernel per call at its tuned
    configuration, replayed from a CUDA graph of R calls (for the
    per-operator env-evals/s). Cold: the R calls rotate over the R input
    sets (more than twice L2 in total); hot: all R calls use the first set,
    which stays L2-resident. Each replay is timed on its own; the median
    over replays, per call, is returned."""
    out = {}
    for op in OPS:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for k in range(R):
                launch(op, sets[0 if hot else k])
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        reps = max(5, K_op // R)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        ev[0].record(stream)
        for r in range(reps):
            g.replay()
            ev[r + 1].record(stream)
        torch.cuda.synchronize()
        out[op] = statistics.median(ev[r].elapsed_time(ev[r + 1]) for r in range(reps)) / R
    return out


def ctypes_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def link_bandwidth(torch, dev, nbytes=256 << 20, reps=5):
    """The host link's copy bandwidth, measured: one cudaMemcpyAsync of
    `nbytes` between pinned host memory and the device each way (and both at
    once, on two streams), timed with CUDA events, best of `reps`. The
    end-to-end leg's ceiling: its per-step bytes over its step time against
    these."""
    n = nbytes // 4
    h = torch.empty(n).pin_memory()
    h2 = torch.empty(n).pin_memory()
    d = torch.empty(n, device=dev)
    d2 = torch.empty(n, device=dev)
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    res = {}
    for name in ("h2d", "d2h", "both"):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            cur = torch.cuda.current_stream()
            a.record(cur)
            s1.wait_stream(cur)
            s2.wait_stream(cur)
            with torch.cuda.stream(s1):
                if name in ("h2d", "both"):
                    d.copy_(h, non_blocking=True)
            with torch.cuda.stream(s2):
                if name in ("d2h", "both"):
                    h2.copy_(d2, non_blocking=True)
            cur.wait_stream(s1)
            cur.wait_stream(s2)
            b.record(cur)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3)
        res[f"{name}_gbs"] = round((2 if name == "both" else 1) * nbytes / best / 1e9, 1)
    res["bytes_per_copy"] = nbytes
    return res


def run_e2e(torch, fst, model, tree, B, links, st, dev, K, warmup, plan=None, slots=3, split=1, packed=False):
    """The same step through the public binding, end to end: every step
    uploads its inputs from pinned host memory, runs the step (the tuned step
    plan) and reads every output back into pinned host memory. Inputs and
    outputs each live in one contiguous block (one copy per direction), and
    the whole step is captured once as a CUDA graph and replayed, as a
    training loop with a fixed step shape would. With slots > 1, that many
    such step graphs (each with its own buffers and stream) alternate, so one
    step's read-back overlaps the next step's upload and compute. The timed
    region ends when the last step's outputs are on the host. packed=True
    reads back M's upper triangle and the Jacobians' support-path columns
    only (the packed layouts of fst_eval, the same information)."""
    nq, nv, nb, nl = tree.nq, tree.nv, tree.n_bodies, len(links)
    in_rows = {"q": nq, "qd": nv, "qdd": nv, "tau": nv}
    out_shapes = {"poses": (nb, 12, B), "J": (nl, 6, nv, B), "tau": (nv, B), "M": (nv, nv, B), "qdd": (nv, B)}
    if packed:
        _, j_rows, m_rows = fst.api.packed_layout(model, links)
        out_shapes.update({"J": (j_rows, B), "M": (m_rows, B)})
    n_in = sum(in_rows.values()) * B
    n_out = sum(int(np.prod(sh)) for sh in out_shapes.values())
    host_in = np.concatenate([np.ascontiguousarray(st[k][:B].T.astype(np.float32)).ravel() for k in in_rows])

    def views(flat, layout):
        out, off = {}, 0
        for k, sh in layout.items():
            sh = (sh, B) if isinstance(sh, int) else sh
            n = int(np.prod(sh))
            out[k] = flat[off:off + n].view(*sh)
            off += n
        return out

    S = []
    for _ in range(slots):
        sl = {"stream": torch.cuda.Stream(device=dev),
              "host_in": torch.from_numpy(host_in.copy()).pin_memory(),
              "dev_in": torch.empty(n_in, device=dev), "dev_out": torch.empty(n_out, device=dev),
              "host_out": torch.empty(n_out).pin_memory(),
              "copy_streams": [torch.cuda.Stream(device=dev) for _ in range(split)]}
        sl["in"], sl["out"] = views(sl["dev_in"], in_rows), views(sl["dev_out"], out_shapes)
        S.append(sl)
    bounds = [n_out * k // split for k in range(split + 1)]

    def step(sl):
        sl["dev_in"].copy_(sl["host_in"], non_blocking=True)
        i = sl["in"]
        if plan is not None:
            plan(i["q"], i["qd"], i["qdd"], i["tau"], sl["out"], packed=packed)
        else:
            fst.api.eval(model, i["q"], i["qd"], i["qdd"], i["tau"], fk=True, links=links, rnea=True, crba=True,
                         aba=True, out=sl["out"], packed=packed)
        if split == 1:
            sl["host_out"].copy_(sl["dev_out"], non_blocking=True)
            return
        # the read-back in `split` chunks on parallel branches (several copy engines)
        cur = torch.cuda.current_stream()
        for k, cs in enumerate(sl["copy_streams"]):
            cs.wait_stream(cur)
            with torch.cuda.stream(cs):
                sl["host_out"][bounds[k]:bounds[k + 1]].copy_(sl["dev_out"][bounds[k]:bounds[k + 1]], non_blocking=True)
        for cs in sl["copy_streams"]:
            cur.wait_stream(cs)

    for sl in S:
        with torch.cuda.stream(sl["stream"]):
            for _ in range(3):
                step(sl)
        torch.cuda.synchronize()
        sl["graph"] = torch.cuda.CUDAGraph()
        with torch.cuda.graph(sl["graph"], stream=sl["stream"]):
            step(sl)
    def replay(k):
        sl = S[k % slots]
        with torch.cuda.stream(sl["stream"]):
            sl["graph"].replay()

    for k in range(max(3, warmup // 10)):
        replay(k)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(cur)
    for sl in S:
        sl["stream"].wait_stream(cur)
    for k in range(K):
        replay(k)
    for sl in S:
        cur.wait_stream(sl["stream"])
    b.record(cur)
    torch.cuda.synchronize()
    return {"ms": a.elapsed_time(b), "h2d": n_in * 4, "d2h": n_out * 4, "slots": slots, "steps": K,
            "readback_chunks": split, "layout": "packed" if packed else "full"}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_step(tree, links, s):
    from oracle import rbd
    rbd.fk(tree, s["q"])
    for l in links:
        rbd.jacobian(tree, s["q"], l)
    rbd.rnea(tree, s["q"], s["qd"], s["qdd"])
    rbd.crba(tree, s["q"])
    rbd.aba(tree, s["q"], s["qd"], s["tau"])


def _oracle_worker(job):
    """One host process of the all-cores baseline: the oracle on its own
    seeded sample of Bs environments for budget_s seconds."""
    seed, Bs, budget_s = job
    from paper_2605_31481_gb300 import workloads as w
    tree, _, links = workload()
    s = w.random_state(tree, Bs, seed=100 + seed)
    oracle_step(tree, links, s)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        oracle_step(tree, links, s)
        n += 1
    return n * Bs, time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_all_cores(budget_s=8.0, Bs=512):
    """The same oracle, one single-threaded process per host core (spawned,
    so no process is forked from one that holds a CUDA context), each on its
    own sample of the workload; env-evals/s summed over processes."""
    import multiprocessing as mp
    n = host_cores()
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [(k, Bs, budget_s) for k in range(n)])
    value = sum(e / t for e, t in res)
    return {"value": round(value, 1), "unit": "env-evals/s", "cores": n, "kind": "oracle",
            "sample": f"{n} processes x {Bs} envs of the same tree, FP64 numpy, 1 thread each, about {budget_s:.0f} s"}


def cpu_baseline(tree, links, args, st=None, gpu_first=None, budget_s=12.0, Bs=512):
    """The FP64 oracle timed on the host (1 thread) over the first Bs
    environments of the step's first input set; when the GPU step's outputs
    for those inputs are given, also their largest per-environment normwise
    error against the oracle (the same check the tests apply)."""
    from oracle import rbd
    from paper_2605_31481_gb300 import workloads as w
    s = {k: v[:Bs] for k, v in st.items()} if st is not None else w.random_state(tree, Bs, seed=1)
    oracle_step(tree, links, s)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        oracle_step(tree, links, s)
        n += 1
    dt = time.perf_counter() - t0
    cpu = {"value": round(n * Bs / dt, 1), "unit": "env-evals/s", "cores": 1, "kind": "oracle",
           "sample": f"{n} passes of FK+4 Jacobians+RNEA+CRBA+ABA over {Bs} envs of the same tree (FP64 numpy, "
                     f"1 thread, {dt:.1f} s)"}
    parity = detail = None
    if gpu_first is not None:
        T = rbd.fk(tree, s["q"])
        ref = {"poses": np.concatenate([T[..., :3, :3].reshape(Bs, -1, 9), T[..., :3, 3]], -1),
               "J": np.stack([rbd.jacobian(tree, s["q"], l) for l in links], 1),
               "tau": rbd.rnea(tree, s["q"], s["qd"], s["qdd"]), "M": rbd.crba(tree, s["q"]),
               "qdd": rbd.aba(tree, s["q"], s["qd"], s["tau"])}
        tol = {"poses": 1e-5, "J": 1e-5, "tau": 1e-4, "M": 1e-4, "qdd": 1e-4}
        parity, p999 = {}, {}
        for k, r in ref.items():
            g = np.moveaxis(gpu_first[k], -1, 0)[:Bs].reshape(Bs, -1)
            r = r.reshape(Bs, -1)
            env = np.abs(g - r).max(1) / np.maximum(np.abs(r).max(1), 1.0)
            err = float(env.max())
            if not err <= tol[k]:
                raise RuntimeError(f"parity check failed: {k} error {err:.3e} > {tol[k]}")
            parity[k] = float(f"{err:.2e}")
            p999[k] = float(f"{np.quantile(env, 0.999):.2e}")
        # forward dynamics: the backward error of the GPU's accelerations
        # (the torque the oracle's inverse dynamics needs for them, against
        # the applied torque) and the conditioning of M, per environment
        qdd_gpu = np.moveaxis(gpu_first["qdd"], -1, 0)[:Bs]
        tau_back = rbd.rnea(tree, s["q"], s["qd"], qdd_gpu)
        bwd = np.abs(tau_back - s["tau"]).max(1) / np.maximum(np.abs(s["tau"]).max(1), 1.0)
        cond = np.linalg.cond(ref["M"])
        detail = {"envs": Bs, "p99_9": p999,
                  "qdd_backward_error": {"max": float(f"{bwd.max():.2e}"),
                                         "p99_9": float(f"{np.quantile(bwd, 0.999):.2e}")},
                  "cond2_M": {"max": float(f"{cond.max():.3g}"), "median": float(f"{np.median(cond):.3g}")}}
    return cpu, parity, detail


def run_reference(args, budget_s=120.0):
    """The FP64 oracle as the reference arm, on the host (rank 0 only). One
    environment-evaluation is all five operators; each step runs one of
    them in turn (FK, the 4 foot Jacobians, RNEA, CRBA, ABA) on a sample of
    the workload's environments, sized from a short probe so that the whole
    --steps K --warmup W run takes about budget_s seconds (at least one and
    at most 256 environments per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import rbd
    from paper_2605_31481_gb300 import workloads as w
    tree, B, links = workload()
    ops = (lambda s: rbd.fk(tree, s["q"]),
           lambda s: [rbd.jacobian(tree, s["q"], l) for l in links],
           lambda s: rbd.rnea(tree, s["q"], s["qd"], s["qdd"]),
           lambda s: rbd.crba(tree, s["q"]),
           lambda s: rbd.aba(tree, s["q"], s["qd"], s["tau"]))

    def op_times(n):
        s = w.random_state(tree, n, seed=1)
        out = []
        for f in ops:
            f(s)
            t0 = time.perf_counter()
            f(s)
            out.append(time.perf_counter() - t0)
        return sum(out) / len(out)

    t1, t64 = op_times(1), op_times(64)
    per_env = max((t64 - t1) / 63, 1e-9)
    target = budget_s / max(args.steps + args.warmup, 1)
    Bs = int(max(1, min(256, (target - t1) / per_env)))
    s = w.random_state(tree, Bs, seed=1)
    for k in range(args.warmup):
        ops[k % len(ops)](s)
    t0 = time.perf_counter()
    for k in range(args.steps):
        ops[k % len(ops)](s)
    tot = time.perf_counter() - t0
    value = Bs * args.steps / len(ops) / tot
    sample = (f"{Bs} of the 4096 envs; each step one of the five operators in turn (FK, 4 Jacobians, RNEA, CRBA, "
              f"ABA), FP64 numpy oracle, 1 thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "env-evals/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot / max(args.steps, 1), 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{tree.name}: 11 revolute DOF branched tree, depth 5, B=4096",
                   "B": B, "step": "+".join(OPS) + " (4 foot Jacobians)", "sample_envs_per_step": Bs},
        "cpu_baseline": {"value": round(value, 1), "unit": "env-evals/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 1), "unit": "env-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=("fst", "reference"), default="fst")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary legs (fwd+bwd, RL-step graph, humanoid sweep) after the timed step")
    ap.add_argument("--e2e-slots", type=int, default=3,
                    help="end-to-end leg: steps in flight (streams with their own buffers)")
    ap.add_argument("--e2e-split", type=int, default=1,
                    help="end-to-end leg: read-back chunks copied on parallel graph branches")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture (else null)")
    ap.add_argument("--plan", default=None,
                    help="run this step plan instead of tuning one, named as the keys of the line's plan.us, "
                         "e.g. 'hybrid[specialized/128|level/128]@100%%+fusedfirst' (for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the host-oracle legs (cpu_baseline is then null; for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.plan is not None:
        from paper_2605_31481_gb300.autotune import StepPlan
        try:
            StepPlan.parse_key(args.plan)
        except ValueError as exc:
            ap.error(str(exc))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fst(args)


if __name__ == "__main__":
    main()
