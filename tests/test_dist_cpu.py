"""Sharded identification across ranks, on CPU with the gloo backend (two
processes): each rank sums the inertial-parameter gradient over its own
contiguous shard of environments, one all-reduce adds the shards, and the
result equals the full-batch gradient. The per-shard gradients come from the
oracle's regressor; this exercises the sharding and reduction the GPU path
uses, without a GPU. The benchmark's whole-job rate (the slowest replica's
time, all replicas' environments) is checked the same way."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import rbd, derivs
from paper_2605_31481_gb300 import sysid
from paper_2605_31481_gb300 import workloads as w


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _grad(tree, s, lo, hi, tau_meas, theta):
    sl = slice(lo, hi)
    r = rbd.rnea(tree, s["q"][sl], s["qd"][sl], s["qdd"][sl], theta=theta) - tau_meas[sl]
    Y = derivs.regressor(tree, s["q"][sl], s["qd"][sl], s["qdd"][sl])
    return np.einsum("bi,bink->nk", 2 * r, Y), float(np.sum(r * r))


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tree = w.chain(7, seed=0)
    B = 61
    s = w.random_state(tree, B, seed=2)
    theta = rbd.Model(tree).theta() * 1.1
    tau_meas = rbd.rnea(tree, s["q"], s["qd"], s["qdd"])
    lo, hi = sysid.shard(B, rank, world)
    g, L = _grad(tree, s, lo, hi, tau_meas, theta)
    buf = torch.from_numpy(np.concatenate([g.ravel(), [L]]))
    sysid.allreduce_sum(buf)
    if rank == 0:
        np.save(out_path, buf.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_gradient_equals_full_batch(tmp_path):
    out = str(tmp_path / "g.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    tree = w.chain(7, seed=0)
    s = w.random_state(tree, 61, seed=2)
    theta = rbd.Model(tree).theta() * 1.1
    g, L = _grad(tree, s, 0, 61, rbd.rnea(tree, s["q"], s["qd"], s["qdd"]), theta)
    ref = np.concatenate([g.ravel(), [L]])
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


def test_allreduce_is_identity_without_a_process_group():
    t = torch.arange(5.0)
    assert torch.equal(sysid.allreduce_sum(t.clone()), t)


def test_shards_cover_the_batch():
    for B in (0, 1, 7, 8192, 8193):
        for world in (1, 2, 3, 8):
            ranges = [sysid.shard(B, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == B
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1


def _rate_worker(rank, world, port, out_path):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.job_rate(10.0 + 5.0 * rank, world, 4096, 100, "cpu")
    if rank == 0:
        np.save(out_path, np.array([ms, value]))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_rate_takes_the_slowest_rank(tmp_path):
    out = str(tmp_path / "r.npy")
    mp.start_processes(_rate_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    ms, value = np.load(out)
    assert ms == 15.0
    assert value == pytest.approx(2 * 4096 * 100 / 0.015, rel=1e-12)
    import bench
    assert bench.job_rate(8.0, 1, 4096, 100, "cpu") == (8.0, 4096 * 100 / 0.008)
