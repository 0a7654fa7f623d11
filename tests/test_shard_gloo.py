"""Slice sharding across ranks, on CPU with two gloo ranks: the per-rank
shards of the synthetic volume are exactly the slices of the whole volume,
the ranges are disjoint and cover it, each rank's solve of its own slices
equals the same slices of the single-process solve (no exchange on the data
path), and the reported time is the max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2009_07226_gb300 import inputs, shard


def test_slice_range_splits():
    for total in (0, 1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            got = [shard.slice_range(total, world, r) for r in range(world)]
            assert sum(c for _, c in got) == total
            assert [s for s, _ in got] == [sum(c for _, c in got[:r]) for r in range(world)]
            assert max(c for _, c in got) - min(c for _, c in got) <= 1
    assert shard.weak_range(64, 3) == (192, 64)
    with pytest.raises(ValueError):
        shard.slice_range(4, 2, 2)
    assert shard.max_over_ranks(2.5) == 2.5      # no process group


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = shard.weak_range(2, rank)
        w = inputs.make_workload("small3d_64", slices=count, slice_offset=first, with_images=False,
                                 volume_slices=2 * world)
        g = oracle.Geometry(n=w["n"], m=w["m"], nd=w["nd"], cos_sin=w["cos_sin"])
        a = oracle.siddon_csr(g)
        at = oracle.transpose(a)
        x, _ = oracle.cgls(lambda X: oracle.project(a, X), lambda Y: oracle.backproject(at, Y),
                           w["sino"].reshape(count, -1), 3)
        t = shard.max_over_ranks(1.0 + rank)
        out[rank] = (first, count, w["sino"], x, t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = [out[r] for r in range(world)]
    whole = inputs.make_workload("small3d_64", slices=2 * world, with_images=False, volume_slices=2 * world)
    g = oracle.Geometry(n=whole["n"], m=whole["m"], nd=whole["nd"], cos_sin=whole["cos_sin"])
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    xw, _ = oracle.cgls(lambda X: oracle.project(a, X), lambda Y: oracle.backproject(at, Y),
                        whole["sino"].reshape(2 * world, -1), 3)
    assert not np.array_equal(whole["sino"][0], whole["sino"][1])
    for r, (first, count, sino, x, t) in enumerate(res):
        assert (first, count) == (2 * r, 2)
        assert np.array_equal(sino, whole["sino"][first:first + count])
        assert np.array_equal(x, xw[first:first + count])
        assert t == float(world)
