"""Slice sharding through the CUDA path: two ranks (spawned processes,
gloo process group for the host-side reduction) each build the plan and
solve their own weak-scaling shard of a synthetic volume with the library's
CGLS, with no data exchange; every rank's slices must equal the same slices
of a single-process solve of the whole volume bit for bit (slices are
independent problems, and a slice's arithmetic does not depend on its
position in the slice tile), and the reported time is the max over ranks.
Both ranks run on the one GPU of this test: their kernels never wait on one
another (the only collective is on the host)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

WORKLOAD = "small3d_64"
PER_RANK, ITERS = 2, 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, storage, out):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import inputs, shard, xct
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        first, count = shard.weak_range(PER_RANK, rank)
        w = inputs.make_workload(WORKLOAD, slices=count, slice_offset=first, with_images=False,
                                 volume_slices=PER_RANK * world)
        y = torch.tensor(w["sino"], dtype=torch.float32, device="cuda")
        with xct.Plan(w["n"], w["m"], w["nd"], storage, cos_sin=w["cos_sin"]) as p:
            x = p.cgls(y, ITERS)
            torch.cuda.synchronize()
        t = shard.max_over_ranks(1.0 + rank)
        out[rank] = (first, count, x.cpu().numpy(), t)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("storage", ["f16", "f32"])
def test_two_ranks_on_the_cuda_path(storage):
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), storage, out), nprocs=world, join=True,
                           start_method="spawn")
        res = [out[r] for r in range(world)]
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import inputs, xct
    whole = inputs.make_workload(WORKLOAD, slices=PER_RANK * world, with_images=False,
                                 volume_slices=PER_RANK * world)
    y = torch.tensor(whole["sino"], dtype=torch.float32, device="cuda")
    with xct.Plan(whole["n"], whole["m"], whole["nd"], storage, cos_sin=whole["cos_sin"]) as p:
        xw = p.cgls(y, ITERS).cpu().numpy()
    assert not np.array_equal(xw[0], xw[1])
    for r, (first, count, x, t) in enumerate(res):
        assert (first, count) == (PER_RANK * r, PER_RANK)
        assert np.array_equal(x, xw[first:first + count]), r
        assert t == float(world)
