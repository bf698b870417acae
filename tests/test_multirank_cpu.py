"""The multi-GPU design, emulated with CPU ranks (gloo, world size 2): each
rank counts the cells of its own z-slab (it needs one halo plane from the
rank below), the ranks sum their int64 curves in one all-reduce, and the
result equals the single-process curves exactly (integer sums are
associative).  No GPU is involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, d, h, w, L, seed, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(seed)
    field = rng.integers(0, L + 2, size=(d, h, w)).astype(np.uint16)   # every rank makes the same field
    bins = oracle.bin_field(field, None, L)
    # rank r owns voxel planes [z0, z1) and the cells with doubled z in [2 z0, 2 z1); the last rank
    # also owns the top boundary plane 2d.  Those cells touch voxel planes z0-1 .. z1-1 only.
    bounds = np.linspace(0, d, world + 1).astype(int)
    z0, z1 = int(bounds[rank]), int(bounds[rank + 1])
    zhi = 2 * z1 - 1 if rank < world - 1 else 2 * d
    lo = max(z0 - 1, 0)
    part = oracle.curves_3d_zrange(np.ascontiguousarray(bins[lo:z1]), L, 2 * z0 - 2 * lo, zhi - 2 * lo)
    # the sub-array's own top plane must not pull in cells of the next slab
    t = torch.from_numpy(np.stack([part[k] for k in ("ec", "perimeter", "area", "volume")]))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        q.put(t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("d,h,w,L", [(9, 7, 8, 5), (16, 12, 10, 9)])
def test_two_rank_slab_allreduce_equals_single_process(d, h, w, L):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, d, h, w, L, 11, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(11)
    field = rng.integers(0, L + 2, size=(d, h, w)).astype(np.uint16)
    want = oracle.ec_curves(field, None, L, 26, 15)
    np.testing.assert_array_equal(got, want)
