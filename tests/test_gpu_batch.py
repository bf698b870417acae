"""ec_batch: one persistent launch over uneven 2D/3D fields of mixed dtypes,
level counts and descriptor sets gives, field by field, the curves of
separate calls and of the oracle."""
import zlib

import numpy as np
import pytest
import torch

import oracle
from paper_2311_11740_gb300 import ec, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ec.Context(0)


def _mixed_fields(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 6
        if kind == 0:
            h, w = (int(v) for v in rng.integers(1, 300, size=2))
            f = workloads.quantize_u8(workloads.grf_2d(int(rng.integers(1 << 30)), h, w, 2.0)).numpy()
            out.append(dict(field=f, thr=None, L=256, conn=int(rng.choice([4, 8])), desc=int(rng.integers(1, 8))))
        elif kind == 1:
            h, w = (int(v) for v in rng.integers(1, 200, size=2))
            f = rng.normal(size=(h, w)).astype(np.float32)
            thr = np.sort(rng.normal(size=int(rng.integers(1, 300)))).astype(np.float32)
            out.append(dict(field=f, thr=thr, L=thr.size, conn=8, desc=7))
        elif kind == 2:
            d, h, w = (int(v) for v in rng.integers(1, 70, size=3))
            f, thr = workloads.config3(n=max(d, h, w), nblobs=8, L=int(rng.integers(2, 700)))
            f = np.ascontiguousarray(f.numpy()[:d, :h, :w])
            out.append(dict(field=f, thr=thr.numpy(), L=thr.numel(), conn=26, desc=int(rng.integers(1, 16))))
        elif kind == 3:
            d, h, w = (int(v) for v in rng.integers(1, 40, size=3))
            f = rng.integers(0, 600, size=(d, h, w)).astype(np.uint16)
            out.append(dict(field=f, thr=None, L=512, conn=26, desc=15))
        elif kind == 4:
            d, h, w = (int(v) for v in rng.integers(1, 30, size=3))
            f = rng.integers(0, 256, size=(d, h, w)).astype(np.uint8)
            thr = np.sort(rng.integers(0, 256, size=40)).astype(np.uint8)
            out.append(dict(field=f, thr=thr, L=40, conn=26, desc=9))
        else:
            h, w = (int(v) for v in rng.integers(1, 90, size=2))
            f = rng.integers(0, 3000, size=(h, w)).astype(np.uint16)
            out.append(dict(field=f, thr=None, L=2999, conn=4, desc=5))
    return out


def _dev(a):
    if a is None:
        return None
    if a.dtype == np.uint16:
        return torch.from_numpy(a.astype(np.int32)).cuda().to(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run_batch(ctx, fields):
    items = [dict(field=_dev(f["field"]), thresholds=_dev(f["thr"]), L=f["L"], connectivity=f["conn"],
                  descriptors=f["desc"]) for f in fields]
    outs = ec.batch(items, ctx=ctx)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], items


@pytest.mark.parametrize("seed", [1, 2])
def test_batch_equals_oracle_and_single_calls(ctx, seed):
    fields = _mixed_fields(seed, 30)
    got, items = _run_batch(ctx, fields)
    for f, g, it in zip(fields, got, items):
        want = oracle.ec_curves(f["field"], f["thr"], f["L"], f["conn"], f["desc"])
        np.testing.assert_array_equal(g, want)
        alone = ec.curve(it["field"], it["thresholds"], L=f["L"], connectivity=f["conn"], descriptors=f["desc"],
                         ctx=ctx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(g, alone.cpu().numpy())


# Narrow 2D fields share a strip between 4 (or 2) row bands of 64 rows; the
# widths sit at and just past the limits (uint8 241 / 510, uint16 248, float32
# 252), the heights cut bands and items anywhere.
@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_batch_banded_narrow_2d_fields(ctx, dtype):
    rng = np.random.default_rng(zlib.crc32(dtype.encode()))
    widths = {"u8": [1, 2, 63, 241, 242, 300, 510, 511], "u16": [3, 248, 249, 510, 511],
              "f32": [5, 252, 253, 509, 510]}[dtype]
    heights = [65, 128, 129, 255, 257, 300, 513]
    fields = []
    for i, w in enumerate(widths):
        h = heights[i % len(heights)]
        g = workloads.grf_2d(int(rng.integers(1 << 30)), h, w, 3.0).numpy()
        if dtype == "u8":
            f, thr, L = workloads.quantize_u8(torch.from_numpy(g)).numpy(), None, 256
        elif dtype == "u16":
            f, thr, L = np.clip(g * 500 + 1500, 0, 3000).astype(np.uint16), None, 3001
        else:
            f = g.astype(np.float32)
            thr, L = np.linspace(f.min(), f.max(), 200).astype(np.float32), 200
        fields.append(dict(field=f, thr=thr, L=L, conn=[8, 4][i % 2], desc=7))
    got, _ = _run_batch(ctx, fields)
    for f, g in zip(fields, got):
        np.testing.assert_array_equal(g, oracle.ec_curves(f["field"], f["thr"], f["L"], f["conn"], f["desc"]))


def test_batch_repeated_calls_reuse_graph(ctx):
    a = _mixed_fields(3, 12)
    b = _mixed_fields(4, 12)
    for fields in (a, b, a):
        got, _ = _run_batch(ctx, fields)
        for f, g in zip(fields, got):
            np.testing.assert_array_equal(g, oracle.ec_curves(f["field"], f["thr"], f["L"], f["conn"], f["desc"]))


def test_batch_large_level_count_and_big_fields(ctx):
    rng = np.random.default_rng(8)
    big3, thr3 = workloads.config3(n=130, nblobs=40, L=1024)
    fields = [
        dict(field=rng.integers(0, 40000, size=(9, 30, 40)).astype(np.uint16), thr=None, L=40000, conn=26, desc=15),
        dict(field=big3.numpy(), thr=thr3.numpy(), L=1024, conn=26, desc=13),
        dict(field=workloads.config1().numpy(), thr=None, L=256, conn=8, desc=7),
    ]
    got, _ = _run_batch(ctx, fields)
    for f, g in zip(fields, got):
        np.testing.assert_array_equal(g, oracle.ec_curves(f["field"], f["thr"], f["L"], f["conn"], f["desc"]))


def test_batch_rejects_bad_field(ctx):
    f = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    t = torch.zeros(3, dtype=torch.float32, device="cuda")
    with pytest.raises(ec.ECError) as e:
        ec.batch([dict(field=f, thresholds=t, connectivity=8)], ctx=ctx)
    assert e.value.status == 1


def test_batch_planar_branch_fields(ctx):
    """Large 3D fields the planar kernel takes run as their own launches on a
    second branch of the batch's graph, beside the persistent kernel for the
    rest; every field still gets the oracle's curves, on repeated calls and
    with the branch's field count changing."""
    f1, t1 = workloads.config3(n=132, nblobs=40, L=700)
    f2, t2 = workloads.config3(n=136, nblobs=30, L=1024)
    u = np.clip(workloads.grf_nd(5, (128, 136, 136), 3.0).numpy() * 300 + 300, 0, 599).astype(np.uint16)
    big = [
        dict(field=f1.numpy(), thr=t1.numpy(), L=700, conn=26, desc=13),
        dict(field=f2.numpy()[:, :, :132].copy(), thr=t2.numpy(), L=1024, conn=26, desc=15),
        dict(field=f1.numpy(), thr=t1.numpy(), L=700, conn=26, desc=1),
        dict(field=u, thr=None, L=600, conn=26, desc=9),
        dict(field=f2.numpy()[:, :, :130].copy(), thr=t2.numpy(), L=1024, conn=26, desc=13),   # rows not 16 B
    ]
    small = _mixed_fields(31, 10)
    for fields in (big + small, big[:2] + small, small + big):
        got, _ = _run_batch(ctx, fields)
        for f, g in zip(fields, got):
            np.testing.assert_array_equal(g, oracle.ec_curves(f["field"], f["thr"], f["L"], f["conn"], f["desc"]))
