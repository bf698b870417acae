"""GPU parity: the CUDA path (through the C ABI) equals the CPU oracle
element by element.  Curves are integers, so the tolerance is zero."""
import itertools
import zlib

import numpy as np
import pytest
import torch

import oracle
from paper_2311_11740_gb300 import ec, workloads

pytestmark = pytest.mark.gpu

ALL2 = ec.EC_DESC_EC | ec.EC_DESC_PERIMETER | ec.EC_DESC_AREA
ALL3 = ALL2 | ec.EC_DESC_VOLUME
ALGOS = [ec.ALGO_PLANAR, ec.ALGO_VOXEL, ec.ALGO_VERTEX]


@pytest.fixture(scope="module")
def ctx(libec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ec.Context(0)


def to_dev(a):
    if a is None:
        return None
    if a.dtype == np.uint16:
        return torch.from_numpy(a.astype(np.int32)).cuda().to(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_curves(ctx, field, thr, L, conn, desc, algo=ec.ALGO_VOXEL, tile_z=0):
    ctx.set_option(ec.EC_OPT_ALGO, algo)
    ctx.set_option(ec.EC_OPT_TILE_Z, tile_z)
    out = ec.curve(to_dev(field), to_dev(thr), L=L, connectivity=conn, descriptors=desc, ctx=ctx)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(ctx, field, thr, L, conn=None, desc=None, algos=ALGOS, tile_z=0):
    conn = conn or (8 if field.ndim == 2 else 26)
    desc = desc or (ALL2 if field.ndim == 2 else ALL3)
    want = oracle.ec_curves(field, thr, L, conn, desc)
    for algo in algos:
        got = gpu_curves(ctx, field, thr, L, conn, desc, algo, tile_z)
        np.testing.assert_array_equal(got, want, err_msg=f"algo={algo} shape={field.shape} L={L}")


def test_exhaustive_binary_3x3(ctx):
    for bits in range(1 << 9):
        a = np.array([(bits >> i) & 1 for i in range(9)], np.uint8).reshape(3, 3)
        for conn in (8, 4):
            check(ctx, a, None, 1, conn=conn)


def test_exhaustive_binary_2x2x2(ctx):
    for bits in range(1 << 8):
        a = np.array([(bits >> i) & 1 for i in range(8)], np.uint8).reshape(2, 2, 2)
        check(ctx, a, None, 1)


SHAPES3 = [(1, 1, 1), (1, 1, 7), (1, 5, 1), (3, 1, 1), (2, 3, 5), (7, 11, 13), (1, 40, 37), (33, 9, 31),
           (32, 8, 32), (31, 7, 33), (65, 17, 3), (5, 64, 65), (40, 1, 70)]


@pytest.mark.parametrize("shape", SHAPES3)
@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_random_3d(ctx, shape, dtype):
    rng = np.random.default_rng(zlib.crc32(repr((shape, dtype)).encode()))
    if dtype == "u8":
        L = int(rng.integers(1, 40))
        f = rng.integers(0, L + 3, size=shape).astype(np.uint8)
        thr = None
    elif dtype == "u16":
        L = int(rng.integers(1, 3000))
        f = rng.integers(0, L + 50, size=shape).astype(np.uint16)
        thr = None if rng.random() < 0.5 else np.sort(rng.integers(0, L + 60, size=L)).astype(np.uint16)
    else:
        L = int(rng.integers(1, 200))
        f = rng.normal(size=shape).astype(np.float32)
        thr = np.sort(rng.normal(size=L)).astype(np.float32)
    check(ctx, f, thr, L)


# float32 fields whose rows are multiples of 4 floats and whose storage
# starts 16-byte aligned take the TMA staging; with at most 1024 levels and
# the descriptor sets EC, EC|AREA|VOLUME or all four they run on the kernel
# with two stacked quads per thread (64 x 32 tiles).  Partial tiles in x, y
# and z, odd heights (a thread's second row outside the field), one-plane
# fields, uniform thresholds (spacing guess) and irregular ones.
SHAPES3_TMA = [(1, 1, 4), (3, 1, 8), (2, 33, 68), (17, 31, 132), (70, 65, 64), (9, 64, 4), (5, 2, 196),
               (130, 3, 12), (1, 32, 64), (33, 97, 100)]


@pytest.mark.parametrize("shape", SHAPES3_TMA)
@pytest.mark.parametrize("uniform", [True, False])
def test_planar_tma_shapes(ctx, shape, uniform):
    rng = np.random.default_rng(zlib.crc32(repr((shape, uniform, "tma")).encode()))
    if uniform:
        f = workloads.grf_nd(int(rng.integers(1 << 30)), shape, 1.5).numpy().astype(np.float32)
        L = int(rng.integers(2, 1025))
        thr = workloads.uniform_thresholds(float(f.min()), float(f.max()), L).numpy()
    else:
        f = rng.normal(size=shape).astype(np.float32)
        L = int(rng.integers(1, 1025))
        thr = np.sort(rng.normal(size=L)).astype(np.float32)
    for desc in (1, 13, 15):
        check(ctx, f, thr, L, desc=desc, algos=[ec.ALGO_PLANAR])


# uint16 fields with identity levels (rows a multiple of 8 values) take the
# same kernel with an 80 x 34 TMA box; out-of-field cells read 0 there, so
# tiles at the field's edge are the ones to test.
SHAPES3_TMA16 = [(1, 1, 8), (3, 5, 16), (2, 33, 72), (17, 31, 136), (70, 65, 64), (9, 64, 8), (33, 97, 104)]


@pytest.mark.parametrize("shape", SHAPES3_TMA16)
def test_planar_tma_uint16_identity_levels(ctx, shape):
    rng = np.random.default_rng(zlib.crc32(repr((shape, "tma16")).encode()))
    for L in (1, 37, 4096):
        f = rng.integers(0, L + 40, size=shape).astype(np.uint16)   # values at and above L too
        for desc in (1, 9):
            check(ctx, f, None, L, desc=desc, algos=[ec.ALGO_PLANAR])
    g = np.clip(workloads.grf_nd(int(rng.integers(1 << 30)), shape, 2.0).numpy() * 600 + 2000, 0, 4095)
    g = g.astype(np.uint16)
    check(ctx, g, None, 4096, desc=9, algos=[ec.ALGO_PLANAR, ec.ALGO_VOXEL])
    for slab in (1, 5, 64):
        got = ec.curve_3d_stream(g, L=4096, descriptors=9, slab_planes=slab, ctx=ctx)
        np.testing.assert_array_equal(got, oracle.ec_curves(g, None, 4096, 26, 9))


# float32 rows that are not a multiple of 16 bytes: the planar kernel stages
# each row itself (16-byte cp.async chunks from the boundary at or below the
# row's first staged element, binned from the row's start phase; cells past
# the row read neighbouring rows' values and are masked by coordinates).
# Widths of every residue mod 4, partial tiles, the field's first and last
# rows (chunks before and past its memory), item depths, and streamed slabs.
SHAPES3_ROWS = [(1, 1, 5), (3, 33, 65), (17, 31, 131), (70, 65, 67), (5, 2, 197), (33, 97, 101), (2, 70, 130),
                (9, 64, 3)]


@pytest.mark.parametrize("shape", SHAPES3_ROWS)
@pytest.mark.parametrize("uniform", [True, False])
def test_planar_row_copies(ctx, shape, uniform):
    rng = np.random.default_rng(zlib.crc32(repr((shape, uniform, "rows")).encode()))
    if uniform:
        f = workloads.grf_nd(int(rng.integers(1 << 30)), shape, 1.5).numpy().astype(np.float32)
        L = int(rng.integers(2, 1025))
        thr = workloads.uniform_thresholds(float(f.min()), float(f.max()), L).numpy()
    else:
        f = rng.normal(size=shape).astype(np.float32)
        L = int(rng.integers(1, 1025))
        thr = np.sort(rng.normal(size=L)).astype(np.float32)
    for desc in (1, 13, 15):
        check(ctx, f, thr, L, desc=desc, algos=[ec.ALGO_PLANAR])
    if shape[0] >= 17:
        check(ctx, f, thr, L, desc=13, algos=[ec.ALGO_PLANAR], tile_z=3)
        for slab in (1, 7):
            got = ec.curve_3d_stream(f, thresholds=thr, descriptors=13, slab_planes=slab, ctx=ctx)
            np.testing.assert_array_equal(got, oracle.ec_curves(f, thr, L, 26, 13))


def test_planar_tma_item_depths_and_constant_field(ctx):
    """Work items of 1..7 and 64 planes; a constant field puts every voxel of a
    block on one level, the largest count the packed area/volume words take
    between two exchanges."""
    f, thr = workloads.config3(n=68, nblobs=25, L=700)
    f, thr = f.numpy(), thr.numpy()
    for tz in (1, 2, 3, 5, 7, 64):
        check(ctx, f, thr, 700, desc=13, algos=[ec.ALGO_PLANAR], tile_z=tz)
    c = np.zeros((96, 64, 128), np.float32)
    for desc in (13, 15):
        check(ctx, c, np.array([-1.0, 0.0, 1.0], np.float32), 3, desc=desc, algos=[ec.ALGO_PLANAR])


# Rows of 16-byte multiples take the cp.async staging (uint8 / uint16, and
# float32 fields whose storage is not 16-byte aligned take plain loads);
# partial tiles in x, y and z.
SHAPES3_ALIGNED = [(3, 17, 80), (9, 33, 144), (66, 5, 48), (1, 1, 16), (2, 19, 208)]


@pytest.mark.parametrize("shape", SHAPES3_ALIGNED)
@pytest.mark.parametrize("dtype", ["u8", "u16"])
def test_random_3d_aligned_rows(ctx, shape, dtype):
    rng = np.random.default_rng(zlib.crc32(repr((shape, dtype, "rows")).encode()))
    smooth = workloads.grf_nd(int(rng.integers(1 << 30)), shape, 2.0).numpy()
    if dtype == "u8":
        f, L, thr = workloads.quantize_u8(torch.from_numpy(smooth)).numpy(), 256, None
    else:
        f = np.clip(smooth * 300 + 1000, 0, 2000).astype(np.uint16)
        L, thr = 700, np.sort(rng.integers(0, 2001, size=700)).astype(np.uint16)
    for desc in (1, 13, 15, 6):
        check(ctx, f, thr, L, desc=desc, algos=[ec.ALGO_PLANAR, ec.ALGO_VOXEL])


def test_3d_unaligned_float_pointer(ctx):
    rng = np.random.default_rng(11)
    shape, L = (7, 20, 64), 90
    vals = rng.normal(size=shape).astype(np.float32)
    thr = np.sort(rng.normal(size=L)).astype(np.float32)
    flat = torch.zeros(vals.size + 1, dtype=torch.float32)
    flat[1:] = torch.from_numpy(vals.reshape(-1))
    dev = flat.cuda()[1:].view(shape)
    assert dev.data_ptr() % 16 != 0
    got = ec.curve(dev, to_dev(thr), L=L, descriptors=ALL3, ctx=ctx)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.ec_curves(vals, thr, L, 26, ALL3))


SHAPES2 = [(1, 1), (1, 9), (7, 1), (3, 5), (17, 255), (16, 256), (15, 257), (64, 300), (65, 513), (200, 3)]


@pytest.mark.parametrize("shape", SHAPES2)
@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_random_2d(ctx, shape, dtype):
    rng = np.random.default_rng(zlib.crc32(repr((shape, dtype, 2)).encode()))
    if dtype == "u8":
        L = int(rng.integers(1, 256))
        f = rng.integers(0, 256, size=shape).astype(np.uint8)
        thr = None if rng.random() < 0.5 else np.sort(rng.integers(0, 256, size=L)).astype(np.uint8)
    elif dtype == "u16":
        L = int(rng.integers(1, 5000))
        f = rng.integers(0, L + 50, size=shape).astype(np.uint16)
        thr = None
    else:
        L = int(rng.integers(1, 300))
        f = rng.normal(size=shape).astype(np.float32)
        thr = np.sort(rng.normal(size=L)).astype(np.float32)
    for conn in (8, 4):
        check(ctx, f, thr, L, conn=conn)


# Rows whose start is 16-byte aligned go through the asynchronous row copies
# (whole 16-byte chunks, zero-filled outside the field); the others through
# per-pixel loads.  Wide fields cover several 1024-pixel strips, the last one
# partial; heights 1-3 leave items shorter than the copy-ahead distance.
SHAPES2_WIDE = [(1, 1024), (2, 1040), (3, 2064), (33, 1536), (5, 1041), (4, 1030), (70, 1088)]


@pytest.mark.parametrize("shape", SHAPES2_WIDE)
@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_wide_2d_strips(ctx, shape, dtype):
    rng = np.random.default_rng(zlib.crc32(repr((shape, dtype, "wide")).encode()))
    smooth = workloads.grf_2d(int(rng.integers(1 << 30)), shape[0], shape[1], 4.0).numpy()
    if dtype == "u8":
        f, L, thr = workloads.quantize_u8(torch.from_numpy(smooth)).numpy(), 256, None
    elif dtype == "u16":
        f, L, thr = (np.clip(smooth * 400 + 2000, 0, 4000)).astype(np.uint16), 4001, None
    else:
        f = smooth.astype(np.float32)
        L = 257
        thr = np.linspace(f.min(), f.max(), L).astype(np.float32)
    for conn in (8, 4):
        check(ctx, f, thr, L, conn=conn, algos=[ec.ALGO_PLANAR, ec.ALGO_VOXEL])


def test_2d_unaligned_field_pointer(ctx):
    # a field whose storage starts one element past an aligned address
    rng = np.random.default_rng(5)
    for dtype, L in ((torch.uint8, 256), (torch.float32, 100)):
        h, w = 9, 2048
        flat = torch.zeros(h * w + 1, dtype=dtype)
        if dtype == torch.uint8:
            vals = torch.from_numpy(rng.integers(0, 256, size=h * w).astype(np.uint8))
            thr = None
        else:
            vals = torch.from_numpy(rng.normal(size=h * w).astype(np.float32))
            thr = np.sort(rng.normal(size=L)).astype(np.float32)
        flat[1:] = vals
        dev = flat.cuda()[1:].view(h, w)
        assert dev.data_ptr() % 16 != 0
        want = oracle.ec_curves(vals.view(h, w).numpy(), thr, L, 8, ALL2)
        got = ec.curve(dev, to_dev(thr), L=L, connectivity=8, descriptors=ALL2, ctx=ctx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), want)


def test_float_special_values(ctx):
    rng = np.random.default_rng(9)
    f = rng.normal(size=(9, 10, 11)).astype(np.float32)
    flat = f.reshape(-1)
    flat[rng.choice(flat.size, 30, replace=False)] = np.nan
    flat[rng.choice(flat.size, 10, replace=False)] = np.inf
    flat[rng.choice(flat.size, 10, replace=False)] = -np.inf
    flat[rng.choice(flat.size, 10, replace=False)] = -0.0
    flat[rng.choice(flat.size, 10, replace=False)] = 0.0
    thr = np.array([-np.inf, -1.0, 0.0, 0.0, 0.0, 0.5, 1.0, 1.0, np.inf], np.float32)
    check(ctx, f, thr, len(thr))
    f2 = f[0].copy()
    check(ctx, f2, thr, len(thr), conn=4)


def test_smoothed_3d_and_tile_z(ctx):
    f, thr = workloads.config3(n=48, nblobs=20, L=97)
    f, thr = f.numpy(), thr.numpy()
    for tz in (1, 2, 7, 48, 64):
        check(ctx, f, thr, len(thr), tile_z=tz)


def test_large_level_counts_use_global_paths(ctx):
    rng = np.random.default_rng(4)
    # more levels than the shared-memory histogram / threshold copies hold
    f = rng.integers(0, 65535, size=(6, 20, 30)).astype(np.uint16)
    check(ctx, f, None, 65535)
    g = rng.normal(size=(5, 17, 23)).astype(np.float32)
    thr = np.sort(rng.normal(size=9000)).astype(np.float32)
    check(ctx, g, thr, len(thr))
    h = rng.integers(0, 30000, size=(300, 200)).astype(np.uint16)
    check(ctx, h, None, 30000, conn=4)


def test_descriptor_subsets(ctx):
    f, thr = workloads.config3(n=24, nblobs=6, L=33)
    f, thr = f.numpy(), thr.numpy()
    for desc in range(1, 16):
        check(ctx, f, thr, len(thr), desc=desc)
    g = workloads.quantize_u8(workloads.grf_2d(3, 40, 50, 2.0)).numpy()
    for desc in range(1, 8):
        check(ctx, g, None, 256, desc=desc)


def test_config1_full(ctx):
    f = workloads.config1().numpy()
    for conn in (8, 4):
        check(ctx, f, None, 256, conn=conn)


# 3D 6-connectivity: every per-voxel and per-vertex path against the oracle's
# reading (cells whose incident voxels are all active); the other descriptors
# do not depend on it.
SHAPES3_C6 = [(1, 1, 1), (2, 3, 5), (7, 11, 13), (33, 9, 31), (5, 64, 65), (16, 40, 68), (70, 3, 8)]


@pytest.mark.parametrize("shape", SHAPES3_C6)
@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_random_3d_6_connectivity(ctx, shape, dtype):
    rng = np.random.default_rng(zlib.crc32(repr((shape, dtype, "c6")).encode()))
    if dtype == "u8":
        L = int(rng.integers(1, 40))
        f = rng.integers(0, L + 3, size=shape).astype(np.uint8)
        thr = None
    elif dtype == "u16":
        L = int(rng.integers(1, 3000))
        f = rng.integers(0, L + 50, size=shape).astype(np.uint16)
        thr = None
    else:
        L = int(rng.integers(1, 200))
        f = workloads.grf_nd(int(rng.integers(1 << 30)), shape, 1.2).numpy().astype(np.float32)
        thr = np.sort(rng.normal(size=L) * f.std() + f.mean()).astype(np.float32)
    for desc in (1, 15):
        check(ctx, f, thr, L, conn=6, desc=desc)


def test_exhaustive_binary_2x2x2_6_connectivity(ctx):
    for bits in range(1 << 8):
        a = np.array([(bits >> i) & 1 for i in range(8)], np.uint8).reshape(2, 2, 2)
        check(ctx, a, None, 1, conn=6)


def test_6_connectivity_streamed_and_batched(ctx):
    f, thr = workloads.config3(n=36, nblobs=12, L=90)
    fh, th = f.numpy(), thr.numpy()
    want = oracle.ec_curves(fh, th, 90, 6, ALL3)
    for slab in (1, 7, 64):
        got = ec.curve_3d_stream(fh, thresholds=th, connectivity=6, descriptors=ALL3, slab_planes=slab, ctx=ctx)
        np.testing.assert_array_equal(got, want)
    g = np.random.default_rng(3).integers(0, 20, size=(9, 10, 11)).astype(np.uint8)
    items = [dict(field=to_dev(fh), thresholds=to_dev(th), L=90, connectivity=6, descriptors=ALL3),
             dict(field=to_dev(g), thresholds=None, L=20, connectivity=26, descriptors=1),
             dict(field=to_dev(g), thresholds=None, L=20, connectivity=6, descriptors=9)]
    outs = ec.batch(items, ctx=ctx)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(outs[0].cpu().numpy(), want)
    np.testing.assert_array_equal(outs[1].cpu().numpy(), oracle.ec_curves(g, None, 20, 26, 1))
    np.testing.assert_array_equal(outs[2].cpu().numpy(), oracle.ec_curves(g, None, 20, 6, 9))


def test_argument_errors(ctx):
    f = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    t = torch.zeros(3, dtype=torch.float32, device="cuda")
    with pytest.raises(ec.ECError) as e:
        ec.curve(f, t, connectivity=5, ctx=ctx)
    assert e.value.status == 1
    with pytest.raises(ec.ECError) as e:
        ec.curve(f, t, connectivity=8, ctx=ctx)
    assert e.value.status == 1
    with pytest.raises(ec.ECError) as e:
        ec.curve(f[0], t, descriptors=ec.EC_DESC_VOLUME, ctx=ctx)
    assert e.value.status == 1
    with pytest.raises(ec.ECError) as e:
        ec.curve(f, None, L=4, ctx=ctx)
    assert e.value.status == 2
    bad = torch.tensor([0.0, 2.0, 1.0], device="cuda")
    ctx.set_option(ec.EC_OPT_VALIDATE, 1)
    try:
        with pytest.raises(ec.ECError) as e:
            ec.curve(f, bad, ctx=ctx)
        assert e.value.status == 1
        ok = ec.curve(f, t, ctx=ctx)
        torch.cuda.synchronize()
        assert ok.shape == (1, 3)
    finally:
        ctx.set_option(ec.EC_OPT_VALIDATE, 0)
    # L == 0 is a no-op
    out = torch.full((1, 1), 7, dtype=torch.int64, device="cuda")
    ec.lib().ec_curve_3d(ctx.handle, f.data_ptr(), ec._dims(f.shape), ec.EC_F32, t.data_ptr(), 0, 26, 1,
                         out.data_ptr(), None)
    torch.cuda.synchronize()
    assert int(out[0, 0]) == 7


@pytest.mark.slow
def test_config3_full_size(ctx):
    """The benchmark workload at full size (512^3 float32, 1024 levels, all
    four descriptors), in the launch configuration the benchmark times."""
    f, thr = workloads.config3(device="cuda")
    fh, th = f.cpu().numpy(), thr.cpu().numpy()
    want = oracle.ec_curves(fh, th, 1024, 26, ALL3)
    ctx.set_option(ec.EC_OPT_ALGO, ec.ALGO_AUTO)
    ctx.set_option(ec.EC_OPT_TILE_Z, 0)
    got = ec.curve(f, thr, descriptors=ALL3, ctx=ctx)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    # the benchmarked descriptor set (EC, area, volume: its own compiled
    # instantiation), by both per-voxel forms; its rows are rows 0, 2, 3 of
    # the all-descriptor curves
    for algo in (ec.ALGO_AUTO, ec.ALGO_VOXEL):
        ctx.set_option(ec.EC_OPT_ALGO, algo)
        got13 = ec.curve(f, thr, descriptors=13, ctx=ctx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got13.cpu().numpy(), want[[0, 2, 3]], err_msg=f"algo {algo}")
    ctx.set_option(ec.EC_OPT_ALGO, ec.ALGO_AUTO)
    # invariants that hold at any size
    assert want[0, -1] == 1 and want[3, -1] == 512 ** 3


@pytest.mark.slow
def test_config2_full_size(ctx):
    u8, f32, thr = workloads.config2(device="cuda")
    want_u8 = oracle.ec_curves(u8.cpu().numpy(), None, 256, 8, ALL2)
    ctx.set_option(ec.EC_OPT_ALGO, ec.ALGO_AUTO)
    got = ec.curve(u8, None, L=256, descriptors=ALL2, ctx=ctx)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), want_u8)
    want_f = oracle.ec_curves(f32.cpu().numpy(), thr.cpu().numpy(), 1024, 8, ALL2)
    got_f = ec.curve(f32, thr, descriptors=ALL2, ctx=ctx)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got_f.cpu().numpy(), want_f)


@pytest.mark.parametrize("lo,hi,L", [(-0.21, 3.7, 1024), (0.0, 1.0, 256), (-1e3, 5e4, 4000), (1.0, 1.0001, 300)])
def test_uniform_threshold_binning_edges(ctx, lo, hi, L):
    """Values exactly on, one ulp below and one ulp above uniform thresholds,
    plus NaN, infinities and signed zeros: the spacing-based binning must
    agree with the x <= t_k definition everywhere."""
    thr = workloads.uniform_thresholds(lo, hi, L).numpy()
    rng = np.random.default_rng(L)
    picks = thr[rng.integers(0, L, size=6000)]
    special = np.array([np.nan] * 50 + [-np.inf, np.inf, -0.0, 0.0, thr[0] - 1, thr[-1] + 1], np.float32)
    vals = np.concatenate([picks, np.nextafter(picks, np.float32(np.inf)),
                           np.nextafter(picks, np.float32(-np.inf)), special]).astype(np.float32)
    f = rng.permutation(np.resize(vals, 24 * 25 * 28)).astype(np.float32).reshape(24, 25, 28)
    check(ctx, f, thr, L, algos=[ec.ALGO_PLANAR, ec.ALGO_VOXEL])


@pytest.mark.parametrize("desc", [1, 5, 13, 15, 8, 2])
def test_histogram_schedules_agree(ctx, desc):
    """One atomic per voxel and warp-aggregated updates give the oracle's curves."""
    f, thr = workloads.config3(n=72, nblobs=30, L=300)
    f, thr = f.numpy(), thr.numpy()
    want = oracle.ec_curves(f, thr, 300, 26, desc)
    try:
        for sched in (1, 2, 3, 0):
            ctx.set_option(ec.EC_OPT_HIST_SCHEDULE, sched)
            np.testing.assert_array_equal(gpu_curves(ctx, f, thr, 300, 26, desc), want, err_msg=f"schedule {sched}")
    finally:
        ctx.set_option(ec.EC_OPT_HIST_SCHEDULE, 0)
