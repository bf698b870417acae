"""GPU parity of the contribution-type map (ec_type_map) and of weighted
curves (ec_apply_weights) against the CPU oracle (oracle/typemap.py).
Counts are integers: the tolerance is zero."""
import zlib

import numpy as np
import pytest
import torch

import oracle
from oracle import typemap as tm
from paper_2311_11740_gb300 import ec, workloads
from tests import _tables

pytestmark = pytest.mark.gpu

ALL2 = ec.EC_DESC_EC | ec.EC_DESC_PERIMETER | ec.EC_DESC_AREA
ALL3 = ALL2 | ec.EC_DESC_VOLUME


@pytest.fixture(scope="module")
def ctx(libec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = ec.Context(0)
    yield c
    c.close()


def to_dev(a):
    if a is None:
        return None
    if a.dtype == np.uint16:
        return torch.from_numpy(a.astype(np.int32)).cuda().to(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_map(ctx, field, thr, L):
    out = ec.type_map(to_dev(field), to_dev(thr), L=L, ctx=ctx)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(ctx, field, thr, L):
    want = tm.type_map(oracle.bin_field(field, thr, L), L)
    got = gpu_map(ctx, field, thr, L)
    np.testing.assert_array_equal(got, want, err_msg=f"shape={field.shape} dtype={field.dtype} L={L}")


def rand_field(rng, shape, dtype, L):
    if dtype == "u8":
        return rng.integers(0, L + 3, size=shape).astype(np.uint8), None
    if dtype == "u16":
        f = rng.integers(0, L + 50, size=shape).astype(np.uint16)
        thr = None if rng.random() < 0.5 else np.sort(rng.integers(0, L + 60, size=L)).astype(np.uint16)
        return f, thr
    f = rng.standard_normal(size=shape).astype(np.float32)
    f.flat[rng.integers(0, f.size, size=max(1, f.size // 50))] = np.nan
    thr = np.sort(rng.standard_normal(L)).astype(np.float32)
    return f, thr


# vertex tiles are 32 x 16 (x, y) and 32 planes deep in 3D, 512 wide and 64 rows in 2D
SHAPES3 = [(1, 1, 1), (1, 1, 9), (2, 3, 5), (31, 7, 31), (32, 8, 32), (33, 9, 40), (40, 17, 66), (5, 70, 3)]
SHAPES2 = [(1, 1), (1, 300), (63, 255), (64, 256), (130, 520), (300, 7)]


@pytest.mark.parametrize("shape", SHAPES3)
@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_random_3d(ctx, shape, dtype):
    rng = np.random.default_rng(zlib.crc32(repr(("tm3", shape, dtype)).encode()))
    L = int(rng.integers(1, 60))
    f, thr = rand_field(rng, shape, dtype, L)
    check(ctx, f, thr, L)


@pytest.mark.parametrize("shape", SHAPES2)
@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_random_2d(ctx, shape, dtype):
    rng = np.random.default_rng(zlib.crc32(repr(("tm2", shape, dtype)).encode()))
    L = int(rng.integers(1, 60))
    f, thr = rand_field(rng, shape, dtype, L)
    check(ctx, f, thr, L)


@pytest.mark.parametrize("L", [1, 2, 255, 1024])
def test_level_counts_3d_shared_histogram(ctx, L):
    """Up to the shared-memory budget (rows of 23 int32 x 1113 levels) the block
    histograms live in shared memory."""
    rng = np.random.default_rng(L)
    f = rng.random((20, 11, 37)).astype(np.float32)
    thr = np.sort(rng.random(L)).astype(np.float32)
    check(ctx, f, thr, L)


@pytest.mark.parametrize("L", [1200, 4096])
def test_many_levels_3d_global_histogram(ctx, L):
    """Beyond the shared-memory budget the kernel adds into the global histogram."""
    rng = np.random.default_rng(L)
    f = rng.integers(0, L, size=(6, 9, 35)).astype(np.uint16)
    check(ctx, f, None, L)


@pytest.mark.parametrize("L", [4096, 6000])
def test_many_levels_2d(ctx, L):
    rng = np.random.default_rng(L + 1)
    f = rng.integers(0, L, size=(40, 300)).astype(np.uint16)
    check(ctx, f, None, L)


def test_smooth_field_with_many_ties(ctx):
    """A quantised smooth field: most neighbourhoods share levels, so equal
    levels must merge."""
    f = workloads.grf_nd(3, (40, 48, 36), 3.0).numpy()
    q = np.clip((f - f.min()) / (f.max() - f.min()) * 12, 0, 12).astype(np.uint8)
    check(ctx, q, None, 13)


def test_exhaustive_binary_2x2x2(ctx):
    """Every 2x2x2 binary field: 27 vertices, one level."""
    for bits in range(256):
        a = np.array([(bits >> i) & 1 for i in range(8)], np.uint8).reshape(2, 2, 2)
        check(ctx, a, None, 1)


def test_columns_sum_to_vertices_and_empty_type(ctx):
    f = np.full((4, 5, 6), 7, np.uint8)          # every voxel above the levels
    got = gpu_map(ctx, f, None, 5)
    assert (got[0] == 5 * 6 * 7).all() and (got[1:] == 0).all()


def _table2_weights():
    _, by_class = _tables.table2()
    rows = sorted(by_class.values(), key=lambda r: r["row"])
    W = [[int(8 * r["EC"]) for r in rows], [int(2 * r["Perim"]) for r in rows],
         [int(4 * r["AreaUsed"]) for r in rows], [int(8 * r["Volume"]) for r in rows]]
    return np.array(W, np.int32), [8, 2, 4, 8]


def _table1_weights():
    t1 = _tables.table1()
    order = ["Q0", "Q1", "Q2", "QD", "Q3", "Q4"]
    rows = [next(t1[m] for m in range(16) if t1[m]["type"] == q) for q in order]
    W = [[int(4 * r["EC8"]) for r in rows], [int(4 * r["EC4"]) for r in rows],
         [int(2 * r["Perim"]) for r in rows], [int(4 * r["Area"]) for r in rows]]
    return np.array(W, np.int32), [4, 4, 2, 4]


def test_weights_give_the_curves_3d(ctx):
    rng = np.random.default_rng(17)
    f, thr = rand_field(rng, (30, 20, 45), "f32", 50)
    counts = ec.type_map(to_dev(f), to_dev(thr), ctx=ctx)
    W, sc = _table2_weights()
    got = ec.apply_weights(counts, W, sc, ctx=ctx).cpu().numpy()
    want = oracle.ec_curves(f, thr, 50, 26, ALL3)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(got, tm.apply_weights(counts.cpu().numpy(), W, sc))


def test_6_connected_weight_row_gives_the_6_connected_curve(ctx):
    """The library's 6-connected vertex table, taken per type, weights the
    type map into the 6-connected EC curve (the connectivity changes only the
    weights)."""
    rng = np.random.default_rng(18)
    f, thr = rand_field(rng, (26, 21, 33), "f32", 40)
    counts = ec.type_map(to_dev(f), to_dev(thr), ctx=ctx)
    tt, t6 = ec.type_table(3), ec.vertex_table_3d_ec6()
    W = np.array([[int(t6[int(np.flatnonzero(tt == t)[0])]) for t in range(ec.NTYPES[3])]], np.int32)
    got = ec.apply_weights(counts, W, [8], ctx=ctx).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.ec_curves(f, thr, 40, 6, 1))


def test_weights_give_the_curves_2d_both_connectivities(ctx):
    rng = np.random.default_rng(19)
    f, _ = rand_field(rng, (90, 333), "u8", 40)
    counts = ec.type_map(to_dev(f), None, L=40, ctx=ctx)
    W, sc = _table1_weights()
    got = ec.apply_weights(counts, W, sc, ctx=ctx).cpu().numpy()
    c = oracle.curves_2d(oracle.bin_field(f, None, 40), 40)
    for d, key in enumerate(("ec8", "ec4", "perimeter", "area")):
        np.testing.assert_array_equal(got[d], c[key], err_msg=key)


def test_weights_not_a_multiple_are_reported(ctx):
    f = np.zeros((3, 3, 3), np.uint8)
    counts = ec.type_map(to_dev(f), None, L=2, ctx=ctx)
    W = np.zeros((1, 22), np.int32)
    W[0, 1] = 1                                   # 8 corner vertices
    out = ec.apply_weights(counts, W, [3], ctx=ctx).cpu().numpy()
    assert (out == np.iinfo(np.int64).min).all()
    ctx.set_option(ec.EC_OPT_VALIDATE, 1)
    try:
        with pytest.raises(ec.ECError):
            ec.apply_weights(counts, W, [3], ctx=ctx)
        assert ec.apply_weights(counts, W, [4], ctx=ctx).cpu().numpy().tolist() == [[2, 2]]
    finally:
        ctx.set_option(ec.EC_OPT_VALIDATE, 0)


def test_weight_sums_are_exact_past_32_bits(ctx):
    """128-bit accumulation: large weights on large counts stay exact, and a
    sum beyond int64 is poisoned rather than wrapped."""
    rng = np.random.default_rng(23)
    f = rng.integers(0, 4, size=(50, 60, 70)).astype(np.uint8)
    counts = ec.type_map(to_dev(f), None, L=4, ctx=ctx)
    c = counts.cpu().numpy()
    W = rng.integers(-2**31, 2**31 - 1, size=(3, 22)).astype(np.int32)
    got = ec.apply_weights(counts, W, None, ctx=ctx).cpu().numpy()
    np.testing.assert_array_equal(got, tm.apply_weights(c, W, [1, 1, 1]))
    big = torch.full((22, 2), 2**40, dtype=torch.int64, device="cuda")
    Wb = np.full((1, 22), 2**31 - 1, np.int32)
    assert (ec.apply_weights(big, Wb, None, ctx=ctx).cpu().numpy() == np.iinfo(np.int64).min).all()


def test_argument_errors(ctx):
    f = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(ec.ECError):
        ec.type_map(f, None, L=70000, ctx=ctx)
    with pytest.raises(ec.ECError):
        ec.type_map(torch.zeros((4, 4), dtype=torch.float32, device="cuda"), None, L=3, ctx=ctx)   # f32 needs thresholds
    counts = ec.type_map(f, None, L=3, ctx=ctx)
    with pytest.raises(ec.ECError):
        ec.apply_weights(counts, np.ones((1, 22), np.int32), [0], ctx=ctx)
    with pytest.raises(ec.ECError):
        ec.apply_weights(counts, np.ones((17, 22), np.int32), None, ctx=ctx)


def test_full_size_benchmark_field(ctx):
    """The 512^3 float32 benchmark field with 1024 levels: sampled levels
    equal the oracle's one-level counts, every column sums to the vertices,
    and Table 2's weights give the library's own curves."""
    field, thr = workloads.config3(device="cuda")
    L = thr.numel()
    counts = ec.type_map(field, thr, ctx=ctx)
    W, sc = _table2_weights()
    curves = ec.apply_weights(counts, W, sc, ctx=ctx)
    ctx.set_option(ec.EC_OPT_ALGO, ec.ALGO_AUTO)
    ref = ec.curve(field, thr, descriptors=ALL3, ctx=ctx)
    torch.cuda.synchronize()
    assert torch.equal(curves, ref)
    c = counts.cpu().numpy()
    assert (c.sum(axis=0) == 513 ** 3).all()
    bins = oracle.bin_field(field.cpu().numpy(), thr.cpu().numpy(), L)
    for k in (0, 137, 600, L - 1):
        np.testing.assert_array_equal(c[:, k], tm.type_counts_at(bins, L, k), err_msg=f"level {k}")
