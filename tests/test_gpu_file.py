"""Low-memory streaming straight from a raw file (ec_curve_3d_file) on the
GPU: curves equal the oracle's for any slab height, offset and dtype, within
the memory cap; unreadable or short files are reported."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_11740_gb300 import ec, workloads

pytestmark = pytest.mark.gpu
ALL3 = 15


@pytest.fixture(scope="module")
def ctx(libec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ec.Context(0)


def write_raw(path, arr, offset=0):
    with open(path, "wb") as fh:
        fh.write(bytes(range(offset % 256)) * (offset // 256) + bytes(range(offset % 256)))
        fh.seek(offset)
        fh.write(np.ascontiguousarray(arr).tobytes())


@pytest.mark.parametrize("slab", [1, 3, 64, 200])
@pytest.mark.parametrize("offset", [0, 13])
def test_file_float_equals_oracle(ctx, tmp_path, slab, offset):
    f, thr = workloads.config3(n=70, nblobs=30, L=211)
    a = f.numpy()
    path = tmp_path / "field.raw"
    write_raw(path, a, offset)
    want = oracle.ec_curves(a, thr.numpy(), 211, 26, ALL3)
    got = ec.curve_3d_file(str(path), a.shape, np.float32, thresholds=thr.numpy(), offset=offset,
                           descriptors=ALL3, slab_planes=slab, ctx=ctx)
    np.testing.assert_array_equal(got, want)


def test_file_integer_dtypes_and_odd_shapes(ctx, tmp_path):
    rng = np.random.default_rng(31)
    for shape in [(1, 5, 7), (9, 33, 17), (40, 64, 65)]:
        u = rng.integers(0, 300, size=shape).astype(np.uint16)
        p = tmp_path / "u16.raw"
        write_raw(p, u)
        want = oracle.ec_curves(u, None, 257, 26, ALL3)
        for slab in (1, 5, 100):
            got = ec.curve_3d_file(str(p), shape, np.uint16, L=257, descriptors=ALL3, slab_planes=slab, ctx=ctx)
            np.testing.assert_array_equal(got, want)
        b = rng.integers(0, 256, size=shape).astype(np.uint8)
        p = tmp_path / "u8.raw"
        write_raw(p, b, offset=7)
        want = oracle.ec_curves(b, None, 256, 26, 1)
        got = ec.curve_3d_file(str(p), shape, np.uint8, L=256, offset=7, descriptors=1, slab_planes=3, ctx=ctx)
        np.testing.assert_array_equal(got, want)


def test_file_large_slabs_read_by_several_threads(ctx, tmp_path):
    """Slabs of 4 MiB and more are split across reader threads."""
    rng = np.random.default_rng(37)
    a = rng.standard_normal((40, 512, 512)).astype(np.float32)   # 1 MiB planes
    thr = np.sort(rng.standard_normal(300)).astype(np.float32)
    p = tmp_path / "big.raw"
    write_raw(p, a, offset=5)
    want = oracle.ec_curves(a, thr, 300, 26, ALL3)
    for slab in (17, 40):    # 18-19 planes per slab read by 4 threads; the whole field by 8
        got = ec.curve_3d_file(str(p), a.shape, np.float32, thresholds=thr, offset=5, descriptors=ALL3,
                               slab_planes=slab, ctx=ctx)
        np.testing.assert_array_equal(got, want)


def test_file_respects_memory_cap(ctx, tmp_path):
    rng = np.random.default_rng(41)
    a = rng.integers(0, 1000, size=(30, 40, 50)).astype(np.uint16)
    p = tmp_path / "cap.raw"
    write_raw(p, a)
    want = oracle.ec_curves(a, None, 1000, 26, 1)
    plane = 40 * 50 * 2
    cap = 3 * 2 * plane * 2 + 64 * 1024     # room for slabs of a few planes only
    got = ec.curve_3d_file(str(p), a.shape, np.uint16, L=1000, descriptors=1, slab_planes=64,
                           device_mem_cap=cap, ctx=ctx)
    np.testing.assert_array_equal(got, want)


def test_file_errors(ctx, tmp_path):
    with pytest.raises(ec.ECError, match="cannot open"):
        ec.curve_3d_file(str(tmp_path / "missing.raw"), (2, 2, 2), np.uint8, L=4, ctx=ctx)
    p = tmp_path / "short.raw"
    write_raw(p, np.zeros((2, 3, 4), np.uint8))
    with pytest.raises(ec.ECError, match="holds 24 bytes"):
        ec.curve_3d_file(str(p), (3, 3, 4), np.uint8, L=4, ctx=ctx)
    with pytest.raises(ec.ECError, match="holds 24 bytes"):
        ec.curve_3d_file(str(p), (2, 3, 4), np.uint8, L=4, offset=1, ctx=ctx)
    # exactly the field: fine
    got = ec.curve_3d_file(str(p), (2, 3, 4), np.uint8, L=4, ctx=ctx)
    assert got.shape == (1, 4) and (got == 1).all()
