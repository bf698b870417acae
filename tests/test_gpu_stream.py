"""Low-memory z-slab streaming (ec_curve_3d_stream) on the GPU: streamed
curves equal the unchunked ones and the oracle, for any slab height, from
host memory or from the on-device hash-box generator, within the memory cap."""
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


def unchunked(ctx, f_dev, thr_dev, L, desc):
    out = ec.curve(f_dev, thr_dev, L=L, descriptors=desc, ctx=ctx)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("slab", [1, 2, 7, 63, 64, 65, 200])
def test_stream_host_float_equals_unchunked(ctx, slab):
    f, thr = workloads.config3(n=70, nblobs=30, L=211)
    want = oracle.ec_curves(f.numpy(), thr.numpy(), 211, 26, ALL3)
    np.testing.assert_array_equal(unchunked(ctx, f.cuda(), thr.cuda(), 211, ALL3), want)
    host = f.pin_memory() if slab % 2 else f   # pinned and pageable sources
    got = ec.curve_3d_stream(host, thresholds=thr.numpy(), descriptors=ALL3, slab_planes=slab, ctx=ctx)
    np.testing.assert_array_equal(got, want)


def test_stream_odd_shapes_and_dtypes(ctx):
    rng = np.random.default_rng(12)
    for shape in [(1, 5, 7), (3, 1, 1), (9, 33, 17), (17, 10, 130)]:
        u = rng.integers(0, 300, size=shape).astype(np.uint16)
        want = oracle.ec_curves(u, None, 257, 26, ALL3)
        for slab in (1, 4, 100):
            got = ec.curve_3d_stream(u, L=257, descriptors=ALL3, slab_planes=slab, ctx=ctx)
            np.testing.assert_array_equal(got, want)
        b = rng.integers(0, 256, size=shape).astype(np.uint8)
        want = oracle.ec_curves(b, None, 256, 26, 1)
        np.testing.assert_array_equal(ec.curve_3d_stream(b, L=256, descriptors=1, slab_planes=3, ctx=ctx), want)


def test_hashbox_generator_matches_oracle_definition(ctx):
    # partial and whole 64 x 32 output tiles, one and several planes, origins
    # on both sides of the 16-bit coordinate wrap
    for origin, n in (((-3, 1000, 2045), (37, 19, 6)), ((0, 0, 0), (64, 32, 1)), ((65530, 7, -2), (130, 70, 3)),
                      ((5, 5, 5), (1, 1, 1)), ((100, 200, 300), (200, 33, 9))):
        dev = ec.gen_hashbox_u16(4, *origin, *n)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dev.cpu().numpy().astype(np.int32),
                                      oracle.hashbox_u16(4, *origin, *n).astype(np.int32), err_msg=repr((origin, n)))


@pytest.mark.parametrize("origin,n", [((0, 0, 0), 512), ((700, 900, 1100), 96)])
def test_hashbox_subbox_streamed_equals_unchunked_and_oracle(ctx, origin, n):
    """The streaming workload's sub-box: curves from the streamed device
    generator equal the unchunked curves of the same box and the oracle on
    the box regenerated on the CPU."""
    x0, y0, z0 = origin
    cpu = oracle.hashbox_u16(4, x0, y0, z0, n, n, n)
    want = oracle.ec_curves(cpu, None, 4096, 26, 13)
    dev = ec.gen_hashbox_u16(4, x0, y0, z0, n, n, n)
    np.testing.assert_array_equal(unchunked(ctx, dev, None, 4096, 13), want)
    spec = ec.HashboxSpec(4, x0, y0, z0, n, n)
    for slab in (1, 2, 63, 64, 65):
        got = ec.hashbox_stream(spec, n, L=4096, descriptors=13, slab_planes=slab, ctx=ctx)
        np.testing.assert_array_equal(got, want, err_msg=f"slab={slab}")


def test_stream_respects_memory_cap(ctx):
    n, nz = 256, 200
    cap = 24 << 20
    spec = ec.HashboxSpec(4, 0, 0, 0, n, n)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lows = []
    got = ec.hashbox_stream(spec, nz, L=4096, descriptors=1, slab_planes=64, device_mem_cap=cap, ctx=ctx,
                            probe=lambda z0, z1: lows.append(torch.cuda.mem_get_info()[0]))
    assert free0 - min(lows) <= cap + (2 << 20)   # allocator granularity
    want = ec.hashbox_stream(spec, nz, L=4096, descriptors=1, slab_planes=64, ctx=ctx)
    np.testing.assert_array_equal(got, want)
    with pytest.raises(ec.ECError) as e:
        ec.hashbox_stream(spec, nz, L=4096, descriptors=1, device_mem_cap=1 << 16, ctx=ctx)
    assert e.value.status == 4


@pytest.mark.slow
def test_full_2048_cube_under_4gb_cap(ctx):
    n = 2048
    cap = 4 << 30
    spec = ec.HashboxSpec(4, 0, 0, 0, n, n)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lows = []
    got = ec.hashbox_stream(spec, n, L=4096, descriptors=ec.EC_DESC_EC | ec.EC_DESC_VOLUME, slab_planes=64,
                            device_mem_cap=cap, ctx=ctx, probe=lambda z0, z1: lows.append(torch.cuda.mem_get_info()[0]))
    assert free0 - min(lows) <= cap + (2 << 20)
    # invariants at any size: every voxel is active at the top level
    assert got[0, -1] == 1
    assert got[1, -1] == n ** 3
    assert np.all(np.diff(got[1]) >= 0)
