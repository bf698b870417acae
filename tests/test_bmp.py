"""BMP input (Sec. 2.3 and Table 5 read their images as BMP files): the reader
on the CPU (row padding, bottom-up and top-down rows, palette and RGB
grayscale, the refusals), and on the GPU the curves of one image and of a
slice stack against the oracle on the same pixels."""
import os
import struct

import numpy as np
import pytest

from paper_2311_11740_gb300 import ec


def write_bmp(path, a, bits=8, top_down=False, palette=None, compression=0):
    """A Windows bitmap (BITMAPINFOHEADER) of uint8 gray values a [h, w]."""
    h, w = a.shape
    row = ((bits * w + 31) // 32) * 4
    if bits == 8:
        pal = palette if palette is not None else [(i, i, i) for i in range(256)]
        inverse = {g: i for i, (b, g2, r) in enumerate(pal) for g in [g2] if b == g2 == r}
        pal_bytes = b"".join(struct.pack("<BBBB", b, g, r, 0) for (b, g, r) in pal)
    else:
        pal_bytes = b""
    data = bytearray()
    rows = range(h) if top_down else range(h - 1, -1, -1)
    for y in rows:
        if bits == 8:
            line = bytes(inverse.get(int(v), 0) for v in a[y])
        else:
            px = bytes(int(v) for v in a[y] for _ in range(3 if bits == 24 else 3)) if bits == 24 else \
                b"".join(bytes((int(v), int(v), int(v), 255)) for v in a[y])
            line = px
        data += line + b"\0" * (row - len(line))
    off = 14 + 40 + len(pal_bytes)
    hdr = struct.pack("<2sIHHI", b"BM", off + len(data), 0, 0, off)
    dib = struct.pack("<IiiHHIIiiII", 40, w, -h if top_down else h, 1, bits, compression, len(data), 2835, 2835,
                      len(pal_bytes) // 4 if bits == 8 else 0, 0)
    with open(path, "wb") as f:
        f.write(hdr + dib + pal_bytes + bytes(data))


@pytest.mark.parametrize("bits", [8, 24, 32])
@pytest.mark.parametrize("top_down", [False, True])
def test_reader_round_trips(libec, tmp_path, bits, top_down):
    rng = np.random.default_rng(bits + 100 * top_down)
    for w in (1, 2, 3, 4, 5, 7, 33):
        a = rng.integers(0, 256, size=(int(rng.integers(1, 9)), w)).astype(np.uint8)
        p = str(tmp_path / f"a{w}.bmp")
        write_bmp(p, a, bits=bits, top_down=top_down)
        np.testing.assert_array_equal(ec.bmp_read(p), a)


def test_reader_palette_maps_indices_to_gray(libec, tmp_path):
    # a shuffled gray palette: the value is the entry's gray level, not the index
    perm = np.random.default_rng(3).permutation(256)
    pal = [(int(g), int(g), int(g)) for g in perm]
    a = np.arange(60, dtype=np.uint8).reshape(6, 10)
    p = str(tmp_path / "pal.bmp")
    write_bmp(p, a, bits=8, palette=pal)
    np.testing.assert_array_equal(ec.bmp_read(p), a)


def test_reader_refusals(libec, tmp_path):
    a = np.zeros((3, 4), np.uint8)
    colour = str(tmp_path / "colour.bmp")
    write_bmp(colour, a, bits=8, palette=[(i, 0, 0) for i in range(256)])
    with pytest.raises(ec.ECError) as e:
        ec.bmp_read(colour)
    assert e.value.status == 2
    comp = str(tmp_path / "rle.bmp")
    write_bmp(comp, a, bits=8, compression=1)
    with pytest.raises(ec.ECError) as e:
        ec.bmp_read(comp)
    assert e.value.status == 2
    short = str(tmp_path / "short.bmp")
    write_bmp(short, np.zeros((40, 40), np.uint8))
    with open(short, "r+b") as f:
        f.truncate(os.path.getsize(short) - 100)
    with pytest.raises(ec.ECError) as e:
        ec.bmp_read(short)
    assert e.value.status == 1
    junk = str(tmp_path / "junk.bmp")
    open(junk, "wb").write(b"PNG" + b"\0" * 100)
    with pytest.raises(ec.ECError):
        ec.bmp_read(junk)


@pytest.mark.gpu
def test_curve_2d_bmp_equals_oracle(libec, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2311_11740_gb300 import workloads
    g = workloads.quantize_u8(workloads.grf_2d(21, 131, 97, 3.0)).numpy()
    for bits, td in ((8, False), (24, True), (32, False)):
        p = str(tmp_path / f"g{bits}.bmp")
        write_bmp(p, g, bits=bits, top_down=td)
        for conn in (8, 4):
            got = ec.curve_2d_bmp(p, L=256, connectivity=conn, descriptors=7)
            np.testing.assert_array_equal(got, oracle.ec_curves(g, None, 256, conn, 7))
    thr = np.unique(np.random.default_rng(5).integers(0, 256, size=40)).astype(np.uint8)
    got = ec.curve_2d_bmp(p, thresholds=thr, descriptors=7)
    np.testing.assert_array_equal(got, oracle.ec_curves(g, thr, thr.size, 8, 7))


@pytest.mark.gpu
def test_curve_3d_bmp_stack_equals_oracle(libec, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2311_11740_gb300 import workloads
    vol = workloads.quantize_u8(workloads.grf_nd(22, (19, 45, 38), 2.0)).numpy()
    paths = []
    for z in range(vol.shape[0]):
        p = str(tmp_path / f"slice_{z:03d}.bmp")
        write_bmp(p, vol[z], bits=8, top_down=bool(z % 2))
        paths.append(p)
    want = oracle.ec_curves(vol, None, 256, 26, 15)
    for slab in (1, 3, 64):
        np.testing.assert_array_equal(ec.curve_3d_bmp(paths, L=256, descriptors=15, slab_planes=slab), want)
    np.testing.assert_array_equal(ec.curve_3d_bmp(paths, L=256, connectivity=6, descriptors=1, slab_planes=4),
                                  oracle.ec_curves(vol, None, 256, 6, 1))
    odd = str(tmp_path / "odd.bmp")
    write_bmp(odd, np.zeros((45, 37), np.uint8))
    with pytest.raises(ec.ECError) as e:
        ec.curve_3d_bmp(paths[:5] + [odd], L=256, slab_planes=2)
    assert e.value.status == 1
