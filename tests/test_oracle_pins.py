"""Pins for the CPU oracle (CPU only).

Each test ties the oracle to something other than itself: values the paper
prints (Tables 1 and 2), closed forms of simple shapes, Gray's bit-quad
formula, a union-find component count, a literal per-level enumeration of the
complex (oracle/brute.py), and invariants that hold for every field.
"""
import itertools

import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import brute
from tests import _tables


def curves2(field, L=None, thresholds=None):
    if L is None:
        L = int(field.max()) + 1
    return oracle.curves_2d(oracle.bin_field(field, thresholds, L), L)


def curves3(field, L=None, thresholds=None):
    if L is None:
        L = int(field.max()) + 1
    return oracle.curves_3d(oracle.bin_field(field, thresholds, L), L)


def binary2(active):
    """0 where active, 1 elsewhere; level 0 of a 1-level filtration."""
    return np.where(active, 0, 1).astype(np.uint8)


def at0_2d(active):
    c = oracle.curves_2d(oracle.bin_field(binary2(active), None, 1), 1)
    return {k: int(v[0]) for k, v in c.items()}


def at0_3d(active):
    c = oracle.curves_3d(oracle.bin_field(binary2(active), None, 1), 1)
    return {k: int(v[0]) for k, v in c.items()}


# ----------------------------------------------------------- closed forms

def test_single_pixel_and_voxel():
    a = np.zeros((5, 7), bool); a[2, 3] = True
    assert at0_2d(a) == dict(ec8=1, ec4=1, perimeter=4, area=1)
    v = np.zeros((4, 5, 6), bool); v[1, 2, 3] = True
    assert at0_3d(v) == dict(ec=1, perimeter=12, area=6, volume=1)


def test_annulus_and_solid_torus():
    a = np.zeros((7, 8), bool); a[1:6, 1:7] = True; a[2:5, 2:6] = False
    r = at0_2d(a)
    assert r["ec8"] == 0 and r["ec4"] == 0
    assert r["area"] == int(a.sum())
    # outer boundary 2*(5+6), inner boundary 2*(3+4)
    assert r["perimeter"] == 22 + 14
    # solid torus: a square ring of voxels, thickness 2 in z
    v = np.zeros((4, 8, 8), bool); v[1:3, 1:7, 1:7] = True; v[1:3, 3:5, 3:5] = False
    r3 = at0_3d(v)
    assert r3["ec"] == 0 and r3["volume"] == int(v.sum())


def test_hollow_cube_shell():
    v = np.zeros((7, 7, 7), bool); v[1:6, 1:6, 1:6] = True; v[2:5, 2:5, 2:5] = False
    r = at0_3d(v)
    assert r["ec"] == 2
    # outer surface 6*25 + inner cavity surface 6*9
    assert r["area"] == 6 * 25 + 6 * 9


def test_disjoint_blobs_count():
    rng = np.random.default_rng(7)
    a = np.zeros((40, 40), bool)
    n = 0
    for by in range(0, 40, 8):
        for bx in range(0, 40, 8):
            if rng.random() < 0.6:
                h, w = rng.integers(1, 6, size=2)
                a[by + 1:by + 1 + h, bx + 1:bx + 1 + w] = True
                n += 1
    r = at0_2d(a)
    assert r["ec8"] == n and r["ec4"] == n
    v = np.zeros((24, 24, 24), bool)
    m = 0
    for bz, by, bx in itertools.product(range(0, 24, 6), repeat=3):
        if rng.random() < 0.5:
            s = rng.integers(1, 4, size=3)
            v[bz + 1:bz + 1 + s[0], by + 1:by + 1 + s[1], bx + 1:bx + 1 + s[2]] = True
            m += 1
    assert at0_3d(v)["ec"] == m


def test_diagonal_pixels_connectivity():
    a = np.zeros((4, 4), bool); a[1, 1] = a[2, 2] = True
    r = at0_2d(a)
    assert r["ec8"] == 1 and r["ec4"] == 2      # Table 1, row QD: V(8-C)=1, V(4-C)=2
    assert r["perimeter"] == 8


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (16, 9), (2, 31)])
def test_full_box_2d(shape):
    h, w = shape
    r = at0_2d(np.ones(shape, bool))
    assert r == dict(ec8=1, ec4=1, perimeter=2 * (h + w), area=h * w)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (5, 1, 7), (6, 6, 6)])
def test_full_box_3d(shape):
    d, h, w = shape
    r = at0_3d(np.ones(shape, bool))
    assert r == dict(ec=1, perimeter=4 * (d + h + w), area=2 * (w * h + h * d + w * d),
                     volume=d * h * w)


def test_all_inactive_is_zero():
    assert at0_2d(np.zeros((5, 6), bool)) == dict(ec8=0, ec4=0, perimeter=0, area=0)
    assert at0_3d(np.zeros((3, 4, 5), bool)) == dict(ec=0, perimeter=0, area=0, volume=0)


@pytest.mark.parametrize("k", [1, 2, 5, 8])
def test_checkerboard(k):
    a = (np.add.outer(np.arange(k), np.arange(k)) % 2 == 0)
    r = at0_2d(a)
    # 8-C: every active pixel touches its diagonal neighbours -> one component,
    # and the inactive pixels are 4-isolated holes in the interior.
    lab8, n8 = ndimage.label(a, structure=np.ones((3, 3)))
    assert r["ec8"] == n8 - _holes(a, bg_struct=ndimage.generate_binary_structure(2, 1))
    assert r["ec4"] == int(a.sum()) - _holes(a, bg_struct=np.ones((3, 3)))


# ------------------------------------------------------------ Gray's formula

def _quads(active):
    p = np.pad(active, 1).astype(np.int64)
    q = p[:-1, :-1] + 2 * p[:-1, 1:] + 4 * p[1:, :-1] + 8 * p[1:, 1:]
    n1 = np.isin(q, [1, 2, 4, 8]).sum()
    n3 = np.isin(q, [7, 11, 13, 14]).sum()
    nd = np.isin(q, [6, 9]).sum()
    return n1, n3, nd


@pytest.mark.parametrize("seed", range(6))
def test_gray_bit_quad_formula(seed):
    """Gray (1971), cited by the paper for the bit-quad neighbourhood:
    chi8 = (n1 - n3 - 2 nD) / 4, chi4 = (n1 - n3 + 2 nD) / 4 over the
    zero-padded 2x2 quads of a binary image."""
    rng = np.random.default_rng(seed)
    a = rng.random((37, 53)) < rng.uniform(0.2, 0.8)
    n1, n3, nd = _quads(a)
    r = at0_2d(a)
    assert 4 * r["ec8"] == n1 - n3 - 2 * nd
    assert 4 * r["ec4"] == n1 - n3 + 2 * nd


# ------------------------------------------------------- union-find counting

def _holes(a, bg_struct):
    pad = np.pad(~a, 1, constant_values=True)
    lab, n = ndimage.label(pad, structure=bg_struct)
    border = set(np.unique(np.concatenate([lab[0], lab[-1], lab[:, 0], lab[:, -1]])))
    return n - len(border - {0})


@pytest.mark.parametrize("seed", range(6))
def test_components_minus_holes(seed):
    rng = np.random.default_rng(100 + seed)
    a = rng.random((45, 38)) < rng.uniform(0.3, 0.7)
    r = at0_2d(a)
    _, n8 = ndimage.label(a, structure=np.ones((3, 3)))
    _, n4 = ndimage.label(a, structure=ndimage.generate_binary_structure(2, 1))
    assert r["ec8"] == n8 - _holes(a, ndimage.generate_binary_structure(2, 1))
    assert r["ec4"] == n4 - _holes(a, np.ones((3, 3)))


# ---------------------------------------------------------------- brute force

def test_exhaustive_binary_3x3_images():
    for bits in range(1 << 9):
        a = np.array([(bits >> i) & 1 for i in range(9)], bool).reshape(3, 3)
        f = binary2(a)
        o = oracle.curves_2d(oracle.bin_field(f, None, 1), 1)
        b = brute.curves_2d(f, [0])
        for key in o:
            assert o[key][0] == b[key][0], (bits, key)


@pytest.mark.parametrize("seed", range(12))
def test_random_multilevel_2d_vs_brute(seed):
    rng = np.random.default_rng(seed)
    h, w = rng.integers(1, 7, size=2)
    L = int(rng.integers(1, 6))
    f = rng.integers(0, L + 2, size=(h, w)).astype(np.uint8)
    o = curves2(f, L)
    b = brute.curves_2d(f, range(L))
    for key in o:
        np.testing.assert_array_equal(o[key], b[key], err_msg=key)


@pytest.mark.parametrize("seed", range(10))
def test_random_multilevel_3d_vs_brute(seed):
    rng = np.random.default_rng(50 + seed)
    d, h, w = rng.integers(1, 5, size=3)
    L = int(rng.integers(1, 5))
    f = rng.integers(0, L + 1, size=(d, h, w)).astype(np.uint8)
    o = curves3(f, L)
    b = brute.curves_3d(f, range(L))
    for key in o:
        np.testing.assert_array_equal(o[key], b[key], err_msg=key)


def test_float_field_vs_brute_with_special_values():
    rng = np.random.default_rng(3)
    f = rng.normal(size=(3, 4, 3)).astype(np.float32)
    f[0, 0, 0] = np.nan
    f[1, 2, 1] = -0.0
    f[2, 3, 2] = np.inf
    f[0, 1, 2] = -np.inf
    t = np.array([-1.0, 0.0, 0.0, 0.5, 2.0], np.float32)   # duplicate level
    o = curves3(f, len(t), t)
    b = brute.curves_3d(f, t)
    for key in o:
        np.testing.assert_array_equal(o[key], b[key], err_msg=key)


# -------------------------------------------------- Tables 1 and 2 of the paper

def test_table2_classes_cover_all_configurations():
    full, by_class = _tables.table2()
    assert len(by_class) == 22
    sizes = {}
    for m in range(256):
        sizes[full[m]["row"]] = sizes.get(full[m]["row"], 0) + 1
    assert sum(sizes.values()) == 256
    assert [sizes[r] for r in range(1, 23)] == [1, 8, 12, 12, 4, 24, 24, 8, 6, 8, 24, 24, 6, 2,
                                                 24, 24, 8, 12, 12, 4, 8, 1]


def test_table2_rows_consistent_with_ec_formula():
    """Every printed row satisfies EC = V - E + F - Vox (Eq. EC_formula)."""
    _, by_class = _tables.table2()
    for row in by_class.values():
        assert row["EC"] == row["V"] - row["E"] + row["F"] - row["Vox"], row["row"]


def _vertex_masks_3d(active):
    d, h, w = active.shape
    p = np.pad(active, 1).astype(np.int64)
    m = np.zeros((d + 1, h + 1, w + 1), np.int64)
    for dz, dy, dx in itertools.product((0, 1), repeat=3):
        m |= p[dz:dz + d + 1, dy:dy + h + 1, dx:dx + w + 1] << (dx + 2 * dy + 4 * dz)
    return m


@pytest.mark.parametrize("seed", range(8))
def test_oracle_equals_sum_of_table2_rows(seed):
    """Summing Table 2's per-vertex values over every grid vertex (with the
    row-10 area erratum applied) equals the oracle's cell counts."""
    full, _ = _tables.table2()
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in rng.integers(1, 9, size=3))
    a = rng.random(shape) < rng.uniform(0.15, 0.85)
    masks = _vertex_masks_3d(a).ravel()
    tot = {k: sum(full[int(m)][k] for m in masks) for k in ("EC", "Perim", "AreaUsed", "Volume")}
    r = at0_3d(a)
    assert tot["EC"] == r["ec"]
    assert tot["Perim"] == r["perimeter"]
    assert tot["AreaUsed"] == r["area"]
    assert tot["Volume"] == r["volume"]


def test_table2_row10_area_erratum_is_detected():
    """The printed area of row 10 (1.75) cannot be right: the oracle, summed
    over a field made of that configuration alone, gives 1.5 per vertex."""
    full, by_class = _tables.table2()
    row10 = next(r for r in by_class.values() if r["row"] == 10)
    assert row10["Area"] != row10["AreaUsed"]
    # a field that is exactly the tripod; its total surface is the sum over all vertices
    a = np.zeros((2, 2, 2), bool)
    for bit in range(8):
        if row10["rep"] >> bit & 1:
            a[bit >> 2 & 1, bit >> 1 & 1, bit & 1] = True
    masks = _vertex_masks_3d(a).ravel()
    printed = sum(full[int(m)]["Area"] for m in masks)
    used = sum(full[int(m)]["AreaUsed"] for m in masks)
    assert at0_3d(a)["area"] == used == 4 * 6 - 2 * 3
    assert printed != used


@pytest.mark.parametrize("seed", range(8))
def test_oracle_equals_sum_of_table1_rows(seed):
    t1 = _tables.table1()
    rng = np.random.default_rng(seed)
    h, w = (int(s) for s in rng.integers(1, 20, size=2))
    a = rng.random((h, w)) < rng.uniform(0.15, 0.85)
    p = np.pad(a, 1).astype(np.int64)
    m = p[:-1, :-1] | p[:-1, 1:] << 1 | p[1:, :-1] << 2 | p[1:, 1:] << 3
    r = at0_2d(a)
    for key, col in (("ec8", "EC8"), ("ec4", "EC4"), ("perimeter", "Perim"), ("area", "Area")):
        assert sum(t1[int(q)][col] for q in m.ravel()) == r[key], key


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(4))
def test_area_volume_are_counts_and_top_level(seed):
    rng = np.random.default_rng(seed)
    f2 = rng.integers(0, 30, size=(23, 17)).astype(np.uint8)
    c2 = curves2(f2, 30)
    bins2 = oracle.bin_field(f2, None, 30)
    for k in range(30):
        assert c2["area"][k] == int((bins2 <= k).sum())
    assert c2["ec8"][-1] == 1 and c2["perimeter"][-1] == 2 * (23 + 17)
    f3 = rng.normal(size=(9, 11, 7)).astype(np.float32)
    t = np.linspace(f3.min(), f3.max(), 40).astype(np.float32)
    t[-1] = f3.max()
    c3 = curves3(f3, 40, t)
    for k in range(40):
        assert c3["volume"][k] == int((f3 <= t[k]).sum())
    assert c3["ec"][-1] == 1
    assert c3["area"][-1] == 2 * (9 * 11 + 11 * 7 + 9 * 7)
    assert c3["perimeter"][-1] == 4 * (9 + 11 + 7)


def test_axis_permutation_and_reflection_invariance():
    rng = np.random.default_rng(11)
    f = rng.integers(0, 12, size=(6, 8, 5)).astype(np.uint8)
    base = curves3(f, 12)
    for perm in itertools.permutations(range(3)):
        g = np.ascontiguousarray(np.transpose(f, perm)[::-1, :, ::-1])
        c = curves3(g, 12)
        for key in base:
            np.testing.assert_array_equal(c[key], base[key], err_msg=str(perm))
    f2 = rng.integers(0, 9, size=(11, 6)).astype(np.uint8)
    b2 = curves2(f2, 9)
    for g in (f2.T, f2[::-1], f2[:, ::-1], f2.T[::-1]):
        c = curves2(np.ascontiguousarray(g), 9)
        for key in b2:
            np.testing.assert_array_equal(c[key], b2[key], err_msg=key)


def test_curves_change_only_at_hit_levels():
    rng = np.random.default_rng(5)
    f = (rng.integers(0, 8, size=(10, 10, 10)) * 3).astype(np.uint8)   # values 0,3,...,21
    c = curves3(f, 24)
    for key, v in c.items():
        for k in range(1, 24):
            if k % 3 != 0:
                assert v[k] == v[k - 1], (key, k)


# ------------------------------------------------------------------- binning

def test_binning_matches_searchsorted_semantics():
    """bin(x) = min{k : x <= t_k} (Eq. sublevel_set); NaN never active;
    -0.0 == +0.0; duplicates allowed."""
    x = np.array([np.nan, -np.inf, np.inf, -0.0, 0.0, 1.0, 1.5, 2.0, 3.0, -5.0], np.float32)
    t = np.array([-1.0, 0.0, 1.0, 1.0, 2.0], np.float32)
    b = oracle.bin_field(x, t, len(t))
    exp = np.searchsorted(t, x, side="left")
    exp[np.isnan(x)] = len(t)
    np.testing.assert_array_equal(b, exp)
    u = np.array([0, 5, 255, 7], np.uint8)
    np.testing.assert_array_equal(oracle.bin_field(u, None, 6), [0, 5, 6, 6])
    tu = np.array([2, 5, 5, 200], np.uint8)
    np.testing.assert_array_equal(oracle.bin_field(u, tu, 4), [0, 1, 4, 3])


# ------------------------------------------------------------ hash-box field

def _fmix32(u):
    u ^= u >> 16
    u = (u * 0x85EBCA6B) & 0xFFFFFFFF
    u ^= u >> 13
    u = (u * 0xC2B2AE35) & 0xFFFFFFFF
    return u ^ (u >> 16)


def test_hashbox_matches_definition():
    seed = (7 << 32) | 4
    a = _fmix32((seed & 0xFFFFFFFF) ^ _fmix32(seed >> 32))
    got = oracle.hashbox_u16(seed, -3, 5, 2046, 4, 3, 2)
    for k, j, i in itertools.product(range(2), range(3), range(4)):
        x, y, z = -3 + i, 5 + j, 2046 + k
        s = 0
        for dz, dy, dx in itertools.product(range(-2, 3), repeat=3):
            hz = _fmix32(a ^ ((z + dz) & 0xFFFFFFFF))
            hy = _fmix32(hz ^ ((y + dy) & 0xFFFFFFFF))
            u = _fmix32(hy ^ (((x + dx) // 2) & 0xFFFFFFFF))
            s += (u >> 16) if (x + dx) % 2 else (u & 0xFFFF)
        assert got[k, j, i] == (s * 4096) // (125 * 65536)
    assert got.max() < 4096
