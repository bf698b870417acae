"""Pins of the type-map oracle (oracle/typemap.py), CPU only.

Each test ties the oracle to something other than itself: the rows, pictures
and f_adj column of Tables 1 and 2 (tests/golden), the symmetry classes of the
square and the cube, the cell-counting oracle (oracle/ec_oracle.c) through
the tables' weights, closed forms and a per-vertex enumeration.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import typemap as tm
from tests import _tables

T1_ORDER = ["Q0", "Q1", "Q2", "QD", "Q3", "Q4"]


def _rand_bins(rng, shape, L):
    b = rng.integers(0, L + 1, size=shape).astype(np.int32)   # L = never active
    return b


# --------------------------------------------------------------- the types

def test_types_follow_table2_rows_and_fadj_column():
    """The representative drawn in each row of Table 2 gets that row's index,
    and its f_adj (of the empty voxels for 5-8 active, per the daggers)
    equals the printed column."""
    _, by_class = _tables.table2()
    tab = tm.type_table(3)
    assert len(by_class) == 22
    for row in by_class.values():
        assert tab[row["rep"]] == row["row"] - 1, row["row"]
        n, adj = tm.type_key(row["rep"], 3)
        assert n == bin(row["rep"]).count("1")
        assert abs(adj - float(row["fadj"])) < 6e-4, (row["row"], adj, row["fadj"])


def test_types_are_the_cube_symmetry_classes():
    """Type = orbit of the neighbourhood under the 48 symmetries of the cube:
    constant on every orbit, and distinct orbits get distinct types."""
    tab = tm.type_table(3)
    orbit = {m: _tables._orbit_min(m, 3) for m in range(256)}
    by_orbit = {}
    for m in range(256):
        by_orbit.setdefault(orbit[m], set()).add(int(tab[m]))
    assert all(len(s) == 1 for s in by_orbit.values())
    assert len({next(iter(s)) for s in by_orbit.values()}) == len(by_orbit) == 22


def test_type_class_sizes():
    """Sizes of the 22 classes in Table 2's row order (they sum to 256)."""
    sizes = np.bincount(tm.type_table(3), minlength=22)
    assert sizes.tolist() == [1, 8, 12, 12, 4, 24, 24, 8, 6, 8, 24, 24, 6, 2, 24, 24, 8, 12, 12, 4, 8, 1]
    assert np.bincount(tm.type_table(2), minlength=6).tolist() == [1, 4, 4, 2, 4, 1]


def test_types_follow_table1_rows():
    """2D: Q0, Q1, Q2, QD, Q3, Q4 in Table 1's order, each mask by its picture's class."""
    t1 = _tables.table1()
    tab = tm.type_table(2)
    for m in range(16):
        assert tab[m] == T1_ORDER.index(t1[m]["type"]), m


def test_fadj_values_of_two_cells():
    """Sec. 2.2: two voxels sharing a face, an edge or only a vertex have
    f_adj 1, sqrt 2, sqrt 3."""
    assert tm.f_adj([(0, 0, 0), (1, 0, 0)]) == 1.0
    assert abs(tm.f_adj([(0, 0, 0), (1, 1, 0)]) - math.sqrt(2)) < 1e-12
    assert abs(tm.f_adj([(0, 0, 0), (1, 1, 1)]) - math.sqrt(3)) < 1e-12


# ----------------------------------------------------------- the type map

def _weights_3d():
    """Integer weights per type from Table 2: 8 EC, 2 perimeter, 4 area (row 10
    erratum applied), 8 volume."""
    _, by_class = _tables.table2()
    rows = sorted(by_class.values(), key=lambda r: r["row"])
    W = [[int(8 * r["EC"]) for r in rows], [int(2 * r["Perim"]) for r in rows],
         [int(4 * r["AreaUsed"]) for r in rows], [int(8 * r["Volume"]) for r in rows]]
    return W, [8, 2, 4, 8]


def _weights_2d():
    t1 = _tables.table1()
    rows = [next(t1[m] for m in range(16) if t1[m]["type"] == q) for q in T1_ORDER]
    W = [[int(4 * r["EC8"]) for r in rows], [int(4 * r["EC4"]) for r in rows],
         [int(2 * r["Perim"]) for r in rows], [int(4 * r["Area"]) for r in rows]]
    return W, [4, 4, 2, 4]


@pytest.mark.parametrize("seed", range(6))
def test_weighted_type_map_equals_cell_counting_3d(seed):
    """Weighting the type map with Table 2's columns gives the EC, perimeter,
    area and volume curves that the cell-counting oracle finds."""
    rng = np.random.default_rng(100 + seed)
    shape = tuple(int(s) for s in rng.integers(1, 9, size=3))
    L = int(rng.integers(1, 9))
    bins = _rand_bins(rng, shape, L)
    counts = tm.type_map(bins, L)
    W, sc = _weights_3d()
    got = tm.apply_weights(counts, W, sc)
    ref = oracle.curves_3d(bins, L)
    for d, key in enumerate(("ec", "perimeter", "area", "volume")):
        np.testing.assert_array_equal(got[d], ref[key], err_msg=key)


@pytest.mark.parametrize("seed", range(6))
def test_weighted_type_map_equals_cell_counting_2d(seed):
    rng = np.random.default_rng(200 + seed)
    shape = tuple(int(s) for s in rng.integers(1, 17, size=2))
    L = int(rng.integers(1, 9))
    bins = _rand_bins(rng, shape, L)
    counts = tm.type_map(bins, L)
    W, sc = _weights_2d()
    got = tm.apply_weights(counts, W, sc)
    ref = oracle.curves_2d(bins, L)
    for d, key in enumerate(("ec8", "ec4", "perimeter", "area")):
        np.testing.assert_array_equal(got[d], ref[key], err_msg=key)


def _enumerate(bins, L):
    """Per-vertex, per-level enumeration straight from the definition: gather
    the cells around each vertex (outside = never active), classify the active
    set by its (count, adjacency) key, count."""
    ndim = bins.ndim
    keys = sorted({tm.type_key(m, ndim) for m in range(1 << (1 << ndim))})
    out = np.zeros((len(keys), L), np.int64)
    shape = bins.shape
    for v in itertools.product(*(range(s + 1) for s in shape)):
        cells = []
        for b in range(1 << ndim):
            off = [(b >> a) & 1 for a in range(ndim)][::-1]      # numpy axis order
            c = tuple(v[i] - 1 + off[i] for i in range(ndim))
            inside = all(0 <= c[i] < shape[i] for i in range(ndim))
            cells.append(int(bins[c]) if inside else L)
        for k in range(L):
            mask = sum(1 << b for b in range(1 << ndim) if cells[b] <= k)
            out[keys.index(tm.type_key(mask, ndim)), k] += 1
    return out


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 2), (3, 2, 4), (1, 5, 1)])
def test_type_map_matches_enumeration_3d(shape):
    rng = np.random.default_rng(sum(shape))
    L = 5
    bins = _rand_bins(rng, shape, L)
    np.testing.assert_array_equal(tm.type_map(bins, L), _enumerate(bins, L))


@pytest.mark.parametrize("shape", [(1, 1), (3, 4), (5, 2), (1, 7)])
def test_type_map_matches_enumeration_2d(shape):
    rng = np.random.default_rng(7 * sum(shape))
    L = 6
    bins = _rand_bins(rng, shape, L)
    np.testing.assert_array_equal(tm.type_map(bins, L), _enumerate(bins, L))


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 5), (2, 2, 7)])
def test_full_box_closed_form_3d(shape):
    """A full d x h x w box: 8 corner vertices of the one-voxel type (row 2),
    the vertices inside its edges of the face-pair type (row 3), inside its
    faces of the square type (row 9), inside the box of the full type (row 22)."""
    d, h, w = shape
    counts = tm.type_map(np.zeros(shape, np.int32), 2)
    exp = np.zeros(22, np.int64)
    exp[1] = 8
    exp[2] = 4 * ((d - 1) + (h - 1) + (w - 1))
    exp[8] = 2 * ((h - 1) * (w - 1) + (d - 1) * (w - 1) + (d - 1) * (h - 1))
    exp[21] = (d - 1) * (h - 1) * (w - 1)
    for k in range(2):
        np.testing.assert_array_equal(counts[:, k], exp)


@pytest.mark.parametrize("shape", [(1, 1), (4, 6)])
def test_full_box_closed_form_2d(shape):
    h, w = shape
    counts = tm.type_map(np.zeros(shape, np.int32), 1)[:, 0]
    assert counts.tolist() == [0, 4, 2 * (h - 1) + 2 * (w - 1), 0, 0, (h - 1) * (w - 1)]


def test_diagonal_pair_is_qd_and_never_active_is_empty():
    b = np.array([[0, 1], [1, 0]], np.int32)      # level 0: the two pixels on one diagonal
    counts = tm.type_map(b, 2)
    assert counts[3, 0] == 1                        # the centre vertex is QD
    assert counts[:, 1].tolist() == [0, 4, 4, 0, 0, 1]
    never = tm.type_map(np.full((3, 3, 3), 4, np.int32), 4)
    assert (never[0] == 64).all() and (never[1:] == 0).all()


def test_counts_sum_to_the_number_of_vertices():
    rng = np.random.default_rng(5)
    bins = _rand_bins(rng, (6, 5, 9), 12)
    counts = tm.type_map(bins, 12)
    assert (counts.sum(axis=0) == 7 * 6 * 10).all()


def test_axis_permutation_and_reflection_invariance():
    rng = np.random.default_rng(9)
    bins = _rand_bins(rng, (4, 5, 6), 7)
    ref = tm.type_map(bins, 7)
    for perm in itertools.permutations(range(3)):
        b = np.transpose(bins, perm)
        np.testing.assert_array_equal(tm.type_map(np.ascontiguousarray(b), 7), ref)
    np.testing.assert_array_equal(tm.type_map(np.ascontiguousarray(bins[::-1, :, ::-1]), 7), ref)


def test_single_level_equals_full_map():
    rng = np.random.default_rng(11)
    bins = _rand_bins(rng, (5, 7, 3), 9)
    full = tm.type_map(bins, 9)
    for k in (0, 4, 8):
        np.testing.assert_array_equal(tm.type_counts_at(bins, 9, k), full[:, k])


def test_apply_weights_rejects_a_non_multiple():
    counts = np.array([[1, 2], [3, 4]], np.int64)
    assert tm.apply_weights(counts, [[2, 4]], [2]).tolist() == [[7, 10]]
    with pytest.raises(ValueError):
        tm.apply_weights(counts, [[1, 0]], [2])


def test_worked_example_of_sec2_vertex_contribution():
    """The single-vertex walk-through of Sec. 2 (tests/golden fixture): the
    central vertex is born as one-face at 0, turns two-face diagonal at 1,
    then three-face, then full; the other 8 vertices of the 3 x 3 grid touch
    one or two pixels each."""
    import os
    rows, want = [], {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sec2_vertex_contribution_example.txt")
    for line in open(path):
        p = line.split()
        if not p or p[0].startswith("#"):
            continue
        if p[0] == "field":
            rows.append([int(v) for v in p[1:]])
        elif p[0] == "level":
            want[int(p[1])] = T1_ORDER.index(p[2])
    bins = np.array(rows, np.int32)
    counts = tm.type_map(bins, 4)
    center_mask = {k: sum(1 << (dx + 2 * dy) for dy in (0, 1) for dx in (0, 1) if bins[dy, dx] <= k) for k in range(4)}
    tab = tm.type_table(2)
    for k, t in want.items():
        assert tab[center_mask[k]] == t, k
    # the whole 3 x 3 vertex grid at the first two levels (the 8 outer vertices see 1 or 2 pixels)
    assert counts[:, 0].tolist() == [5, 4, 0, 0, 0, 0]
    assert counts[:, 1].tolist() == [2, 6, 0, 1, 0, 0]
    assert counts[:, 3].tolist() == [0, 4, 4, 0, 0, 1]
