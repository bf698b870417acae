"""Pins of the 6-connected EC reading (CPU only).

Reading: under face adjacency a cell of the cubical grid is in the complex
when ALL its incident voxels are active (cells enter at the maximum of the
incident levels), so chi6 = #voxels - #face pairs + #2x2 squares - #cubes.
What fixes it without trusting the oracle's own formula:
  * chi = b0 - b1 + b2 on every 2x2x2 binary image: b0 from 6-connected
    component counts (scipy.ndimage.label), no cavities (every background
    voxel touches the outside), and a tunnel exactly when the six active
    voxels ring a main diagonal (the two inactive ones opposite corners);
  * the duality with the complement: in a box padded by one layer of
    background, chi6(F) = chi26(complement) - 1 (chi26 from the closed-complex
    oracle, pinned by Tables 1 and 2 elsewhere);
  * the same reading in 2D equals the 4-connected EC of Table 1 (the oracle's
    4-C column, pinned by brute force and Gray's formula elsewhere);
  * closed forms: contacts along an edge or at a vertex separate, a hollow
    shell has chi 2, a ring of voxels chi 0, a box chi 1, nothing chi 0.
"""
import numpy as np
import pytest

import oracle

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def chi6_binary(a):
    """chi6 of a binary 3D image (active = 1) through the oracle."""
    return int(oracle.ec6_3d(np.where(a.astype(bool), 0, 1).astype(np.int32), 1)[0])


def chi26_binary(a):
    return int(oracle.curves_3d(np.where(a.astype(bool), 0, 1).astype(np.int32), 1)["ec"][0])


def test_every_2x2x2_image_is_components_minus_tunnels():
    structure = scipy_ndimage.generate_binary_structure(3, 1)   # face adjacency
    tunnels_seen = 0
    for bits in range(256):
        a = np.array([(bits >> i) & 1 for i in range(8)], np.uint8).reshape(2, 2, 2)
        _, ncomp = scipy_ndimage.label(a, structure=structure)
        off = [i for i in range(8) if not (bits >> i) & 1]
        tunnel = len(off) == 2 and (off[0] ^ off[1]) == 7   # opposite corners: a ring of six
        tunnels_seen += tunnel
        assert chi6_binary(a) == ncomp - int(tunnel), bits
    assert tunnels_seen == 4


def test_duality_with_the_complement_on_random_binary_images():
    rng = np.random.default_rng(61)
    for trial in range(300):
        shape = tuple(int(v) for v in rng.integers(1, 6, size=3))
        a = (rng.random(shape) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        padded = np.zeros(tuple(s + 2 for s in shape), np.uint8)
        padded[1:-1, 1:-1, 1:-1] = a
        assert chi6_binary(a) == chi26_binary(1 - padded) - 1, (trial, shape)


def test_every_level_of_a_multi_level_field_is_its_binary_image():
    rng = np.random.default_rng(62)
    for trial in range(40):
        shape = tuple(int(v) for v in rng.integers(1, 7, size=3))
        L = int(rng.integers(1, 9))
        bins = rng.integers(0, L + 1, size=shape).astype(np.int32)
        curve = oracle.ec6_3d(bins, L)
        for k in range(L):
            assert curve[k] == chi6_binary(bins <= k), (trial, k)


def test_the_same_reading_in_2d_is_table_1_four_connectivity():
    rng = np.random.default_rng(63)
    for trial in range(200):
        h, w = (int(v) for v in rng.integers(1, 12, size=2))
        L = int(rng.integers(1, 12))
        bins = rng.integers(0, L + 1, size=(h, w)).astype(np.int32)
        np.testing.assert_array_equal(oracle.ec_dual_2d(bins, L), oracle.curves_2d(bins, L)["ec4"])


def test_closed_forms():
    def box(shape, cells):
        a = np.zeros(shape, np.uint8)
        for c in cells:
            a[c] = 1
        return a
    assert chi6_binary(box((2, 2, 2), [(0, 0, 0)])) == 1
    assert chi6_binary(box((2, 2, 2), [(0, 0, 0), (0, 1, 1)])) == 2      # edge contact
    assert chi6_binary(box((2, 2, 2), [(0, 0, 0), (1, 1, 1)])) == 2      # vertex contact
    assert chi6_binary(box((2, 2, 2), [(0, 0, 0), (0, 0, 1)])) == 1      # face contact
    shell = np.ones((3, 3, 3), np.uint8)
    shell[1, 1, 1] = 0
    assert chi6_binary(shell) == 2
    ring = np.ones((1, 3, 3), np.uint8)
    ring[0, 1, 1] = 0
    assert chi6_binary(ring) == 0
    diag_ring = box((1, 3, 3), [(0, 0, 1), (0, 1, 0), (0, 1, 2), (0, 2, 1)])   # 4 voxels touching by edges
    assert chi6_binary(diag_ring) == 4
    assert chi6_binary(np.ones((3, 4, 5), np.uint8)) == 1
    assert chi6_binary(np.zeros((3, 4, 5), np.uint8)) == 0
    # under 26-connectivity the edge- and vertex-contact pairs are one component
    assert chi26_binary(box((2, 2, 2), [(0, 0, 0), (1, 1, 1)])) == 1


def test_public_layout_uses_the_6_connected_row():
    rng = np.random.default_rng(64)
    f = rng.integers(0, 6, size=(5, 6, 7)).astype(np.uint8)
    c26 = oracle.ec_curves(f, None, 5, 26, 15)
    c6 = oracle.ec_curves(f, None, 5, 6, 15)
    np.testing.assert_array_equal(c6[1:], c26[1:])   # perimeter, area, volume do not depend on it
    np.testing.assert_array_equal(c6[0], oracle.ec6_3d(oracle.bin_field(f, None, 5), 5))
