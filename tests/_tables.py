"""Load the transcribed Tables 1 and 2 (tests/golden) and expand them to all
16 / 256 neighbourhood configurations through the square / cube symmetry
groups.  Test helper only; it shares nothing with the oracle or the CUDA path.

Bit convention for a neighbourhood mask: corner (x, y[, z]) in {0,1}^n has bit
x + 2y (+ 4z).  The contribution values are geometric, so they do not depend on
which picture axis is called x, y or z.
"""
from __future__ import annotations

import itertools
import os
from fractions import Fraction

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            yield line.split()


def _orbit_min(mask, n):
    corners = list(itertools.product((0, 1), repeat=n))
    best = None
    for perm in itertools.permutations(range(n)):
        for flips in itertools.product((0, 1), repeat=n):
            m = 0
            for c in corners:
                bit = sum(c[a] << a for a in range(n))
                if mask >> bit & 1:
                    img = [c[perm[a]] ^ flips[a] for a in range(n)]
                    m |= 1 << sum(img[a] << a for a in range(n))
            best = m if best is None else min(best, m)
    return best


def table1():
    """dict mask(0..15) -> {type, V8, E8, F8, EC8, V4, E4, F4, EC4, Perim, Area} as Fractions."""
    by_class = {}
    for r in _rows("table1_2d_vertex_contributions.txt"):
        typ, cells = r[0], r[1]
        vals = [Fraction(v) for v in r[2:]]
        mask = 0
        if cells != "-":
            for c in cells.split(";"):
                x, y = (int(t) for t in c.strip("()").split(","))
                mask |= 1 << (x + 2 * y)
        keys = ("V8", "E8", "F8", "EC8", "V4", "E4", "F4", "EC4", "Perim", "Area")
        by_class[_orbit_min(mask, 2)] = dict(type=typ, **dict(zip(keys, vals)))
    return {m: by_class[_orbit_min(m, 2)] for m in range(16)}


def table2():
    """dict mask(0..255) -> row dict with Fractions (Area = printed, AreaUsed = erratum-corrected)."""
    by_class = {}
    for r in _rows("table2_3d_vertex_contributions.txt"):
        row, fadj, corners = int(r[0]), r[1], r[2]
        vals = [Fraction(v) for v in r[3:]]
        mask = 0
        if corners != "-":
            for c in corners.split(";"):
                x, y, z = (int(ch) for ch in c)
                mask |= 1 << (x + 2 * y + 4 * z)
        keys = ("V", "E", "F", "Vox", "EC", "Perim", "Area", "Volume", "AreaUsed")
        cls = _orbit_min(mask, 3)
        assert cls not in by_class, f"row {row} duplicates a class"
        by_class[cls] = dict(row=row, fadj=fadj, rep=mask, **dict(zip(keys, vals)))
    return {m: by_class[_orbit_min(m, 3)] for m in range(256)}, by_class
