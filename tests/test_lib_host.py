"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every function its header declares, and its per-vertex tables reproduce the
paper's Tables 1 and 2."""
import os
import re
from fractions import Fraction

import numpy as np

from tests import _tables

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ec_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(libec):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(libec, n), n


def test_vertex_table_3d_matches_table2(libec):
    from paper_2311_11740_gb300 import ec
    t = ec.vertex_table_3d()
    full, _ = _tables.table2()
    for m in range(256):
        row = full[m]
        assert Fraction(int(t[m, 0]), 8) == row["EC"], (m, row["row"])
        assert Fraction(int(t[m, 1]), 2) == row["Perim"], (m, row["row"])
        assert Fraction(int(t[m, 2]), 4) == row["AreaUsed"], (m, row["row"])
        assert Fraction(int(t[m, 3]), 8) == row["Volume"], (m, row["row"])


def test_vertex_table_2d_matches_table1(libec):
    from paper_2311_11740_gb300 import ec
    t = ec.vertex_table_2d()
    t1 = _tables.table1()
    for m in range(16):
        row = t1[m]
        assert Fraction(int(t[m, 0]), 4) == row["EC8"], m
        assert Fraction(int(t[m, 1]), 4) == row["EC4"], m
        assert Fraction(int(t[m, 2]), 2) == row["Perim"], m
        assert Fraction(int(t[m, 3]), 4) == row["Area"], m


def test_regrouped_closed_forms_equal_tables(libec):
    from paper_2311_11740_gb300 import ec
    assert ec.selfcheck_rules() == 0


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2311_11740_gb300 import ec
    monkeypatch.setattr(ec, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ec, "_lib", None)
    try:
        ec.lib()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("expected a failure")


def test_type_tables_match_the_oracle_classifier(libec):
    """The library's mask -> type tables (Table 1/2 pictures closed under the
    square/cube symmetries) equal the oracle's count-and-f_adj classifier."""
    from oracle import typemap as tm
    from paper_2311_11740_gb300 import ec
    for ndim in (2, 3):
        np.testing.assert_array_equal(ec.type_table(ndim), tm.type_table(ndim))


def test_type_table_rows_carry_the_paper_weights(libec):
    """Every mask of a type has the type's Table 2 weights (the table the
    kernels use agrees with the printed row of the mask's type)."""
    from paper_2311_11740_gb300 import ec
    tt = ec.type_table(3)
    _, by_class = _tables.table2()
    rows = {r["row"] - 1: r for r in by_class.values()}
    vt = ec.vertex_table_3d()
    for m in range(256):
        r = rows[int(tt[m])]
        assert Fraction(int(vt[m, 0]), 8) == r["EC"] and Fraction(int(vt[m, 3]), 8) == r["Volume"], m


def test_bench_type_weights_are_table2_columns(libec):
    """bench.py weights the type map with the library's per-mask table taken
    at one mask of each type; those weights are Table 2's columns (8 EC, 2
    perimeter, 4 area with the row-10 erratum, 8 volume) in row order."""
    from paper_2311_11740_gb300 import ec
    tt, vt = ec.type_table(3), ec.vertex_table_3d()
    W = np.stack([vt[int(np.flatnonzero(tt == t)[0])] for t in range(22)], axis=1)
    _, by_class = _tables.table2()
    rows = sorted(by_class.values(), key=lambda r: r["row"])
    want = np.array([[int(8 * r["EC"]) for r in rows], [int(2 * r["Perim"]) for r in rows],
                     [int(4 * r["AreaUsed"]) for r in rows], [int(8 * r["Volume"]) for r in rows]])
    np.testing.assert_array_equal(W, want)


def test_vertex_table_3d_ec6_sums_to_the_oracle_and_is_constant_per_type(libec):
    """The 6-connected per-vertex EC table: summed over every vertex of random
    binary fields it gives 8 x the oracle's 6-connected EC, and it is constant
    on each vertex type (so it serves as an ec_apply_weights row)."""
    import oracle
    from paper_2311_11740_gb300 import ec
    t6 = ec.vertex_table_3d_ec6()
    types = ec.type_table(3)
    for ty in range(int(types.max()) + 1):
        assert len(set(t6[types == ty].tolist())) == 1, ty
    rng = np.random.default_rng(66)
    for trial in range(60):
        shape = tuple(int(v) for v in rng.integers(1, 7, size=3))
        a = (rng.random(shape) < rng.uniform(0.2, 0.9)).astype(np.int64)
        p = np.zeros(tuple(s + 2 for s in shape), np.int64)
        p[1:-1, 1:-1, 1:-1] = a
        d, h, w = p.shape
        masks = np.zeros((d - 1, h - 1, w - 1), np.int64)
        for b in range(8):
            dx, dy, dz = b & 1, (b >> 1) & 1, b >> 2
            masks |= p[dz:dz + d - 1, dy:dy + h - 1, dx:dx + w - 1] << b
        want = int(oracle.ec6_3d(np.where(a.astype(bool), 0, 1).astype(np.int32), 1)[0])
        assert int(t6[masks].sum()) == 8 * want, trial
