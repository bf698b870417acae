"""Vertex-contribution type map: the count of every vertex type at every level.

TEST INFRASTRUCTURE ONLY: the product path never imports this module.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it.
It shares no code with the CUDA path.

Definitions followed (Laky & Zavala, arXiv 2311.11740):

* Vertices (Sec. 2, Algorithm 1; Sec. 2.2, Algorithm 3 with Algorithm 4's
  neighbourhood fill): the grid vertices of an h x w image are the
  (h+1)(w+1) corners of its pixels, those of a d x h x w field the
  (d+1)(h+1)(w+1) corners of its voxels.  A vertex's neighbourhood is the
  2 x 2 (2 x 2 x 2) block of top cells that share it; cells outside the field
  are never active (the paper fills them with the sentinel M+1).
* Level k (k = 0 .. L-1): a top cell is active iff its bin is <= k, its bin
  being min{j : value <= t_j} (L when none, NaN included).
* Types (Table 1 in 2D, Table 2 in 3D): a neighbourhood's type is its class of
  active-cell patterns.  Sec. 2.2 tells the classes apart by the number of
  active cells and by f_adj, the sum of the Euclidean distances between all
  pairs of active cells (cell centres at the corners of a unit square/cube);
  for 5 or more active cells of a 3D neighbourhood the table uses f_adj of
  the empty cells instead (the dagger note of Table 2; the text names 5, 6
  and 7, the table's daggers also mark the full neighbourhood, f_adj 0).  In 2D the only pair of
  classes with the same count is told apart by the distance of the two
  active pixels (Algorithm 1's adjacency test).  The paper's rows run by
  number of active cells, then by increasing f_adj; type t here is row t of
  the table counted from 0 (type 0 = the empty neighbourhood).
* Type map: counts[t][k] = the number of vertices whose neighbourhood is of
  type t at level k.  The paper accumulates born/dies arrays per type and
  back-calculates the empty type (Sec. 2.1 "Parallel Implementation"); their
  running sums are these counts.  Here the counts are taken straight from
  the definition, level by level.
* Weighted curves (Sec. 4 "Discussion": any descriptor that is a weighted sum
  of vertex contributions follows from the same map by changing the weights):
  curve_d[k] = sum_t W[d][t] counts[t][k] / scale[d].

Neighbourhood mask convention: the cell at offset (dx, dy[, dz]) in {0,1}^n
from the vertex's lower corner has bit dx + 2 dy (+ 4 dz), x the fastest axis
of the field.
"""
from __future__ import annotations

import functools
import itertools
import math

import numpy as np

NTYPES = {2: 6, 3: 22}


def corners(ndim: int):
    """Corner coordinates of the 2^ndim cells of a neighbourhood, indexed by bit."""
    return [tuple((b >> a) & 1 for a in range(ndim)) for b in range(1 << ndim)]


def f_adj(points) -> float:
    """Sum of Euclidean distances over all pairs of points (the f_adj equation of Sec. 2.2)."""
    s = 0.0
    for p, q in itertools.combinations(points, 2):
        s += math.sqrt(sum((a - b) ** 2 for a, b in zip(p, q)))
    return s


def type_key(mask: int, ndim: int):
    """(number of active cells, adjacency measure) that tells the types apart.

    3D: f_adj of the active cells, or of the empty cells for 5-8 active cells
    (Table 2, dagger).  2D: the distance between the two active pixels when
    exactly two are active (Algorithm 1), else 0.
    """
    cs = corners(ndim)
    act = [cs[b] for b in range(1 << ndim) if mask >> b & 1]
    n = len(act)
    if ndim == 2:
        adj = f_adj(act) if n == 2 else 0.0
    else:
        emp = [cs[b] for b in range(8) if not mask >> b & 1]
        adj = f_adj(emp) if n >= 5 else f_adj(act)
    return (n, round(adj, 9))


@functools.lru_cache(maxsize=None)
def type_table(ndim: int) -> np.ndarray:
    """Type of every neighbourhood mask: the rank of its key among the distinct keys (read-only)."""
    keys = [type_key(m, ndim) for m in range(1 << (1 << ndim))]
    order = sorted(set(keys))
    assert len(order) == NTYPES[ndim]
    rank = {k: i for i, k in enumerate(order)}
    tab = np.array([rank[k] for k in keys], dtype=np.int64)
    tab.setflags(write=False)
    return tab


def _active_padded(bins: np.ndarray, k: int) -> np.ndarray:
    """Active cells at level k with one never-active cell of collar on every side."""
    act = np.zeros(tuple(s + 2 for s in bins.shape), dtype=bool)
    act[tuple(slice(1, -1) for _ in bins.shape)] = bins <= k
    return act


def _vertex_masks(act: np.ndarray) -> np.ndarray:
    """Neighbourhood mask of every vertex from the padded activity array."""
    ndim = act.ndim
    nv = tuple(s - 1 for s in act.shape)                  # vertices per axis: n + 1
    m = np.zeros(nv, dtype=np.uint8)             # at most 8 bits
    for b, off in enumerate(corners(ndim)):
        # off = (dx, dy[, dz]); numpy axes run (z,) y, x
        sl = tuple(slice(o, o + n) for o, n in zip(reversed(off), nv))
        m |= act[sl].astype(np.uint8) << np.uint8(b)
    return m


def type_counts_at(bins: np.ndarray, L: int, k: int) -> np.ndarray:
    """counts[t] at one level k (0 <= k < L): classify every vertex, then count."""
    assert 0 <= k < L
    tab = type_table(bins.ndim)
    m = _vertex_masks(_active_padded(bins, k))
    return np.bincount(tab[m].ravel(), minlength=NTYPES[bins.ndim]).astype(np.int64)


def type_map(bins: np.ndarray, L: int) -> np.ndarray:
    """counts[t][k] for every type and level, int64 [T][L] (the definition, level by level)."""
    out = np.zeros((NTYPES[bins.ndim], L), dtype=np.int64)
    for k in range(L):
        out[:, k] = type_counts_at(bins, L, k)
    return out


def apply_weights(counts: np.ndarray, weights, scales) -> np.ndarray:
    """curve_d[k] = sum_t W[d][t] counts[t][k] / scale[d], exact (Python integers).

    Raises ValueError when a sum is not a multiple of its scale.
    """
    W = [[int(v) for v in row] for row in weights]
    T, L = counts.shape
    out = np.zeros((len(W), L), dtype=np.int64)
    for d, row in enumerate(W):
        assert len(row) == T
        s = int(scales[d])
        for k in range(L):
            tot = sum(row[t] * int(counts[t, k]) for t in range(T))
            if tot % s:
                raise ValueError(f"row {d} level {k}: {tot} is not a multiple of {s}")
            out[d, k] = tot // s
    return out
