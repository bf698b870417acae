"""Literal per-level enumeration of the closed cubical complex (tiny grids).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  O(cells * L) pure
Python: for every level k it lists the active top cells (value <= t_k,
Eq. sublevel_set), adds every face, edge and vertex of each of them (the
closure rule stated after Eq. sublevel_set), and counts cells by dimension for
chi = V - E + F - C (Eq. EC_formula).  Boundary measures are counted cell by
cell from the same active set.  4-connected EC is computed topologically
(components minus holes), not from the vertex table, so it is an independent
check of the oracle's Table-1 reading.

Cells use doubled integer coordinates: a coordinate is odd on the span of a top
cell and even on a grid plane; the dimension of a cell is its number of odd
coordinates.
"""
from __future__ import annotations

import itertools
from collections import deque

import numpy as np


def _closure_2d(active):
    cells = set()
    for (y, x) in active:
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                cells.add((2 * y + 1 + dy, 2 * x + 1 + dx))
    return cells


def _closure_3d(active):
    cells = set()
    for (z, y, x) in active:
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    cells.add((2 * z + 1 + dz, 2 * y + 1 + dy, 2 * x + 1 + dx))
    return cells


def _components(mask, neighbours):
    """Connected components of True cells of a 2D boolean array (BFS)."""
    h, w = mask.shape
    seen = np.zeros_like(mask, dtype=bool)
    comps = []
    for y in range(h):
        for x in range(w):
            if mask[y, x] and not seen[y, x]:
                comp = []
                q = deque([(y, x)])
                seen[y, x] = True
                while q:
                    cy, cx = q.popleft()
                    comp.append((cy, cx))
                    for dy, dx in neighbours:
                        ny, nx = cy + dy, cx + dx
                        if 0 <= ny < h and 0 <= nx < w and mask[ny, nx] and not seen[ny, nx]:
                            seen[ny, nx] = True
                            q.append((ny, nx))
                comps.append(comp)
    return comps


N4 = [(-1, 0), (1, 0), (0, -1), (0, 1)]
N8 = N4 + [(-1, -1), (-1, 1), (1, -1), (1, 1)]


def euler_2d_topological(active: np.ndarray, fg_conn: int) -> int:
    """#components of the foreground minus #bounded background components,
    with the complementary connectivity for the background (8/4 or 4/8)."""
    fg_n = N8 if fg_conn == 8 else N4
    bg_n = N4 if fg_conn == 8 else N8
    # pad with background so that every unbounded background region touches the frame
    pad = np.zeros((active.shape[0] + 2, active.shape[1] + 2), dtype=bool)
    pad[1:-1, 1:-1] = active
    n_fg = len(_components(pad, fg_n))
    bg = _components(~pad, bg_n)
    h, w = pad.shape
    holes = 0
    for comp in bg:
        if not any(y in (0, h - 1) or x in (0, w - 1) for y, x in comp):
            holes += 1
    return n_fg - holes


def curves_2d(values: np.ndarray, thresholds) -> dict:
    """values: 2D array; thresholds: iterable of levels t_k.  Active iff x <= t_k
    (numpy comparison in the array's dtype; NaN is never active)."""
    h, w = values.shape
    out = {k: [] for k in ("ec8", "ec4", "perimeter", "area")}
    for t in thresholds:
        act = values <= t
        active = [(y, x) for y in range(h) for x in range(w) if act[y, x]]
        cells = _closure_2d(active)
        counts = [0, 0, 0]
        for c in cells:
            counts[(c[0] & 1) + (c[1] & 1)] += 1
        out["ec8"].append(counts[0] - counts[1] + counts[2])
        out["ec4"].append(euler_2d_topological(act, 4))
        # perimeter: edges of the grid with exactly one active incident pixel
        per = 0
        for Y in range(2 * h + 1):
            for X in range(2 * w + 1):
                if (Y & 1) + (X & 1) != 1:
                    continue
                if Y & 1:   # vertical edge between pixels (y, x-1) and (y, x)
                    y, xs = (Y - 1) // 2, (X // 2 - 1, X // 2)
                    inc = [act[y, x] if 0 <= x < w else False for x in xs]
                else:       # horizontal edge between (y-1, x) and (y, x)
                    x, ys = (X - 1) // 2, (Y // 2 - 1, Y // 2)
                    inc = [act[y, x] if 0 <= y < h else False for y in ys]
                per += int(sum(inc) == 1)
        out["perimeter"].append(per)
        out["area"].append(len(active))
    return {k: np.array(v, dtype=np.int64) for k, v in out.items()}


def _crease(active4):
    """active4: dict slot->bool for slots (a, b) in {0,1}^2 around an edge."""
    on = [s for s, v in active4.items() if v]
    if len(on) in (1, 3):
        return 1
    if len(on) == 2:
        (a0, b0), (a1, b1) = on
        return 2 if (a0 != a1 and b0 != b1) else 0
    return 0


def curves_3d(values: np.ndarray, thresholds) -> dict:
    d, h, w = values.shape
    dims = (d, h, w)
    out = {k: [] for k in ("ec", "perimeter", "area", "volume")}
    for t in thresholds:
        act = values <= t
        active = [(z, y, x) for z in range(d) for y in range(h) for x in range(w) if act[z, y, x]]
        cells = _closure_3d(active)
        counts = [0, 0, 0, 0]
        for c in cells:
            counts[(c[0] & 1) + (c[1] & 1) + (c[2] & 1)] += 1
        out["ec"].append(counts[0] - counts[1] + counts[2] - counts[3])

        def is_act(idx):
            return all(0 <= idx[a] < dims[a] for a in range(3)) and bool(act[idx])

        area = 0
        per = 0
        for C in itertools.product(range(2 * d + 1), range(2 * h + 1), range(2 * w + 1)):
            odd = [c & 1 for c in C]
            nodd = sum(odd)
            if nodd == 2:   # face: incident voxels on both sides of its even axis
                e = odd.index(0)
                base = [(c - 1) // 2 for c in C]
                inc = []
                for side in (-1, 0):
                    idx = list(base)
                    idx[e] = C[e] // 2 + side
                    inc.append(is_act(tuple(idx)))
                area += int(sum(inc) == 1)
            elif nodd == 1:  # edge: 4 incident voxels around it
                axes = [a for a in range(3) if odd[a] == 0]
                base = [(c - 1) // 2 for c in C]
                a4 = {}
                for sa in (0, 1):
                    for sb in (0, 1):
                        idx = list(base)
                        idx[axes[0]] = C[axes[0]] // 2 - 1 + sa
                        idx[axes[1]] = C[axes[1]] // 2 - 1 + sb
                        a4[(sa, sb)] = is_act(tuple(idx))
                per += _crease(a4)
        out["area"].append(area)
        out["perimeter"].append(per)
        out["volume"].append(len(active))
    return {k: np.array(v, dtype=np.int64) for k, v in out.items()}
