"""CPU oracle for EC / perimeter / area / volume curves (test infrastructure).

TEST INFRASTRUCTURE ONLY: the product path never imports this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may use it.  It shares no code with the CUDA path.

The arithmetic lives in ``ec_oracle.c`` (plain cell counting of the closed
cubical complex; see that file's header for the definitions it follows and the
paper passages they come from).  This module compiles it with gcc/OpenMP and
wraps it with ctypes and numpy.  ``brute.py`` holds the literal per-level
enumeration used to pin the oracle on tiny grids; ``typemap.py`` counts the
vertex types of Tables 1 and 2 at every level (the contribution-type map).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ec_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DTYPE_CODES = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2}


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.oracle_bin.argtypes = [P, I64, ctypes.c_int, P, I32, P]
            lib.oracle_curves_2d.argtypes = [P, I64, I64, I32, P, P, P, P]
            lib.oracle_curves_3d.argtypes = [P, I64, I64, I64, I32, P, P, P, P]
            lib.oracle_curves_3d_zrange.argtypes = [P, I64, I64, I64, I32, I64, I64, P, P, P, P]
            lib.oracle_hashbox_u16.argtypes = [ctypes.c_uint64, I64, I64, I64, I64, I64, I64, P]
            lib.oracle_ec6_3d.argtypes = [P, I64, I64, I64, I32, P]
            lib.oracle_ec_dual_2d.argtypes = [P, I64, I64, I32, P]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    """Threads the oracle uses from now on (n < 1: the OpenMP default).  For
    timing only: results do not depend on it."""
    _load().oracle_set_threads(int(n))


def bin_field(field: np.ndarray, thresholds, L: int) -> np.ndarray:
    """bin(x) = min{k : x <= t_k}, L if none (Eq. sublevel_set), int32."""
    field = np.ascontiguousarray(field)
    code = DTYPE_CODES[field.dtype]
    if thresholds is not None:
        thresholds = np.ascontiguousarray(thresholds, dtype=field.dtype)
        assert thresholds.size == L
    out = np.empty(field.shape, dtype=np.int32)
    rc = _load().oracle_bin(_ptr(field), field.size, code, _ptr(thresholds), L, _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_bin failed ({rc})")
    return out


def curves_2d(bins: np.ndarray, L: int) -> dict:
    """EC (8- and 4-connected), perimeter and area curves of a binned 2D field."""
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    h, w = bins.shape
    out = {k: np.zeros(L, dtype=np.int64) for k in ("ec8", "ec4", "perimeter", "area")}
    rc = _load().oracle_curves_2d(_ptr(bins), h, w, L, _ptr(out["ec8"]), _ptr(out["ec4"]),
                                  _ptr(out["perimeter"]), _ptr(out["area"]))
    if rc != 0:
        raise ValueError(f"oracle_curves_2d failed ({rc})")
    return out


def curves_3d(bins: np.ndarray, L: int) -> dict:
    """EC (26-connected), crease perimeter, surface area and volume curves of a
    binned 3D field."""
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    d, h, w = bins.shape
    out = {k: np.zeros(L, dtype=np.int64) for k in ("ec", "perimeter", "area", "volume")}
    rc = _load().oracle_curves_3d(_ptr(bins), d, h, w, L, _ptr(out["ec"]), _ptr(out["perimeter"]),
                                  _ptr(out["area"]), _ptr(out["volume"]))
    if rc != 0:
        raise ValueError(f"oracle_curves_3d failed ({rc})")
    return out


def curves_3d_zrange(bins: np.ndarray, L: int, zlo: int, zhi: int) -> dict:
    """Curves of only the cells whose doubled z coordinate is in [zlo, zhi]
    (the whole field is [0, 2d]); disjoint ranges add up."""
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    d, h, w = bins.shape
    out = {k: np.zeros(L, dtype=np.int64) for k in ("ec", "perimeter", "area", "volume")}
    rc = _load().oracle_curves_3d_zrange(_ptr(bins), d, h, w, L, zlo, zhi, _ptr(out["ec"]), _ptr(out["perimeter"]),
                                         _ptr(out["area"]), _ptr(out["volume"]))
    if rc != 0:
        raise ValueError(f"oracle_curves_3d_zrange failed ({rc})")
    return out


def ec6_3d(bins: np.ndarray, L: int) -> np.ndarray:
    """EC curve of a binned 3D field under 6-connectivity: cells whose incident
    voxels are all active, #voxels - #face pairs + #squares - #cubes."""
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    d, h, w = bins.shape
    out = np.zeros(L, dtype=np.int64)
    rc = _load().oracle_ec6_3d(_ptr(bins), d, h, w, L, _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_ec6_3d failed ({rc})")
    return out


def ec_dual_2d(bins: np.ndarray, L: int) -> np.ndarray:
    """The same reading in 2D (cells whose incident pixels are all active):
    #pixels - #edge pairs + #2x2 squares, the 4-connected EC."""
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    h, w = bins.shape
    out = np.zeros(L, dtype=np.int64)
    rc = _load().oracle_ec_dual_2d(_ptr(bins), h, w, L, _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_ec_dual_2d failed ({rc})")
    return out


EC, PERIMETER, AREA, VOLUME = 1, 2, 4, 8


def ec_curves(field: np.ndarray, thresholds, L: int, connectivity: int, descriptors: int) -> np.ndarray:
    """Curves in the public API's output layout: int64 [popcount(descriptors)][L],
    rows ordered EC, perimeter, area, volume."""
    bins = bin_field(field, thresholds, L)
    rows = []
    if field.ndim == 2:
        c = curves_2d(bins, L)
        if descriptors & EC:
            rows.append(c["ec8"] if connectivity == 8 else c["ec4"])
        if descriptors & PERIMETER:
            rows.append(c["perimeter"])
        if descriptors & AREA:
            rows.append(c["area"])
    else:
        c = curves_3d(bins, L)
        if connectivity == 6:
            c["ec"] = ec6_3d(bins, L)
        for bit, key in ((EC, "ec"), (PERIMETER, "perimeter"), (AREA, "area"), (VOLUME, "volume")):
            if descriptors & bit:
                rows.append(c[key])
    if not rows:
        return np.zeros((0, L), dtype=np.int64)
    return np.stack(rows)


def hashbox_u16(seed: int, x0: int, y0: int, z0: int, nx: int, ny: int, nz: int) -> np.ndarray:
    """The hash-box field of the low-memory workload, regenerated on the CPU
    (MurmurHash3-finaliser counter hash smoothed by a 5^3 box), shape (nz, ny, nx)."""
    out = np.empty((nz, ny, nx), dtype=np.uint16)
    rc = _load().oracle_hashbox_u16(seed, x0, y0, z0, nx, ny, nz, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_hashbox_u16 failed")
    return out
