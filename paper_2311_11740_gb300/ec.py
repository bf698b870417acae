"""Python binding of libec (ctypes).  Argument marshalling only: every step of
the computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  If the library is not built, every call raises.

Names follow the C ABI in include/ec.h.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libec.so")

EC_U8, EC_U16, EC_F32 = 0, 1, 2
EC_DESC_EC, EC_DESC_PERIMETER, EC_DESC_AREA, EC_DESC_VOLUME = 1, 2, 4, 8
EC_OPT_ALGO, EC_OPT_VALIDATE, EC_OPT_TILE_Z, EC_OPT_GRID, EC_OPT_PROFILE, EC_OPT_HIST_SCHEDULE = 1, 2, 3, 4, 5, 6
EC_OPT_AUTOTUNE = 7
EC_OPT_TEST_GIVE_UP = 8
ALGO_AUTO, ALGO_VOXEL, ALGO_VERTEX, ALGO_PLANAR = 0, 1, 2, 3
STATUS = {0: "EC_OK", 1: "EC_ERR_ARG", 2: "EC_ERR_DTYPE", 3: "EC_ERR_UNSUPPORTED", 4: "EC_ERR_OOM",
          5: "EC_ERR_CUDA", 6: "EC_ERR_TIMEOUT", 7: "EC_ERR_OVERFLOW", 8: "EC_ERR_BUSY"}


class ECError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class FieldDesc(ctypes.Structure):
    _fields_ = [("field", ctypes.c_void_p), ("ndim", ctypes.c_int32), ("dims", ctypes.c_int64 * 3),
                ("dtype", ctypes.c_int32), ("thresholds", ctypes.c_void_p), ("L", ctypes.c_int32),
                ("connectivity", ctypes.c_int32), ("descriptors", ctypes.c_uint32),
                ("out", ctypes.c_void_p)]


SLAB_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                           ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libec.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libec.so is missing ({LIB_PATH}); build it with "
                                   "paper_2311_11740_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
            L.ec_last_error.restype = ctypes.c_char_p
            L.ec_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.c_int]
            L.ec_ctx_destroy.argtypes = [P]
            L.ec_ctx_set_option.argtypes = [P, ctypes.c_int, I64]
            L.ec_ctx_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)]
            for fn in (L.ec_curve_2d, L.ec_curve_3d):
                fn.argtypes = [P, P, ctypes.POINTER(I64), ctypes.c_int, P, I32, ctypes.c_int, U32, P, P]
            L.ec_curve_3d_stream.argtypes = [P, P, SLAB_FN, P, ctypes.POINTER(I64), ctypes.c_int, P, I32,
                                             ctypes.c_int, U32, I64, ctypes.c_size_t, P]
            L.ec_batch.argtypes = [P, ctypes.POINTER(FieldDesc), I32, P]
            L.ec_batch_tuned_plan.argtypes = [P, ctypes.POINTER(FieldDesc), I32, ctypes.POINTER(I32)]
            L.ec_workspace_bytes.argtypes = [ctypes.c_int, I32, ctypes.POINTER(I64), I32, U32]
            L.ec_workspace_bytes.restype = ctypes.c_size_t
            L.ec_vertex_table_2d.argtypes = [P]
            L.ec_vertex_table_3d.argtypes = [P]
            L.ec_vertex_table_3d_ec6.argtypes = [P]
            L.ec_bmp_read.argtypes = [ctypes.c_char_p, P, P]
            L.ec_curve_2d_bmp.argtypes = [P, ctypes.c_char_p, P, I32, ctypes.c_int, ctypes.c_uint32, P]
            L.ec_curve_3d_bmp.argtypes = [P, P, I64, P, I32, ctypes.c_int, ctypes.c_uint32, I64, ctypes.c_size_t, P]
            L.ec_selfcheck_rules.restype = I64
            L.ec_server_create.argtypes = [P, ctypes.c_size_t, I32, ctypes.POINTER(P)]
            L.ec_server_submit.argtypes = [P, ctypes.POINTER(FieldDesc), ctypes.POINTER(ctypes.c_uint64)]
            L.ec_server_submit_many.argtypes = [P, ctypes.POINTER(FieldDesc), I32, ctypes.POINTER(ctypes.c_uint64)]
            L.ec_server_reset_stats.argtypes = [P]
            L.ec_server_wait_all.argtypes = [P, I64]
            L.ec_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int32)]
            L.ec_server_wait.argtypes = [P, ctypes.c_uint64, I64, ctypes.POINTER(ctypes.c_int32)]
            L.ec_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
            L.ec_server_destroy.argtypes = [P]
            L.ec_tuned_plan.argtypes = [P, I32, ctypes.c_int, I32, U32, ctypes.POINTER(I64), ctypes.POINTER(I32)]
            L.ec_gen_hashbox_u16.argtypes = [ctypes.c_uint64, I64, I64, I64, I64, I64, I64, P, P]
            L.ec_type_map.argtypes = [P, I32, P, ctypes.POINTER(I64), ctypes.c_int, P, I32, P, P]
            L.ec_apply_weights.argtypes = [P, I32, P, I32, I32, ctypes.POINTER(I32), ctypes.POINTER(I32), P, P]
            L.ec_type_table.argtypes = [I32, P]
            L.ec_curve_3d_file.argtypes = [P, ctypes.c_char_p, I64, ctypes.POINTER(I64), ctypes.c_int, P, I32,
                                           ctypes.c_int, U32, I64, ctypes.c_size_t, P]
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise ECError(rc, lib().ec_last_error().decode(errors="replace"))


def _dims(shape):
    return (ctypes.c_int64 * len(shape))(*shape)


_TORCH_CODES = None


def dtype_code(t) -> int:
    """ec_dtype code of a torch tensor or numpy array."""
    global _TORCH_CODES
    if isinstance(t, np.ndarray):
        return {np.dtype(np.uint8): EC_U8, np.dtype(np.uint16): EC_U16, np.dtype(np.float32): EC_F32}[t.dtype]
    import torch
    if _TORCH_CODES is None:
        _TORCH_CODES = {torch.uint8: EC_U8, torch.uint16: EC_U16, torch.float32: EC_F32}
    return _TORCH_CODES[t.dtype]


_NP_DTYPES = {EC_U8: np.uint8, EC_U16: np.uint16, EC_F32: np.float32}


def n_rows(descriptors: int) -> int:
    return bin(descriptors & 0xF).count("1")


class Context:
    """An ec_ctx on one CUDA device (tables, plan cache, scratch)."""

    def __init__(self, device: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().ec_ctx_create(ctypes.byref(h), device))
        self.handle = h

    def set_option(self, option: int, value: int):
        _check(lib().ec_ctx_set_option(self.handle, option, int(value)))

    def tuned_plan(self, ndim, dtype, L, descriptors, dims):
        """(tile_z, grid, schedule) the autotuner chose for a shape class, or None."""
        out = (ctypes.c_int32 * 3)()
        rc = lib().ec_tuned_plan(self.handle, ndim, dtype, L, descriptors, _dims(dims), out)
        return None if rc else tuple(out)

    def profile_read(self):
        """(summed kernel ms, launches) since the last read (EC_OPT_PROFILE)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().ec_ctx_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        if getattr(self, "handle", None):
            lib().ec_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = {}


def default_context(device: int = 0) -> Context:
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


_RAW_STREAM = None


def _stream_ptr(stream, device):
    """The CUDA stream handle to launch on: `stream`'s, else the device's
    current stream (read without building a Stream object when torch offers
    that)."""
    global _RAW_STREAM
    import torch
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream)
    if _RAW_STREAM is None:
        _RAW_STREAM = getattr(torch._C, "_cuda_getCurrentRawStream", False)
    if _RAW_STREAM:
        return ctypes.c_void_p(_RAW_STREAM(device))
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def curve(field, thresholds=None, L=None, connectivity=None, descriptors=EC_DESC_EC, out=None,
          ctx: Context | None = None, stream=None):
    """EC (and other descriptor) curves of a CUDA tensor field (2D or 3D).

    Returns an int64 CUDA tensor [popcount(descriptors), L] (rows EC,
    perimeter, area, volume).  Calls ec_curve_2d / ec_curve_3d."""
    import torch
    assert field.is_cuda and field.is_contiguous(), "field must be a contiguous CUDA tensor"
    dev = field.device.index if field.device.index is not None else torch.cuda.current_device()
    ctx = ctx or default_context(dev)
    if thresholds is not None:
        assert thresholds.is_cuda and thresholds.dtype == field.dtype and thresholds.is_contiguous()
        L = thresholds.numel() if L is None else L
    if L is None:
        raise ValueError("L is required with identity levels")
    ndim = field.dim()
    if connectivity is None:
        connectivity = 8 if ndim == 2 else 26
    if out is None:
        out = torch.empty((n_rows(descriptors), L), dtype=torch.int64, device=field.device)
    fn = lib().ec_curve_2d if ndim == 2 else lib().ec_curve_3d
    _check(fn(ctx.handle, ctypes.c_void_p(field.data_ptr()), _dims(field.shape), dtype_code(field),
              ctypes.c_void_p(thresholds.data_ptr() if thresholds is not None else 0), int(L),
              int(connectivity), int(descriptors), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, dev)))
    return out


def curve_3d_stream(field_host=None, producer=None, dims=None, dtype=None, thresholds=None, L=None,
                    connectivity=26, descriptors=EC_DESC_EC, slab_planes=64, device_mem_cap=0,
                    ctx: Context | None = None, device: int = 0, user=None):
    """Low-memory z-slab streaming (ec_curve_3d_stream).  field_host: a host
    numpy array / CPU tensor (pinned for overlapped copies) or None with a
    producer callback producer(z0, z1, dst_ptr, stream_ptr) -> int.  Returns a
    numpy int64 array [rows, L]."""
    ctx = ctx or default_context(device)
    if field_host is not None:
        arr = field_host
        ptr = arr.data_ptr() if hasattr(arr, "data_ptr") else arr.ctypes.data
        dims = tuple(arr.shape)
        dtype = dtype_code(arr)
    else:
        ptr = 0
    thr_ptr = 0
    thr_keep = None
    if thresholds is not None:
        thr_keep = np.ascontiguousarray(thresholds)
        thr_ptr = thr_keep.ctypes.data
        L = thr_keep.size if L is None else L
    out = np.zeros((n_rows(descriptors), L), dtype=np.int64)
    if producer is not None:
        cb = SLAB_FN(lambda _u, z0, z1, dst, st: int(producer(z0, z1, dst, st)))
    else:
        cb = SLAB_FN()
    _check(lib().ec_curve_3d_stream(ctx.handle, ctypes.c_void_p(ptr), cb, ctypes.c_void_p(user or 0),
                                    _dims(dims), int(dtype), ctypes.c_void_p(thr_ptr), int(L),
                                    int(connectivity), int(descriptors), int(slab_planes),
                                    ctypes.c_size_t(int(device_mem_cap)), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def _desc(field, thresholds, L, connectivity, descriptors, out) -> FieldDesc:
    d = FieldDesc()
    d.field = field.data_ptr() if hasattr(field, "data_ptr") else field.ctypes.data
    d.ndim = len(field.shape)
    dims = list(field.shape) + [0] * (3 - len(field.shape))
    d.dims[:] = dims
    d.dtype = dtype_code(field)
    if thresholds is not None:
        d.thresholds = thresholds.data_ptr() if hasattr(thresholds, "data_ptr") else thresholds.ctypes.data
    else:
        d.thresholds = None
    d.L = int(L)
    d.connectivity = int(connectivity or (8 if d.ndim == 2 else 26))
    d.descriptors = int(descriptors)
    d.out = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    return d


class Batch:
    """A batch of fields (dicts {field, thresholds, L, connectivity,
    descriptors} with CUDA tensors) with its int64 CUDA outputs allocated
    once; run() calls ec_batch on it and may be repeated."""

    def __init__(self, fields, ctx: Context | None = None):
        import torch
        self.dev = fields[0]["field"].device.index or 0
        self.ctx = ctx or default_context(self.dev)
        self.fields = fields
        self.outs, descs = [], []
        for f in fields:
            L = f.get("L") or f["thresholds"].numel()
            o = torch.empty((n_rows(f.get("descriptors", 1)), L), dtype=torch.int64, device=f["field"].device)
            self.outs.append(o)
            descs.append(_desc(f["field"], f.get("thresholds"), L, f.get("connectivity"), f.get("descriptors", 1),
                               o))
        self.arr = (FieldDesc * len(descs))(*descs)

    def run(self, stream=None):
        _check(lib().ec_batch(self.ctx.handle, self.arr, len(self.arr), _stream_ptr(stream, self.dev)))
        return self.outs

    def tuned_plan(self):
        """(3D item depth, grid, 2D item rows) the autotuner keeps for this
        batch's mix class, or None if it has none."""
        out = (ctypes.c_int32 * 3)()
        rc = lib().ec_batch_tuned_plan(self.ctx.handle, self.arr, len(self.arr), out)
        return None if rc != 0 else tuple(out)


def batch(fields, ctx: Context | None = None, stream=None):
    """ec_batch over a list of dicts {field, thresholds, L, connectivity,
    descriptors} with CUDA tensors; returns the list of int64 CUDA outputs."""
    return Batch(fields, ctx).run(stream)


class Server:
    """The continuous-batching request loop (ec_server_*).  Request fields are
    host arrays / CPU tensors (copied in) or CUDA tensors (read in place);
    outputs are host numpy arrays filled when done."""

    def __init__(self, device_mem_budget: int, max_slots: int = 8, ctx: Context | None = None, device: int = 0):
        self.ctx = ctx or default_context(device)
        h = ctypes.c_void_p()
        _check(lib().ec_server_create(self.ctx.handle, ctypes.c_size_t(int(device_mem_budget)), int(max_slots),
                                      ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def _prepare(self, field, thresholds, L, connectivity, descriptors):
        if hasattr(field, "data_ptr"):
            field = field.contiguous()
        if thresholds is not None:
            if hasattr(thresholds, "data_ptr"):
                thresholds = thresholds.detach().contiguous().cpu().numpy()
            thresholds = np.ascontiguousarray(thresholds, dtype=_NP_DTYPES[dtype_code(field)])
            L = thresholds.size if L is None else L
        out = np.zeros((n_rows(descriptors), L), dtype=np.int64)
        return _desc(field, thresholds, L, connectivity, descriptors, out), (field, thresholds, out)

    def submit(self, field, thresholds=None, L=None, connectivity=None, descriptors=EC_DESC_EC):
        """field: host numpy array or CPU torch tensor (page-locked memory
        overlaps the copies); thresholds: host array of the field's dtype."""
        d, keep = self._prepare(field, thresholds, L, connectivity, descriptors)
        t = ctypes.c_uint64()
        _check(lib().ec_server_submit(self.handle, ctypes.byref(d), ctypes.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def submit_many(self, requests):
        """Queue a burst of requests, each (field, thresholds, L, descriptors)
        or a dict of submit()'s arguments, in order under one lock; returns the
        tickets.  All or none are queued."""
        descs, keeps = [], []
        for r in requests:
            kw = r if isinstance(r, dict) else dict(zip(("field", "thresholds", "L", "descriptors"), r))
            d, keep = self._prepare(kw["field"], kw.get("thresholds"), kw.get("L"), kw.get("connectivity"),
                                    kw.get("descriptors", EC_DESC_EC))
            descs.append(d)
            keeps.append(keep)
        n = len(descs)
        arr = (FieldDesc * n)(*descs)
        tickets = (ctypes.c_uint64 * n)()
        _check(lib().ec_server_submit_many(self.handle, arr, n, tickets))
        for t, keep in zip(tickets, keeps):
            self._keep[t] = keep
        return list(tickets)

    def poll(self, ticket):
        done, st = ctypes.c_int(), ctypes.c_int32()
        _check(lib().ec_server_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(st)))
        return bool(done.value), st.value

    def wait(self, ticket, timeout_ms: int = 60000):
        st = ctypes.c_int32()
        _check(lib().ec_server_wait(self.handle, ticket, int(timeout_ms), ctypes.byref(st)))
        if st.value != 0:
            raise ECError(st.value, "request failed")
        return self._keep[ticket][2]

    def result(self, ticket):
        return self._keep[ticket][2]

    def wait_all(self, timeout_ms: int = 600000):
        """Block until every request submitted so far is done."""
        _check(lib().ec_server_wait_all(self.handle, int(timeout_ms)))

    def reset_stats(self):
        _check(lib().ec_server_reset_stats(self.handle))

    def stats(self):
        out = (ctypes.c_double * 5)()
        _check(lib().ec_server_stats(self.handle, out))
        return dict(count=out[0], p50_us=out[1], p99_us=out[2], mean_us=out[3], span_us=out[4])

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().ec_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HashboxSpec(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("x0", ctypes.c_int64), ("y0", ctypes.c_int64), ("z0", ctypes.c_int64),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64)]


def gen_hashbox_u16(seed, x0, y0, z0, nx, ny, nz, device=0, stream=None):
    """The low-memory workload's hash-box field on the device (uint16 tensor
    (nz, ny, nx)), generated by the library's kernel."""
    import torch
    out = torch.empty((nz, ny, nx), dtype=torch.uint16, device=f"cuda:{device}")
    _check(lib().ec_gen_hashbox_u16(int(seed), int(x0), int(y0), int(z0), int(nx), int(ny), int(nz),
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, device)))
    return out


def hashbox_stream(spec: HashboxSpec, nz: int, thresholds=None, L=4096, descriptors=EC_DESC_EC,
                   slab_planes=64, device_mem_cap=0, ctx: Context | None = None, device: int = 0, probe=None):
    """ec_curve_3d_stream over a device-generated hash box (the library's own
    producer).  probe(z0, z1), if given, is called before each slab."""
    ctx = ctx or default_context(device)
    raw = ctypes.cast(lib().ec_hashbox_producer, ctypes.c_void_p).value
    if probe is None:
        cb = SLAB_FN(raw)
        user = ctypes.addressof(spec)
    else:
        inner = SLAB_FN(raw)

        def _wrapped(u, z0, z1, dst, st):
            probe(z0, z1)
            return inner(u, z0, z1, dst, st)
        cb = SLAB_FN(_wrapped)
        user = ctypes.addressof(spec)
    thr_ptr, thr_keep = 0, None
    if thresholds is not None:
        thr_keep = np.ascontiguousarray(thresholds, dtype=np.uint16)
        thr_ptr = thr_keep.ctypes.data
        L = thr_keep.size
    out = np.zeros((n_rows(descriptors), L), dtype=np.int64)
    dims = (int(nz), int(spec.ny), int(spec.nx))
    _check(lib().ec_curve_3d_stream(ctx.handle, None, cb, ctypes.c_void_p(user), _dims(dims), EC_U16,
                                    ctypes.c_void_p(thr_ptr), int(L), 26, int(descriptors), int(slab_planes),
                                    ctypes.c_size_t(int(device_mem_cap)), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def curve_3d_file(path, dims, dtype, thresholds=None, L=None, offset=0, connectivity=26,
                  descriptors=EC_DESC_EC, slab_planes=64, device_mem_cap=0, ctx: Context | None = None,
                  device: int = 0):
    """Curves of a 3D field stored raw in a file (ec_curve_3d_file).  dims =
    (d, h, w); dtype an ec dtype code or numpy dtype; thresholds a host array
    (or None for identity levels with L).  Returns int64 numpy [rows, L]."""
    ctx = ctx or default_context(device)
    code = dtype if isinstance(dtype, int) else {np.dtype(np.uint8): EC_U8, np.dtype(np.uint16): EC_U16,
                                                  np.dtype(np.float32): EC_F32}[np.dtype(dtype)]
    thr = None
    if thresholds is not None:
        thr = np.ascontiguousarray(np.asarray(thresholds, dtype=_NP_DTYPES[code]))
        L = thr.size if L is None else L
    if L is None:
        raise ValueError("L is required with identity levels")
    out = np.zeros((n_rows(descriptors), L), dtype=np.int64)
    _check(lib().ec_curve_3d_file(ctx.handle, os.fsencode(path), int(offset), _dims(dims), code,
                                  None if thr is None else thr.ctypes.data_as(ctypes.c_void_p), int(L),
                                  int(connectivity), int(descriptors), int(slab_planes),
                                  ctypes.c_size_t(int(device_mem_cap)), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def bmp_read(path) -> np.ndarray:
    """The pixels of a grayscale BMP as uint8 [h, w], row 0 = the top row (ec_bmp_read)."""
    dims = (ctypes.c_int64 * 2)()
    _check(lib().ec_bmp_read(os.fsencode(path), dims, None))
    out = np.zeros((dims[0], dims[1]), dtype=np.uint8)
    _check(lib().ec_bmp_read(os.fsencode(path), dims, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def curve_2d_bmp(path, thresholds=None, L=None, connectivity=8, descriptors=EC_DESC_EC,
                 ctx: Context | None = None, device: int = 0):
    """Curves of one grayscale BMP image (ec_curve_2d_bmp): int64 numpy [rows, L]."""
    ctx = ctx or default_context(device)
    thr = None if thresholds is None else np.ascontiguousarray(np.asarray(thresholds, dtype=np.uint8))
    L = (thr.size if thr is not None else None) if L is None else L
    if L is None:
        raise ValueError("L is required with identity levels")
    out = np.zeros((n_rows(descriptors), L), dtype=np.int64)
    _check(lib().ec_curve_2d_bmp(ctx.handle, os.fsencode(path),
                                 None if thr is None else thr.ctypes.data_as(ctypes.c_void_p), int(L),
                                 int(connectivity), int(descriptors), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def curve_3d_bmp(paths, thresholds=None, L=None, connectivity=26, descriptors=EC_DESC_EC, slab_planes=64,
                 device_mem_cap=0, ctx: Context | None = None, device: int = 0):
    """Curves of a stack of BMP slices, paths[z] = plane z (ec_curve_3d_bmp): int64 numpy [rows, L]."""
    ctx = ctx or default_context(device)
    thr = None if thresholds is None else np.ascontiguousarray(np.asarray(thresholds, dtype=np.uint8))
    L = (thr.size if thr is not None else None) if L is None else L
    if L is None:
        raise ValueError("L is required with identity levels")
    enc = [os.fsencode(p) for p in paths]
    arr = (ctypes.c_char_p * len(enc))(*enc)
    out = np.zeros((n_rows(descriptors), L), dtype=np.int64)
    _check(lib().ec_curve_3d_bmp(ctx.handle, ctypes.cast(arr, ctypes.c_void_p), len(enc),
                                 None if thr is None else thr.ctypes.data_as(ctypes.c_void_p), int(L),
                                 int(connectivity), int(descriptors), int(slab_planes),
                                 ctypes.c_size_t(int(device_mem_cap)), out.ctypes.data_as(ctypes.c_void_p)))
    return out


NTYPES = {2: 6, 3: 22}


def type_map(field, thresholds=None, L=None, out=None, ctx: Context | None = None, stream=None):
    """Contribution-type map of a CUDA tensor field (ec_type_map): int64 CUDA
    tensor [T, L], counts[t][k] = vertices of type t (Table 1 / Table 2 row
    order) at level k."""
    import torch
    assert field.is_cuda and field.is_contiguous(), "field must be a contiguous CUDA tensor"
    dev = field.device.index if field.device.index is not None else torch.cuda.current_device()
    ctx = ctx or default_context(dev)
    if thresholds is not None:
        assert thresholds.is_cuda and thresholds.dtype == field.dtype and thresholds.is_contiguous()
        L = thresholds.numel() if L is None else L
    if L is None:
        raise ValueError("L is required with identity levels")
    ndim = field.dim()
    if ndim not in NTYPES:
        raise ValueError("field must be 2D or 3D")
    if out is None:
        out = torch.empty((NTYPES[ndim], L), dtype=torch.int64, device=field.device)
    _check(lib().ec_type_map(ctx.handle, ndim, ctypes.c_void_p(field.data_ptr()), _dims(field.shape),
                             dtype_code(field),
                             ctypes.c_void_p(thresholds.data_ptr() if thresholds is not None else 0), int(L),
                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, dev)))
    return out


def apply_weights(counts, weights, scales=None, out=None, ctx: Context | None = None, stream=None):
    """Weighted curves from a type map (ec_apply_weights): out[d][k] =
    sum_t weights[d][t] counts[t][k] / scales[d]; counts an int64 CUDA tensor
    [T, L], weights an integer array [nd, T]."""
    import torch
    assert counts.is_cuda and counts.dtype == torch.int64 and counts.is_contiguous()
    dev = counts.device.index if counts.device.index is not None else torch.cuda.current_device()
    ctx = ctx or default_context(dev)
    W = np.ascontiguousarray(np.asarray(weights, dtype=np.int32))
    if W.ndim != 2 or W.shape[1] != counts.shape[0]:
        raise ValueError("weights must be [nd, T]")
    nd, T = W.shape
    L = counts.shape[1]
    sc = None if scales is None else np.ascontiguousarray(np.asarray(scales, dtype=np.int32))
    if out is None:
        out = torch.empty((nd, L), dtype=torch.int64, device=counts.device)
    I32P = ctypes.POINTER(ctypes.c_int32)
    _check(lib().ec_apply_weights(ctx.handle, T, ctypes.c_void_p(counts.data_ptr()), L, nd,
                                  W.ctypes.data_as(I32P), None if sc is None else sc.ctypes.data_as(I32P),
                                  ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, dev)))
    return out


def type_table(ndim: int) -> np.ndarray:
    """Type of every neighbourhood mask (bit x + 2y (+ 4z)), from the library."""
    out = np.zeros(1 << (1 << ndim), np.int32)
    _check(lib().ec_type_table(ndim, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def vertex_table_2d() -> np.ndarray:
    out = np.zeros((16, 4), np.int32)
    _check(lib().ec_vertex_table_2d(out.ctypes.data_as(ctypes.c_void_p)))
    return out


def vertex_table_3d() -> np.ndarray:
    out = np.zeros((256, 4), np.int32)
    _check(lib().ec_vertex_table_3d(out.ctypes.data_as(ctypes.c_void_p)))
    return out


def vertex_table_3d_ec6() -> np.ndarray:
    """8 * EC per 8-bit vertex mask under 3D 6-connectivity (int32 [256])."""
    out = np.zeros(256, dtype=np.int32)
    _check(lib().ec_vertex_table_3d_ec6(out.ctypes.data_as(ctypes.c_void_p)))
    return out


def selfcheck_rules() -> int:
    return int(lib().ec_selfcheck_rules())
