"""The allocation-free 3D entry point (ec_curve_3d_noalloc), called through
the C ABI, gives the same curves as ec_curve_3d.  Curves are integers, so the
tolerance is zero.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2311_11740_gb300 import ec, workloads

pytestmark = pytest.mark.gpu


def _noalloc(field, thr, L, desc, out):
    fn = ec.lib().ec_curve_3d_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_void_p, ctypes.c_int32,
                   ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    rc = fn(ctypes.c_void_p(field.data_ptr()), ec._dims(field.shape), ec.dtype_code(field),
            ctypes.c_void_p(thr.data_ptr() if thr is not None else 0), int(L), 26, int(desc),
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_noalloc_matches_ec_curve_3d_on_two_calls(libec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f, thr = workloads.config3(n=96, nblobs=40, L=257, device="cuda")
    ctx = ec.Context(0)
    want = ec.curve(f, thr, descriptors=15, ctx=ctx).cpu().numpy()
    g = ec.gen_hashbox_u16(4, 0, 0, 0, 70, 50, 30)
    want_g = ec.curve(g, None, L=4096, descriptors=13, ctx=ctx).cpu().numpy()
    for _ in range(2):   # two calls in a row: the shared scratch must start clean each time
        out = torch.full((4, 257), -1, dtype=torch.int64, device="cuda")
        assert _noalloc(f, thr, 257, 15, out) == 0, ec.lib().ec_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        out_g = torch.full((3, 4096), -1, dtype=torch.int64, device="cuda")
        assert _noalloc(g, None, 4096, 13, out_g) == 0, ec.lib().ec_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out_g.cpu().numpy(), want_g)


def test_noalloc_equals_oracle_and_covers_every_kernel_branch(libec):
    """Against the CPU oracle directly, on the fast kernel, on the generic
    kernel the fast one hands over to (more levels than the fast kernel's
    16-bit keys hold), and at exactly the scratch's 65536 histogram entries
    (4 descriptors x 16384 levels: the global-histogram variant)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    rng = np.random.default_rng(12)
    cases = []
    f, thr = workloads.config3(n=40, nblobs=10, L=65)
    cases.append((f.numpy(), thr.numpy(), 65, 15))
    cases.append((rng.integers(0, 40000, size=(5, 9, 21)).astype(np.uint16), None, 32768, 9))
    cases.append((rng.integers(0, 17000, size=(6, 11, 19)).astype(np.uint16), None, 16384, 15))
    for fh, th, L, desc in cases:
        want = oracle.ec_curves(fh, th, L, 26, desc)
        fd = torch.from_numpy(fh.astype(np.int32)).cuda().to(torch.uint16) if fh.dtype == np.uint16 \
            else torch.from_numpy(fh).cuda()
        td = None if th is None else torch.from_numpy(th).cuda()
        for _ in range(2):
            out = torch.full(want.shape, -1, dtype=torch.int64, device="cuda")
            assert _noalloc(fd, td, L, desc, out) == 0, ec.lib().ec_last_error()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), want, err_msg=f"L={L} desc={desc}")


def test_noalloc_rejects_requests_beyond_its_scratch(libec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = torch.zeros((4, 4, 4), dtype=torch.uint16, device="cuda")
    out = torch.zeros((4, 20000), dtype=torch.int64, device="cuda")
    assert _noalloc(f, None, 20000, 15, out) == 1   # EC_ERR_ARG
    assert b"65536" in ec.lib().ec_last_error()
