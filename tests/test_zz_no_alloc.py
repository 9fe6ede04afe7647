"""The allocation-free grid sort (sph_bin_and_sort_noalloc) against the
context-based sph_bin_and_sort.

The allocation-free entry point exists for callers that cannot allocate
device memory (a framework that owns all device memory, a plugin given only
its buffers, a loop that must not call cudaMalloc); its scratch is a fixed
device array inside the library.  This file is collected last on purpose: if
it fails, a run that stops at the first failure has already run every other
test.
"""
import ctypes

import numpy as np
import pytest

from helpers import need_gpu, pos_h_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def _entry():
    from paper_1807_08116_gb300 import native as nv
    f = nv.lib().sph_bin_and_sort_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(nv.SphGrid),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return f


def _noalloc_sort(ph, log2_M, grid=None):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    n = len(ph)
    x = torch.as_tensor(ph, device="cuda")
    key = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    start = torch.full(((1 << log2_M) + 1,), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    g = None if grid is None else ctypes.byref(nv.SphGrid(
        grid["x0"], grid["y0"], grid["z0"], grid["log2_L0"], grid["n_levels"], grid["log2_M"]))
    rc = _entry()(x.data_ptr(), n, log2_M, g, key.data_ptr(), start.data_ptr(), perm.data_ptr(),
                  torch.cuda.current_stream().cuda_stream)
    assert rc == nv.SPH_OK
    torch.cuda.synchronize()
    return key.cpu().numpy(), start.cpu().numpy(), perm.cpu().numpy()


def _context_sort(ph, log2_M, grid=None):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    n = len(ph)
    ctx = nv.Ctx(n, 1024, log2_M=log2_M)
    key = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty((1 << log2_M) + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    nv.sph_bin_and_sort(ctx, torch.as_tensor(ph, device="cuda"), grid=grid, key=key,
                        cell_start=start, perm=perm)
    torch.cuda.synchronize()
    return key.cpu().numpy(), start.cpu().numpy(), perm.cpu().numpy()


def test_noalloc_sort_equals_context_sort_twice_in_a_row():
    # two different particle sets back to back: the second call must not see
    # anything the first one left in the shared scratch array
    a = ics.single_halo(8192, 0, seed=11)
    ph_a = pos_h_of(a["r"], a["h"])
    b = ics.two_halo(20000, 0, seed=12)
    ph_b = pos_h_of(b["r"], b["h"])
    grid_b = dict(x0=-40.0, y0=-40.0, z0=-40.0, log2_L0=-5, n_levels=12, log2_M=17)
    got_a = _noalloc_sort(ph_a, 14)
    got_b = _noalloc_sort(ph_b, 17, grid_b)
    ref_a = _context_sort(ph_a, 14)
    ref_b = _context_sort(ph_b, 17, grid_b)
    for got, ref in ((got_a, ref_a), (got_b, ref_b)):
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)
    # and once more on the first set, after the larger one
    again = _noalloc_sort(ph_a, 14)
    for g, r in zip(again, ref_a):
        assert np.array_equal(g, r)


def test_noalloc_rejects_sizes_beyond_its_limit():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    f = _entry()
    # checked on the host before any launch: no buffers are touched
    assert f(None, 65537, 17, None, None, None, None, None) == nv.SPH_ERR_INVALID_ARG
    assert f(None, 10, 18, None, None, None, None, None) == nv.SPH_ERR_INVALID_ARG
