"""The allocation-free grid sort (sph_bin_and_sort_noalloc) against the
context-based sph_bin_and_sort and against the oracle's binning and stable
counting sort, bit for bit.

The allocation-free entry point exists for callers that cannot allocate
device memory (a framework that owns all device memory, a plugin given only
its buffers, a loop that must not call cudaMalloc); its scratch is a fixed
device array inside the library.  This file is collected last on purpose: if
it fails, a run that stops at the first failure has already run every other
test.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from helpers import need_gpu, pos_h_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "sphgb.h")


def _limit(name):
    """A limit as the public header states it."""
    with open(HEADER) as f:
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", f.read())
    return int(m.group(1))


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


def _context_sort(ph, log2_M, grid=None, want_grid=False):
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
    out = (key.cpu().numpy(), start.cpu().numpy(), perm.cpu().numpy())
    return (out, ctx.grid()) if want_grid else out


def _oracle_sort(orc, ph, grid):
    # the plain definition: bin every particle, then a stable counting sort
    _, _, key = orc.bin_particles(ph, grid)
    _, start, perm = orc.counting_sort(key, 1 << grid["log2_M"])
    return key, start, perm


def test_noalloc_sort_equals_context_sort_twice_in_a_row(orc):
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
    # and directly against the oracle's binning and stable counting sort
    for g, o in zip(got_b, _oracle_sort(orc, ph_b, grid_b)):
        assert np.array_equal(g, o)


def test_noalloc_sort_at_its_largest_size(orc):
    # n_gas and 2^log2_M both at the stated limits with a derived grid: every
    # part of the fixed scratch layout is used at its largest extent
    d = ics.two_halo(32768, 0, seed=13)
    ph = pos_h_of(d["r"], d["h"])
    assert len(ph) == _limit("SPH_NOALLOC_MAX_GAS") == 65536
    log2_M = _limit("SPH_NOALLOC_MAX_LOG2_M")
    got = _noalloc_sort(ph, log2_M)
    ref, g = _context_sort(ph, log2_M, want_grid=True)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    for a, b in zip(got, _oracle_sort(orc, ph, g)):
        assert np.array_equal(a, b)
    # a second call on other data, then the first again: nothing carries over
    o = ics.single_halo(40000, 0, seed=14)
    other = pos_h_of(o["r"], o["h"])
    got_o = _noalloc_sort(other, log2_M)
    for a, b in zip(got_o, _context_sort(other, log2_M)):
        assert np.array_equal(a, b)
    again = _noalloc_sort(ph, log2_M)
    for a, b in zip(again, ref):
        assert np.array_equal(a, b)


def test_noalloc_rejects_sizes_beyond_its_limit():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    f = _entry()
    # checked on the host before any launch: no buffers are touched
    n_max, m_max = _limit("SPH_NOALLOC_MAX_GAS"), _limit("SPH_NOALLOC_MAX_LOG2_M")
    assert f(None, n_max + 1, m_max, None, None, None, None, None) == nv.SPH_ERR_INVALID_ARG
    assert f(None, 10, m_max + 1, None, None, None, None, None) == nv.SPH_ERR_INVALID_ARG
