"""Failure detection on the device without a fault: a bounded mbarrier wait
that cannot complete (a transaction no copy will bring) runs out after a
short limit, the kernel records SPH_FLAG_TIMEOUT and returns, the host reads
the status through the C ABI, and the context stays usable."""
import time

import numpy as np
import pytest

from helpers import need_gpu, pos_m_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports(orc):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    assert nv.pp_gravity_status() == 0
    nv.sph_set_wait_limit_ns(5_000_000)          # 5 ms
    try:
        t0 = time.perf_counter()
        nv.sph_wait_probe()
        torch.cuda.synchronize()
        took = time.perf_counter() - t0
        flags = nv.pp_gravity_status()
        assert flags == nv.SPH_FLAG_TIMEOUT
        assert took < 1.0                        # gave up after the short limit
        assert nv.pp_gravity_status() == 0       # read and cleared
    finally:
        nv.sph_set_wait_limit_ns(0)
    # the context is intact: the TMA-fed kernel still runs and agrees with the oracle
    d = ics.single_halo(2048, 2048, seed=9)
    pm = pos_m_of(d["r"], d["m"])
    x = torch.as_tensor(pm, device="cuda")
    out = torch.empty_like(x)
    nv.pp_gravity(x, out)
    torch.cuda.synchronize()
    assert nv.pp_gravity_status() == 0
    g, _ = orc.gravity(pm)
    a = out[:, :3].cpu().numpy().astype(np.float64)
    assert np.sqrt(((a - g) ** 2).sum() / (g ** 2).sum()) < 1e-6


def test_wait_limit_rejects_out_of_range():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    for bad in (-1, 10, 61_000_000_000):
        with pytest.raises(nv.SphError) as ex:
            nv.sph_set_wait_limit_ns(bad)
        assert ex.value.code == nv.SPH_ERR_INVALID_ARG
