"""pp_gravity_rows, the per-GPU share of the particle partition (Sect. 3:
N/k particles per GPU), through the C ABI: row ranges against the FP64 oracle,
bitwise equal to the same rows of pp_gravity under the same plan, and the
sharding module on one rank."""
import numpy as np
import pytest

from helpers import MAX_TOL, RMS_TOL, err, need_gpu, pos_m_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def test_rows_match_the_oracle_and_the_whole_launch(orc):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    d = ics.two_halo(2500, 2000, seed=71)
    pm = pos_m_of(d["r"], d["m"])
    n = len(pm)
    x = torch.as_tensor(pm, device="cuda")
    ranges = [(0, n), (0, 1), (1000, 1001), (5, 777), (n - 3, n), (2048, 4096 + 513)]
    acc, pot = orc.gravity(pm)
    for R in (2, 4, 8):
        nv.sph_gravity_tune(R, 1)
        try:
            whole = torch.empty_like(x)
            nv.pp_gravity(x, whole, flags=nv.SPH_GRAV_POTENTIAL)
            for i0, i1 in ranges:
                out = torch.full((i1 - i0, 4), float("nan"), device="cuda")
                nv.pp_gravity_rows(x, i0, i1, out, flags=nv.SPH_GRAV_POTENTIAL)
                torch.cuda.synchronize()
                assert torch.equal(out, whole[i0:i1]), (R, i0, i1)
        finally:
            nv.sph_gravity_tune(0)
    # the planned (unforced) launch of each range against the oracle
    for i0, i1 in ranges:
        out = torch.empty((i1 - i0, 4), device="cuda")
        nv.pp_gravity_rows(x, i0, i1, out, flags=nv.SPH_GRAV_POTENTIAL)
        torch.cuda.synchronize()
        g = out.cpu().numpy().astype(np.float64)
        rms, mx = err(g[:, :3], acc[i0:i1])
        assert rms <= RMS_TOL and mx <= MAX_TOL, (i0, i1, rms, mx)
        prms, pmx = err(g[:, 3:], pot[i0:i1, None])
        assert prms <= RMS_TOL and pmx <= MAX_TOL, (i0, i1)
    assert nv.pp_gravity_status() == 0


def test_rows_arguments():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    x = torch.zeros((10, 4), device="cuda")
    out = torch.zeros((0, 4), device="cuda")
    nv.pp_gravity_rows(x, 4, 4, out)             # empty range: no-op
    for i0, i1 in ((-1, 2), (3, 2), (0, 11)):
        rc = nv.lib().pp_gravity_rows(x.data_ptr(), 10, i0, i1, 1.0, 0.01, out.data_ptr(), 0, None)
        assert rc == nv.SPH_ERR_INVALID_ARG


def test_sharded_gravity_on_one_rank_is_the_whole_set():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.shard import owned_rows, sharded_gravity
    d = ics.single_halo(3000, 3001, seed=72)
    pm = torch.as_tensor(pos_m_of(d["r"], d["m"]), device="cuda")
    n = pm.shape[0]
    assert owned_rows(n) == (0, n)
    out = torch.empty_like(pm)
    sharded_gravity(pm, n, out)
    ref = torch.empty_like(pm)
    nv.pp_gravity_rows(pm, 0, n, ref)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
