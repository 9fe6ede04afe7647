"""pp_gravity (Eq. 4) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from helpers import MAX_TOL, RMS_TOL, err, max_plain, need_gpu, pos_m_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def _gpu_gravity(pm, G=1.0, eps=0.01, flags=0):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    x = torch.as_tensor(pm, device="cuda")
    out = torch.full_like(x, float("nan"))
    nv.pp_gravity(x, out, G=G, eps=eps, flags=flags)
    torch.cuda.synchronize()
    assert nv.pp_gravity_status() == 0
    return out.cpu().numpy().astype(np.float64)


def test_single_halo_all_rows(orc):
    d = ics.single_halo(8192, 8192, seed=0)
    pm = pos_m_of(d["r"], d["m"])
    from paper_1807_08116_gb300 import native as nv
    g = _gpu_gravity(pm, flags=nv.SPH_GRAV_POTENTIAL)
    acc, pot = orc.gravity(pm)
    rms, mx = err(g[:, :3], acc)
    print(f"gravity 16384: rms {rms:.2e} max {mx:.2e} (plain max "
          f"{max_plain(g[:, :3], acc):.2e})")
    assert rms <= RMS_TOL and mx <= MAX_TOL
    prms, pmx = err(g[:, 3:], pot[:, None])
    assert prms <= RMS_TOL and pmx <= MAX_TOL
    # Newton's third law holds to FP32 rounding
    m = pm[:, 3].astype(np.float64)
    assert np.abs((m[:, None] * g[:, :3]).sum(0)).max() < 1e-5 * (m[:, None] * np.abs(g[:, :3])).sum()


@pytest.mark.parametrize("n", [1, 2, 3, 31, 1000, 1023, 1024, 1025, 3000, 4097, 9999])
def test_ragged_sizes(orc, n):
    rng = np.random.default_rng(n)
    pm = pos_m_of(rng.normal(size=(n, 3)), rng.uniform(0.5, 1.5, n) / n)
    from paper_1807_08116_gb300 import native as nv
    g = _gpu_gravity(pm, G=0.7, eps=0.05, flags=nv.SPH_GRAV_POTENTIAL)
    acc, pot = orc.gravity(pm, G=0.7, eps=0.05)
    if n == 1:
        assert np.all(g == 0.0)      # no other body: no force, no potential
        return
    rms, mx = err(g[:, :3], acc)
    assert rms <= RMS_TOL and mx <= MAX_TOL, (rms, mx)
    # the potential leaves j = i out inside the sum (not subtracted after it),
    # so it stays accurate when the self term m_i / eps would dominate
    prms, pmx = err(g[:, 3:], pot[:, None])
    assert prms <= RMS_TOL and pmx <= MAX_TOL, (prms, pmx)


def test_empty_is_noop():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    x = torch.zeros((0, 4), device="cuda")
    nv.pp_gravity(x, x.clone())


def test_unsoftened_and_coincident(orc):
    rng = np.random.default_rng(4)
    pm = pos_m_of(rng.uniform(-1, 1, size=(700, 3)), np.full(700, 1e-3))
    g = _gpu_gravity(pm, eps=0.0)
    acc, _ = orc.gravity(pm, eps=0.0)
    rms, mx = err(g[:, :3], acc)
    assert rms <= RMS_TOL and mx <= MAX_TOL
    two = np.array([[0.5, 0.5, 0.5, 1.0], [0.5, 0.5, 0.5, 2.0]], np.float32)
    assert np.all(_gpu_gravity(two, eps=0.0)[:, :3] == 0.0)


def test_two_halo_sampled_rows(orc):
    d = ics.two_halo(131072, 131072, seed=1)
    pm = pos_m_of(d["r"], d["m"])
    from paper_1807_08116_gb300 import native as nv
    g = _gpu_gravity(pm, flags=nv.SPH_GRAV_POTENTIAL)
    rows = np.random.default_rng(0).choice(len(pm), 512, replace=False)
    acc, pot = orc.gravity(pm, rows=rows)
    rms, mx = err(g[rows, :3], acc)
    print(f"gravity 524288 sample: rms {rms:.2e} max {mx:.2e} (plain max "
          f"{max_plain(g[rows, :3], acc):.2e})")
    assert rms <= RMS_TOL and mx <= MAX_TOL
    prms, pmx = err(g[rows, 3:], pot[:, None])
    assert prms <= RMS_TOL and pmx <= MAX_TOL


def test_large_collision_sampled_rows(orc):
    # the full 2 x (1M gas + 1M dark) collision, launched as the step does
    d = ics.two_halo(1048576, 1048576, seed=2)
    pm = pos_m_of(d["r"], d["m"])
    g = _gpu_gravity(pm)
    rows = np.random.default_rng(1).choice(len(pm), 128, replace=False)
    acc, _ = orc.gravity(pm, rows=rows)
    rms, mx = err(g[rows, :3], acc)
    print(f"gravity 4194304 sample: rms {rms:.2e} max {mx:.2e} (plain max "
          f"{max_plain(g[rows, :3], acc):.2e})")
    assert rms <= RMS_TOL and mx <= MAX_TOL
    assert np.all(np.isfinite(g))


def test_plans_cover_cluster_split_and_determinism():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    R, S = nv.sph_gravity_plan(16384)
    assert S > 1          # small problems split sources over a cluster
    R2, S2 = nv.sph_gravity_plan(4194304)
    assert R2 >= 1 and S2 >= 1
    rng = np.random.default_rng(9)
    pm = pos_m_of(rng.normal(size=(20000, 3)), np.full(20000, 5e-5))
    a = _gpu_gravity(pm)
    b = _gpu_gravity(pm)
    assert np.array_equal(a, b)


def test_compensation_helps(orc):
    d = ics.two_halo(32768, 32768, seed=6)
    pm = pos_m_of(d["r"], d["m"])
    from paper_1807_08116_gb300 import native as nv
    rows = np.arange(0, len(pm), 97)
    acc, _ = orc.gravity(pm, rows=rows)
    k = err(_gpu_gravity(pm)[rows, :3], acc)[0]
    nk = err(_gpu_gravity(pm, flags=nv.SPH_GRAV_NO_KAHAN)[rows, :3], acc)[0]
    print(f"kahan rms {k:.2e}, plain rms {nk:.2e}")
    assert k <= nk * 1.05


@pytest.mark.parametrize("R,S", [(2, 1), (4, 1), (8, 1), (2, 16), (4, 4), (8, 2)])
def test_every_launch_plan(orc, R, S):
    from paper_1807_08116_gb300 import native as nv
    rng = np.random.default_rng(R * 100 + S)
    n = 6001
    pm = pos_m_of(rng.normal(size=(n, 3)), rng.uniform(0.5, 1.5, n) / n)
    acc, pot = orc.gravity(pm)
    need_gpu()
    nv.sph_gravity_tune(R, S)
    try:
        g = _gpu_gravity(pm, flags=nv.SPH_GRAV_POTENTIAL)
    finally:
        nv.sph_gravity_tune(0)
    rms, mx = err(g[:, :3], acc)
    assert rms <= RMS_TOL and mx <= MAX_TOL, (R, S, rms, mx)
    prms, pmx = err(g[:, 3:], pot[:, None])
    assert prms <= RMS_TOL and pmx <= MAX_TOL


def test_autotuner_picks_a_timed_plan(orc):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.tune import tune_gravity
    rng = np.random.default_rng(12)
    pm = pos_m_of(rng.normal(size=(20000, 3)), np.full(20000, 5e-5))
    x = torch.as_tensor(pm, device="cuda")
    try:
        best, res = tune_gravity(x, reps=1)
        assert best in res and res[best] == min(res.values())
        assert nv.sph_gravity_plan(20000) == best
        g = _gpu_gravity(pm)
    finally:
        nv.sph_gravity_tune(0)
    acc, _ = orc.gravity(pm)
    rms, mx = err(g[:, :3], acc)
    assert rms <= RMS_TOL and mx <= MAX_TOL
