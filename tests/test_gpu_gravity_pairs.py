"""pp_gravity_pairs (Eq. 4 with every pair evaluated once) through the C ABI
against the FP64 oracle: ragged block counts, the diagonal-only case, the
potential and its self term, bitwise reproducibility, the fall-backs to the
one-sided kernel, and whole simulations that take the pair-once path."""
import numpy as np
import pytest

from helpers import MAX_TOL, RMS_TOL, err, max_plain, need_gpu, pos_m_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture
def low_threshold():
    """Use the pair-once kernel down to n = 1 for the duration of a test."""
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    nv.pp_gravity_pairs_min_n(1)
    try:
        yield nv
    finally:
        nv.pp_gravity_pairs_min_n(0)


def _pairs(pm, G=1.0, eps=0.01, flags=0, work=True):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    x = torch.as_tensor(pm, device="cuda")
    out = torch.full_like(x, float("nan"))
    w = nv.pp_gravity_pairs_workspace(len(pm)) if work else None
    nv.pp_gravity_pairs(x, out, w, G=G, eps=eps, flags=flags)
    torch.cuda.synchronize()
    assert nv.pp_gravity_status() == 0
    return out.cpu().numpy().astype(np.float64)


def _onesided(pm, G=1.0, eps=0.01, flags=0):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    x = torch.as_tensor(pm, device="cuda")
    out = torch.full_like(x, float("nan"))
    nv.pp_gravity(x, out, G=G, eps=eps, flags=flags)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_workspace_size_and_eligibility():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    assert nv.pp_gravity_pairs_workspace_bytes(0) == 4096
    assert nv.pp_gravity_pairs_workspace_bytes(1000) == 4096 + 32 * 1000
    assert nv.pp_gravity_pairs_eligible(16384, 0.01)
    assert not nv.pp_gravity_pairs_eligible(16383, 0.01)
    assert not nv.pp_gravity_pairs_eligible(1 << 20, 0.0)            # unsoftened
    assert not nv.pp_gravity_pairs_eligible(1 << 20, 0.01, nv.SPH_GRAV_NO_KAHAN)
    nv.sph_gravity_tune(4, 1)
    try:
        assert not nv.pp_gravity_pairs_eligible(1 << 20, 0.01)       # a fixed one-sided plan
    finally:
        nv.sph_gravity_tune(0)


@pytest.mark.parametrize("n", [1, 2, 33, 1023, 1024, 1025, 2048, 2049, 5000, 9999])
def test_ragged_block_counts(orc, low_threshold, n):
    # 1 block (diagonal tile only) up to 10 blocks with a ragged last block
    nv = low_threshold
    rng = np.random.default_rng(n)
    pm = pos_m_of(rng.normal(size=(n, 3)), rng.uniform(0.5, 1.5, n) / n)
    g = _pairs(pm, G=0.7, eps=0.05, flags=nv.SPH_GRAV_POTENTIAL)
    acc, pot = orc.gravity(pm, G=0.7, eps=0.05)
    if n == 1:
        assert np.all(g == 0.0)      # the self term of the potential cancels exactly
        return
    rms, mx = err(g[:, :3], acc)
    assert rms <= RMS_TOL and mx <= MAX_TOL, (rms, mx)
    prms, pmx = err(g[:, 3:], pot[:, None])
    assert prms <= RMS_TOL and pmx <= MAX_TOL, (prms, pmx)


@pytest.mark.parametrize("case", ["equal", "one_block_heavier", "ragged_equal", "one_body_off"])
def test_equal_mass_tiles(orc, low_threshold, case):
    # tiles whose bodies all share one mass take the sums without the mass
    # factors; tiles with another mass, a body off by one ulp, or a ragged
    # last block take the general form: both against the oracle, with the
    # potential, and the two forms agree where they meet
    nv = low_threshold
    n = 5000 if case == "ragged_equal" else 5120
    rng = np.random.default_rng(11)
    m = np.full(n, 1.0 / n, np.float32)
    if case == "one_block_heavier":
        m[2048:3072] *= np.float32(3.0)
    if case == "one_body_off":
        m[777] = np.nextafter(m[777], np.float32(1.0))
    pm = pos_m_of(rng.normal(size=(n, 3)), m)
    g = _pairs(pm, G=0.7, eps=0.05, flags=nv.SPH_GRAV_POTENTIAL)
    acc, pot = orc.gravity(pm, G=0.7, eps=0.05)
    rms, mx = err(g[:, :3], acc)
    assert rms <= RMS_TOL and mx <= MAX_TOL, (case, rms, mx)
    prms, pmx = err(g[:, 3:], pot[:, None])
    assert prms <= RMS_TOL and pmx <= MAX_TOL, (case, prms, pmx)
    mm = pm[:, 3].astype(np.float64)
    assert np.abs((mm[:, None] * g[:, :3]).sum(0)).max() < 1e-5 * (mm[:, None] * np.abs(g[:, :3])).sum()


def test_single_halo_all_rows_and_momentum(orc, low_threshold):
    nv = low_threshold
    d = ics.single_halo(8192, 8192, seed=0)
    pm = pos_m_of(d["r"], d["m"])
    g = _pairs(pm, flags=nv.SPH_GRAV_POTENTIAL)
    acc, pot = orc.gravity(pm)
    rms, mx = err(g[:, :3], acc)
    print(f"pairs 16384: rms {rms:.2e} max {mx:.2e} (plain max "
          f"{max_plain(g[:, :3], acc):.2e})")
    assert rms <= RMS_TOL and mx <= MAX_TOL
    prms, pmx = err(g[:, 3:], pot[:, None])
    assert prms <= RMS_TOL and pmx <= MAX_TOL
    # each pair's two contributions are exact negatives before the fixed-point
    # rounding of the tile sums: total momentum change at that rounding level
    m = pm[:, 3].astype(np.float64)
    assert np.abs((m[:, None] * g[:, :3]).sum(0)).max() < 1e-5 * (m[:, None] * np.abs(g[:, :3])).sum()


def test_bitwise_reproducible(low_threshold):
    rng = np.random.default_rng(3)
    n = 70001
    pm = pos_m_of(rng.normal(size=(n, 3)), rng.uniform(0.5, 1.5, n) / n)
    a = _pairs(pm, flags=low_threshold.SPH_GRAV_POTENTIAL)
    b = _pairs(pm, flags=low_threshold.SPH_GRAV_POTENTIAL)
    assert np.array_equal(a, b)


def test_fallbacks_equal_onesided(low_threshold):
    nv = low_threshold
    rng = np.random.default_rng(5)
    pm = pos_m_of(rng.uniform(-1, 1, size=(3000, 3)), np.full(3000, 1e-3))
    # unsoftened: the one-sided kernel with its coincident-pair guard
    assert np.array_equal(_pairs(pm, eps=0.0), _onesided(pm, eps=0.0))
    # NO_KAHAN asks for the one-sided plain sums
    f = nv.SPH_GRAV_NO_KAHAN
    assert np.array_equal(_pairs(pm, flags=f), _onesided(pm, flags=f))
    # no scratch
    assert np.array_equal(_pairs(pm, work=False), _onesided(pm))
    # a fixed one-sided plan
    nv.sph_gravity_tune(2, 1)
    try:
        assert np.array_equal(_pairs(pm), _onesided(pm))
    finally:
        nv.sph_gravity_tune(0)


def test_scale_follows_units(orc, low_threshold):
    # the fixed-point scale comes from sum |m| and eps: tiny and huge unit
    # systems give the same relative accuracy
    rng = np.random.default_rng(8)
    n = 3000
    r = rng.normal(size=(n, 3))
    m = rng.uniform(0.5, 1.5, n) / n
    for L, M in ((1e-6, 1e-20), (1e5, 1e25)):
        pm = pos_m_of(r * L, m * M)
        g = _pairs(pm, G=1.0, eps=0.05 * L)
        acc, _ = orc.gravity(pm, G=1.0, eps=0.05 * L)
        rms, mx = err(g[:, :3], acc)
        assert rms <= RMS_TOL and mx <= MAX_TOL, (L, M, rms, mx)


def test_two_halo_sampled_rows(orc):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    d = ics.two_halo(131072, 131072, seed=1)
    pm = pos_m_of(d["r"], d["m"])
    assert nv.pp_gravity_pairs_eligible(len(pm), 0.01)
    g = _pairs(pm, flags=nv.SPH_GRAV_POTENTIAL)
    rows = np.random.default_rng(0).choice(len(pm), 512, replace=False)
    acc, pot = orc.gravity(pm, rows=rows)
    rms, mx = err(g[rows, :3], acc)
    print(f"pairs 524288 sample: rms {rms:.2e} max {mx:.2e} (plain max "
          f"{max_plain(g[rows, :3], acc):.2e})")
    assert rms <= RMS_TOL and mx <= MAX_TOL
    prms, pmx = err(g[rows, 3:], pot[:, None])
    assert prms <= RMS_TOL and pmx <= MAX_TOL


def test_large_collision_sampled_rows(orc):
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    d = ics.two_halo(1048576, 1048576, seed=2)
    pm = pos_m_of(d["r"], d["m"])
    g = _pairs(pm)
    rows = np.random.default_rng(1).choice(len(pm), 256, replace=False)
    acc, _ = orc.gravity(pm, rows=rows)
    rms, mx = err(g[rows, :3], acc)
    print(f"pairs 4194304 sample: rms {rms:.2e} max {mx:.2e} (plain max "
          f"{max_plain(g[rows, :3], acc):.2e})")
    assert rms <= RMS_TOL and mx <= MAX_TOL
    # the one-sided kernel (per-tile Kahan sums) on the same rows, for the
    # record: the pair-once kernel's in-tile sums are plain FP32, its sums
    # across tiles exact in fixed point
    torch = need_gpu()
    x = torch.as_tensor(pm, device="cuda")
    o = torch.empty_like(x)
    nv.pp_gravity(x, o)
    torch.cuda.synchronize()
    g1 = o.cpu().numpy().astype(np.float64)
    rms1, mx1 = err(g1[rows, :3], acc)
    print(f"one-sided (Kahan) 4194304 same rows: rms {rms1:.2e} max {mx1:.2e} (plain max "
          f"{max_plain(g1[rows, :3], acc):.2e})")
    assert rms1 <= RMS_TOL and mx1 <= MAX_TOL


def test_simulation_takes_pair_path(orc):
    need_gpu()
    from paper_1807_08116_gb300.sim import Simulation
    d = ics.two_halo(32768, 32768, seed=12)
    sim = Simulation(d)
    assert "grav_work" in sim.t
    sim.initial_rhs()
    rows = np.random.default_rng(2).choice(d["n"], 256, replace=False)
    pm = pos_m_of(d["r"], d["m"])
    acc, _ = orc.gravity(pm, rows=rows)
    g = sim.t["grav"].cpu().numpy().astype(np.float64)
    rms, mx = err(g[rows, :3], acc)
    assert rms <= RMS_TOL and mx <= MAX_TOL
    sim.step(1e-3)
    # the same run with the one-sided kernel agrees to force rounding
    ref = Simulation(d, pairs=False)
    assert "grav_work" not in ref.t
    ref.initial_rhs()
    ref.step(1e-3)
    rv, _ = err(sim.velocities(), ref.velocities())
    assert rv < 1e-6


def _batch_ics():
    # uneven sizes across block boundaries, a gas-free and a dark-free one,
    # and a 3-body simulation (one diagonal tile)
    return [ics.two_halo(3000, 2500, seed=31), ics.single_halo(0, 1800, seed=32),
            ics.single_halo(1300, 0, seed=33), ics.two_halo(700, 900, seed=34),
            ics.single_halo(2, 1, seed=35)]


@pytest.mark.parametrize("shape", [(128, 8), (128, 6), (128, 10), (256, 8)])
def test_batched_matches_oracle_per_simulation(orc, low_threshold, shape):
    # every block shape a plan may name: blocks of 1024, 768, 1280, 2048 bodies
    torch = need_gpu()
    nv = low_threshold
    from paper_1807_08116_gb300.sim import assemble_batch
    lst = _batch_ics()
    ic, go, do, so = assemble_batch(lst)
    batch = nv.Batch(go, do, torch.as_tensor(so, device="cuda"))
    pm = torch.as_tensor(pos_m_of(ic["r"], ic["m"]), device="cuda")
    work = nv.pp_gravity_pairs_workspace(pm.shape[0])
    nv.pp_gravity_pairs_plan(*shape)
    try:
        out = torch.full_like(pm, float("nan"))
        nv.pp_gravity_pairs_batched(batch, pm, out, work, flags=nv.SPH_GRAV_POTENTIAL)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        again = torch.full_like(pm, float("nan"))
        nv.pp_gravity_pairs_batched(batch, pm, again, work, flags=nv.SPH_GRAV_POTENTIAL)
        assert np.array_equal(again.cpu().numpy().astype(np.float64), got)   # reproducible
    finally:
        nv.pp_gravity_pairs_plan(0)
    for s, d in enumerate(lst):
        cols = np.concatenate([np.arange(go[s], go[s + 1]), ic["n_gas"] + np.arange(do[s], do[s + 1])])
        acc, pot = orc.gravity(pos_m_of(d["r"], d["m"]))
        rms, mx = err(got[cols, :3], acc)
        assert rms <= RMS_TOL and mx <= MAX_TOL, (s, rms, mx)
        prms, pmx = err(got[cols, 3:], pot[:, None])
        assert prms <= RMS_TOL and pmx <= MAX_TOL, (s, prms, pmx)


def test_batched_mixed_and_equal_masses(orc, low_threshold):
    # one simulation of the batch with unequal masses (its full tiles take the
    # general form) beside equal-mass ones (their full tiles take the
    # equal-mass form): each against the oracle on its own
    torch = need_gpu()
    nv = low_threshold
    from paper_1807_08116_gb300.sim import assemble_batch
    lst = _batch_ics()
    rng = np.random.default_rng(36)
    lst[0] = dict(lst[0], m=lst[0]["m"] * rng.uniform(0.5, 1.5, len(lst[0]["m"])))
    ic, go, do, so = assemble_batch(lst)
    batch = nv.Batch(go, do, torch.as_tensor(so, device="cuda"))
    pm = torch.as_tensor(pos_m_of(ic["r"], ic["m"]), device="cuda")
    work = nv.pp_gravity_pairs_workspace(pm.shape[0])
    out = torch.full_like(pm, float("nan"))
    nv.pp_gravity_pairs_batched(batch, pm, out, work, flags=nv.SPH_GRAV_POTENTIAL)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    for s, d in enumerate(lst):
        cols = np.concatenate([np.arange(go[s], go[s + 1]), ic["n_gas"] + np.arange(do[s], do[s + 1])])
        acc, pot = orc.gravity(pos_m_of(d["r"], d["m"]))
        rms, mx = err(got[cols, :3], acc)
        assert rms <= RMS_TOL and mx <= MAX_TOL, (s, rms, mx)
        prms, pmx = err(got[cols, 3:], pot[:, None])
        assert prms <= RMS_TOL and pmx <= MAX_TOL, (s, prms, pmx)


def test_batched_falls_back_without_scratch():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.sim import assemble_batch
    ic, go, do, so = assemble_batch(_batch_ics())
    batch = nv.Batch(go, do, torch.as_tensor(so, device="cuda"))
    pm = torch.as_tensor(pos_m_of(ic["r"], ic["m"]), device="cuda")
    a, b = torch.empty_like(pm), torch.empty_like(pm)
    nv.pp_gravity_pairs_batched(batch, pm, a, None)      # no scratch: the one-sided batch kernel
    nv.pp_gravity_batched(batch, pm, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_batched_simulation_takes_pair_path(orc):
    need_gpu()
    from paper_1807_08116_gb300.sim import Simulation, assemble_batch
    lst = [ics.two_halo(20000, 20000, seed=51), ics.single_halo(15000, 15000, seed=52)]
    ic, go, do, so = assemble_batch(lst)
    b = Simulation(ic, batch_offsets=(go, do, so))
    assert "grav_work" in b.t
    b.initial_rhs()
    g = b.t["grav"].cpu().numpy().astype(np.float64)
    for s, d in enumerate(lst):
        cols = b.sim_slices(s)
        rows = np.random.default_rng(s).choice(len(cols), 200, replace=False)
        acc, _ = orc.gravity(pos_m_of(d["r"], d["m"]), rows=rows)
        rms, mx = err(g[cols][rows, :3], acc)
        assert rms <= RMS_TOL and mx <= MAX_TOL, (s, rms, mx)


def test_batched_pair_path_graph_replay_equals_step():
    torch = need_gpu()
    from paper_1807_08116_gb300.sim import Simulation, assemble_batch
    lst = [ics.two_halo(20000, 20000, seed=53), ics.single_halo(15000, 15000, seed=54)]
    ic, go, do, so = assemble_batch(lst)
    a = Simulation(ic, batch_offsets=(go, do, so))
    b = Simulation(ic, batch_offsets=(go, do, so))
    for sim in (a, b):
        sim.initial_rhs()
        sim.step(1e-3)
    b.capture(1e-3)
    for _ in range(2):
        a.step(1e-3)
        b.replay()
    torch.cuda.synchronize()
    assert np.array_equal(a.positions(), b.positions())
    assert np.array_equal(a.velocities(), b.velocities())


def test_threshold_autotuner():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.tune import tune_pairs_threshold

    def make(n):
        q = n // 4
        d = ics.two_halo(q, q, seed=60)
        return torch.as_tensor(pos_m_of(d["r"], d["m"]), device="cuda")
    try:
        thr, res = tune_pairs_threshold(make, sizes=(4096, 65536, 131072), reps=2)
        assert set(res) == {4096, 65536, 131072}
        # the timed crossover is applied, and the pair-once kernel wins at the top
        assert res[131072][1] < res[131072][0]
        assert thr is not None and thr <= 131072
        assert nv.pp_gravity_pairs_eligible(thr, 0.01)
        assert not nv.pp_gravity_pairs_eligible(thr - 1, 0.01)
    finally:
        nv.pp_gravity_pairs_min_n(0)
    assert nv.pp_gravity_pairs_eligible(16384, 0.01)


def test_batched_scale_per_simulation(orc, low_threshold):
    # simulations of very different mass (and unit) scales in one batch: each
    # keeps the fixed-point resolution of its own sum |m|
    torch = need_gpu()
    nv = low_threshold
    from paper_1807_08116_gb300.sim import assemble_batch
    a = ics.two_halo(3000, 2500, seed=61)
    b = ics.single_halo(1300, 900, seed=62)
    b = dict(b, m=b["m"] * 1e-10, r=b["r"] * 1e-3)
    lst = [a, b]
    ic, go, do, so = assemble_batch(lst)
    batch = nv.Batch(go, do, torch.as_tensor(so, device="cuda"))
    pm = torch.as_tensor(pos_m_of(ic["r"], ic["m"]), device="cuda")
    out = torch.full_like(pm, float("nan"))
    nv.pp_gravity_pairs_batched(batch, pm, out, nv.pp_gravity_pairs_workspace(pm.shape[0]),
                                eps=1e-5, flags=nv.SPH_GRAV_POTENTIAL)
    torch.cuda.synchronize()
    assert nv.pp_gravity_status() == 0
    got = out.cpu().numpy().astype(np.float64)
    for s, d in enumerate(lst):
        cols = np.concatenate([np.arange(go[s], go[s + 1]), ic["n_gas"] + np.arange(do[s], do[s + 1])])
        acc, pot = orc.gravity(pos_m_of(d["r"], d["m"]), eps=1e-5)
        rms, mx = err(got[cols, :3], acc)
        assert rms <= RMS_TOL and mx <= MAX_TOL, (s, rms, mx)
        prms, pmx = err(got[cols, 3:], pot[:, None])
        assert prms <= RMS_TOL and pmx <= MAX_TOL, (s, prms, pmx)
