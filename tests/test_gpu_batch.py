"""Batches of independent simulations (the ensemble form): batched gravity is
bitwise equal to per-simulation launches; batched steps reproduce separate
runs; a CUDA-graph replay of a step equals the step."""
import numpy as np
import pytest

from helpers import err, need_gpu, pos_m_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def _ics():
    # uneven sizes, one gas-free and one dark-free simulation, a 3-particle one
    out = [ics.two_halo(3000, 2500, seed=31), ics.single_halo(0, 1800, seed=32),
           ics.single_halo(1300, 0, seed=33), ics.two_halo(700, 900, seed=34)]
    tiny = ics.single_halo(2, 1, seed=35)
    out.append(tiny)
    return out


def test_batched_gravity_is_bitwise_per_simulation():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.sim import assemble_batch
    lst = _ics()
    ic, go, do, so = assemble_batch(lst)
    batch = nv.Batch(go, do, torch.as_tensor(so, device="cuda"))
    pm = torch.as_tensor(pos_m_of(ic["r"], ic["m"]), device="cuda")
    for R in (2, 4, 8):
        batch.set_plan(R)
        out = torch.full_like(pm, float("nan"))
        nv.pp_gravity_batched(batch, pm, out, flags=nv.SPH_GRAV_POTENTIAL)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        nv.sph_gravity_tune(R, 1)
        try:
            for s, d in enumerate(lst):
                cols = np.concatenate([np.arange(go[s], go[s + 1]), ic["n_gas"] + np.arange(do[s], do[s + 1])])
                x = torch.as_tensor(pos_m_of(d["r"], d["m"]), device="cuda")
                o = torch.empty_like(x)
                nv.pp_gravity(x, o, flags=nv.SPH_GRAV_POTENTIAL)
                torch.cuda.synchronize()
                assert np.array_equal(got[cols], o.cpu().numpy()), (R, s)
        finally:
            nv.sph_gravity_tune(0)
    assert nv.pp_gravity_status() == 0


@pytest.mark.parametrize("pairs", [False, True])
def test_batched_steps_match_separate_runs(orc, pairs):
    # pairs=False: the batch and the lone runs use the one-sided gravity
    # kernels and agree to 1e-7; pairs=True: the batch (17,300 bodies) takes
    # the pair-once kernel while the lone runs stay one-sided, so they agree
    # to the force tolerance
    need_gpu()
    from paper_1807_08116_gb300.sim import Simulation, assemble_batch
    lst = _ics()[:4]
    ic, go, do, so = assemble_batch(lst)
    b = Simulation(ic, batch_offsets=(go, do, so), pairs=pairs)
    assert ("grav_work" in b.t) == pairs
    b.initial_rhs()
    singles = [Simulation(d, pairs=False) for d in lst]
    for s in singles:
        s.initial_rhs()
    for _ in range(3):
        b.step(1e-3)
        for s in singles:
            s.step(1e-3)
    rb, vb = b.positions(), b.velocities()
    for s, sim in enumerate(singles):
        cols = b.sim_slices(s)
        assert np.abs(rb[cols] - sim.positions()).max() < 1e-10
        rv, mv = err(vb[cols], sim.velocities())
        assert rv < (1e-6 if pairs else 1e-7), (s, rv)
    # and the batch against the FP64 oracle on the largest simulation
    d = lst[0]
    ref = orc.OracleSim(d["r"].T, d["v"].T, d["e"], d["m"], d["h"], d["n_gas"])
    ref.initial_rhs()
    for _ in range(3):
        ref.step(1e-3)
    cols = b.sim_slices(0)
    assert np.abs(rb[cols] - ref.r.T).max() < 1e-9


def test_graph_replay_equals_step():
    torch = need_gpu()
    from paper_1807_08116_gb300.sim import Simulation, assemble_batch
    lst = _ics()[:3]
    ic, go, do, so = assemble_batch(lst)
    a = Simulation(ic, batch_offsets=(go, do, so))
    b = Simulation(ic, batch_offsets=(go, do, so))
    for sim in (a, b):
        sim.initial_rhs()
        sim.step(1e-3)
    b.capture(1e-3)
    for _ in range(3):
        a.step(1e-3)
        b.replay()
    torch.cuda.synchronize()
    assert np.array_equal(a.positions(), b.positions())
    assert np.array_equal(a.velocities(), b.velocities())
