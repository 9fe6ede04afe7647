"""The time step of Eq. 17 taken inside the force pass (sph_forces_cfl) and the
adaptive step built on it (sph_step_cfl): bitwise equal to the standalone
sph_cfl_dt and to a fixed step of the same size, and capturable in a CUDA
graph."""
import numpy as np
import pytest

from helpers import need_gpu
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def _sim(seed=70, n=4096):
    need_gpu()
    from paper_1807_08116_gb300.sim import Simulation
    sim = Simulation(ics.single_halo(n, n, seed=seed))
    sim.initial_rhs()
    return sim


def test_fused_time_step_equals_standalone():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    sim = _sim()
    sim.step(1e-3)
    t, ng = sim.t, sim.n_gas
    m = t["mass"][:ng]
    # forces at the current state, then the standalone step
    nv.sph_forces(sim.ctx, t["vel_e"], t["rho"], m, t["acc_hyd"])
    acc_a = t["acc_hyd"].clone()
    dt_a = torch.empty(1, dtype=torch.float32, device="cuda")
    dti_a = torch.empty(ng, dtype=torch.float32, device="cuda")
    nv.sph_cfl_dt(sim.ctx, t["vel_e"], t["rho"], m, acc_a, t["grav"], 0.5, dt_a, dti_a)
    # the same in one pass
    acc_b = torch.full_like(acc_a, float("nan"))
    dt_b = torch.empty(1, dtype=torch.float32, device="cuda")
    dti_b = torch.empty(ng, dtype=torch.float32, device="cuda")
    nv.sph_forces_cfl(sim.ctx, ng, t["vel_e"], t["rho"], m, acc_b, t["grav"], 0.5, 1.0, dt_b, dti_b)
    torch.cuda.synchronize()
    assert torch.equal(acc_a, acc_b)
    assert torch.equal(dti_a, dti_b)
    assert float(dt_a) == float(dt_b) and 0 < float(dt_b) < 1
    # the cap
    nv.sph_forces_cfl(sim.ctx, ng, t["vel_e"], t["rho"], m, acc_b, t["grav"], 0.5, 1e-9, dt_b)
    assert float(dt_b) == np.float32(1e-9)


@pytest.mark.parametrize("lanes", [1, 4])
def test_adaptive_steps_equal_fixed_steps(lanes):
    need_gpu()
    a, b = _sim(71), _sim(71)
    a.set_lanes(lanes)
    b.set_lanes(lanes)
    dts = []
    for _ in range(3):
        dt = float(a.step_cfl(C=0.5, dt_max=1e-2).item())   # first: right after the initial RHS
        dts.append(dt)
        b.step(dt)
    assert all(0 < d <= 1e-2 for d in dts)
    assert np.array_equal(a.positions(), b.positions())
    assert np.array_equal(a.velocities(), b.velocities())
    # each step's size is min(dt_max, the standalone Eq. 17 value) at the state
    # the step started from (forces refreshed there first)
    from paper_1807_08116_gb300 import native as nv
    c = _sim(71)
    c.set_lanes(lanes)
    for d in dts:
        expect = min(np.float32(1e-2), np.float32(c.cfl_dt(0.5)))
        assert expect == np.float32(d)
        c.step(d)
        t = c.t
        nv.sph_forces(c.ctx, t["vel_e"], t["rho"], t["mass"][:c.n_gas], t["acc_hyd"])


def test_adaptive_step_in_a_graph():
    torch = need_gpu()
    a, b = _sim(72), _sim(72)
    for sim in (a, b):
        sim.step_cfl()
    b.capture_cfl()
    for _ in range(3):
        da = float(a.step_cfl().item())
        b.replay()
        torch.cuda.synchronize()
        assert float(b.dt_used.item()) == da
    assert np.array_equal(a.positions(), b.positions())


def test_adaptive_step_needs_gas():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.sim import Simulation
    sim = Simulation(ics.single_halo(0, 2048, seed=73))
    sim.initial_rhs()
    with pytest.raises(nv.SphError) as ex:
        sim.step_cfl()
    assert ex.value.code == nv.SPH_ERR_INVALID_ARG
