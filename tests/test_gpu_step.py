"""Leapfrog update (Eqs. 12-16) and whole steps through the C ABI against the
FP64 oracle."""
import numpy as np
import pytest

from helpers import err, need_gpu
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def test_integrate_matches_oracle_bitwise(orc):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    rng = np.random.default_rng(0)
    n, ng = 3001, 1200
    r = rng.normal(size=(3, n))
    v = rng.normal(size=(3, n))
    e = rng.uniform(0.1, 1, ng)
    acc = rng.normal(size=(ng, 4)).astype(np.float32)
    grav = rng.normal(size=(n, 4)).astype(np.float32)
    mass = rng.uniform(1, 2, n).astype(np.float32)
    h = rng.uniform(0.1, 0.2, ng).astype(np.float32)
    dt = 1e-3
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    tr, tv, te = cu(r.ravel()), cu(v.ravel()), cu(e)
    tvs, tes = torch.zeros_like(tv), torch.zeros_like(te)
    pm = torch.empty((n, 4), device="cuda")
    ph = torch.empty((ng, 4), device="cuda")
    ve = torch.empty((ng, 4), device="cuda")
    nv.integrate_step(nv.SPH_PREDICT, dt, n, ng, tr, tv, te, tvs, tes, cu(acc), cu(grav),
                      cu(mass), cu(h), pm, ph, ve)
    acc2 = rng.normal(size=(ng, 4)).astype(np.float32)
    grav2 = rng.normal(size=(n, 4)).astype(np.float32)
    nv.integrate_step(nv.SPH_CORRECT, dt, n, ng, tr, tv, te, tvs, tes, cu(acc2), cu(grav2),
                      cu(mass), cu(h), None, None, ve)
    torch.cuda.synchronize()

    ro, vo, eo = r.copy(), v.copy(), e.copy()
    vs, es = np.zeros_like(vo), np.zeros_like(eo)
    orc.predict(ng, dt, ro, vo, eo, vs, es, acc[:, :3].astype(np.float64), acc[:, 3].astype(np.float64),
                grav[:, :3].astype(np.float64))
    pm_ref = np.empty((n, 4), np.float32)
    pm_ref[:, :3] = ro.T
    pm_ref[:, 3] = mass
    assert np.array_equal(pm.cpu().numpy(), pm_ref)
    assert np.array_equal(ph.cpu().numpy()[:, 3], h)
    orc.correct(ng, dt, vo, eo, vs, es, acc2[:, :3].astype(np.float64),
                acc2[:, 3].astype(np.float64), grav2[:, :3].astype(np.float64))
    assert np.array_equal(tr.cpu().numpy(), ro.ravel())
    assert np.array_equal(tv.cpu().numpy(), vo.ravel())
    assert np.array_equal(te.cpu().numpy(), eo)
    ve_ref = np.empty((ng, 4), np.float32)
    ve_ref[:, :3] = vo[:, :ng].T
    ve_ref[:, 3] = eo
    assert np.array_equal(ve.cpu().numpy(), ve_ref)


def _run_pair(orc, d, nsteps, dt=1e-3):
    need_gpu()
    from paper_1807_08116_gb300.sim import Simulation
    sim = Simulation(d)
    sim.initial_rhs()
    ref = orc.OracleSim(d["r"].T, d["v"].T, d["e"], d["m"], d["h"], d["n_gas"])
    ref.initial_rhs()
    # the first right-hand side, element by element
    a0 = sim.t["acc_hyd"].cpu().numpy().astype(np.float64)
    g0 = sim.t["grav"].cpu().numpy().astype(np.float64)
    res = dict(grav0=err(g0[:, :3], ref.grav))
    if d["n_gas"]:
        res["hydro0"] = err(a0[:, :3], ref.a_hyd)
        res["rho0"] = err(sim.t["rho"].cpu().numpy(), ref.rho)
    for _ in range(nsteps):
        sim.step(dt)
        ref.step(dt)
    return sim, ref, res


def test_single_halo_rhs_and_ten_steps(orc):
    # 8192 gas + 8192 dark, 1 RHS + 10 steps of dt = 1e-3
    d = ics.single_halo(8192, 8192, seed=0)
    sim, ref, res = _run_pair(orc, d, 10)
    print({k: f"rms {v[0]:.2e} max {v[1]:.2e}" for k, v in res.items()})
    assert res["grav0"][0] <= 1e-6 and res["grav0"][1] <= 1e-4
    assert res["hydro0"][0] <= 1e-6 and res["hydro0"][1] <= 1e-4
    assert res["rho0"][0] <= 1e-6
    r = sim.positions()
    v = sim.velocities()
    dr = np.abs(r - ref.r.T).max()
    rv, mv = err(v, ref.v.T)
    e = sim.t["e"].cpu().numpy()
    re_, me_ = err(e, ref.e)
    print(f"after 10 steps: |dr|max {dr:.2e}, v rms {rv:.2e} max {mv:.2e}, e rms {re_:.2e}")
    # force errors ~1e-7 relative integrate to position errors ~dt^2 |a| 1e-7
    assert dr < 1e-9
    assert rv < 1e-6 and mv < 1e-4
    assert re_ < 1e-6


def test_collisionless_run(orc):
    d = ics.single_halo(0, 4096, seed=4)
    sim, ref, res = _run_pair(orc, d, 5)
    assert res["grav0"][0] <= 1e-6
    assert np.abs(sim.positions() - ref.r.T).max() < 1e-9


def test_conservation_two_halo():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.sim import Simulation
    d = ics.two_halo(16384, 16384, seed=3)
    sim = Simulation(d, grav_flags=nv.SPH_GRAV_POTENTIAL)
    sim.initial_rhs()
    d0 = sim.diagnostics()
    E0 = d0["kinetic"] + d0["thermal"] + d0["potential"]
    for _ in range(20):
        sim.step(1e-3)
    d1 = sim.diagnostics()
    E1 = d1["kinetic"] + d1["thermal"] + d1["potential"]
    pscale = np.sqrt(2 * d0["kinetic"] * d0["mass"])
    print(f"dE/E {abs(E1 - E0) / abs(E0):.2e}, dp {np.abs(d1['momentum'] - d0['momentum']).max() / pscale:.2e}")
    assert abs(E1 - E0) < 1e-4 * abs(E0)
    assert np.abs(d1["momentum"] - d0["momentum"]).max() < 1e-6 * pscale


def test_rerun_is_bitwise_identical():
    need_gpu()
    from paper_1807_08116_gb300.sim import Simulation
    d = ics.two_halo(4096, 4096, seed=8)
    outs = []
    for _ in range(2):
        sim = Simulation(d)
        sim.initial_rhs()
        for _ in range(3):
            sim.step(1e-3)
        outs.append((sim.positions(), sim.velocities(), sim.t["e"].cpu().numpy()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_step_size_from_cfl_condition(orc):
    need_gpu()
    from paper_1807_08116_gb300.sim import Simulation
    d = ics.single_halo(4096, 4096, seed=6)
    sim = Simulation(d)
    sim.initial_rhs()
    dt = sim.cfl_dt(0.5)
    ref = orc.OracleSim(d["r"].T, d["v"].T, d["e"], d["m"], d["h"], d["n_gas"])
    ref.initial_rhs()
    ng = d["n_gas"]
    Q = ref.a_hyd + ref.grav[:ng]
    odt, _ = orc.cfl_dt(ref.pos_h(), ref.vel_e(), ref.rho.astype(np.float32), Q, ref.dedt, C=0.5)
    assert 0 < dt < 1
    assert abs(dt - odt) < 1e-4 * odt
    sim.step(dt)      # and the step accepts it
