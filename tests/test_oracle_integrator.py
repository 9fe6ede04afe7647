"""Pins of the oracle's predictor-corrector scheme (Eqs. 12-16) with gravity
evaluated once per step (Sect. 2.2).

For collisionless particles the scheme with gravity taken at r(t + dt) and
reused by the next predictor is algebraically velocity Verlet:
  r_{n+1} = r_n + dt v_n + dt^2/2 g_n,  v_{n+1} = v_n + dt/2 (g_n + g_{n+1}).
The test integrates that form independently (using the oracle's gravity as a
library primitive, on the same FP32 working copies of the positions) and
compares trajectories.
"""
import numpy as np

from paper_1807_08116_gb300 import ics


def _pos_m(r, m):
    pm = np.empty((r.shape[1], 4), np.float32)
    pm[:, :3] = r.T
    pm[:, 3] = m
    return pm


def test_dark_only_equals_velocity_verlet(orc):
    d = ics.single_halo(0, 512, seed=9)
    r0 = d["r"].T.copy()
    v0 = d["v"].T.copy()
    m = d["m"]
    dt, nstep = 2e-3, 25
    sim = orc.OracleSim(r0, v0, np.zeros(0), m, np.zeros(0, np.float32), n_gas=0)
    sim.initial_rhs()
    for _ in range(nstep):
        sim.step(dt)

    r, v = r0.copy(), v0.copy()
    g = orc.gravity(_pos_m(r, m))[0].T
    for _ in range(nstep):
        r = r + dt * v + 0.5 * dt * dt * g
        g_new = orc.gravity(_pos_m(r, m))[0].T
        v = v + 0.5 * dt * (g + g_new)
        g = g_new
    assert np.max(np.abs(sim.r - r)) < 1e-12
    assert np.max(np.abs(sim.v - v)) < 1e-11


def test_gas_run_energy_is_nearly_conserved(orc):
    # with gas, total energy is not exactly conserved (density and force
    # kernels differ, h is adaptive), but it must stay close over a short run
    d = ics.single_halo(1024, 1024, seed=3)
    sim = orc.OracleSim(d["r"].T, d["v"].T, d["e"], d["m"], d["h"], d["n_gas"])
    sim.initial_rhs()
    e0 = sum(sim.energies())
    for _ in range(10):
        sim.step(1e-3)
    e1 = sum(sim.energies())
    # measured drift ~2e-9; a sign slip in de/dt would give ~1e-5
    assert abs(e1 - e0) < 2e-7 * abs(e0)
    assert np.all(np.isfinite(sim.r)) and np.all(np.isfinite(sim.e))


def test_predict_and_correct_formulas(orc):
    # one particle, fixed accelerations: predictor and corrector of Eqs. 12-16
    r = np.array([[1.0], [2.0], [3.0]])
    v = np.array([[0.5], [-0.5], [0.25]])
    e = np.array([2.0])
    vs = np.zeros_like(v)
    es = np.zeros_like(e)
    a = np.array([[0.1, 0.2, 0.3]])
    g = np.array([[-1.0, 0.0, 1.0]])
    de = np.array([0.7])
    dt = 0.1
    orc.predict(1, dt, r, v, e, vs, es, a, de, g)
    q = (a + g)[0]
    vt = np.array([0.5, -0.5, 0.25]) + dt * q
    assert np.allclose(v[:, 0], vt, rtol=0, atol=1e-15)
    assert np.allclose(r[:, 0], np.array([1.0, 2.0, 3.0]) + dt / 2 * (vt + [0.5, -0.5, 0.25]),
                       rtol=0, atol=1e-15)
    assert abs(e[0] - (2.0 + dt * 0.7)) < 1e-15
    a2 = np.array([[0.0, -0.2, 0.1]])
    de2 = np.array([-0.3])
    orc.correct(1, dt, v, e, vs, es, a2, de2, g)
    q2 = (a2 + g)[0]
    assert np.allclose(v[:, 0], 0.5 * (np.array([0.5, -0.5, 0.25]) + vt) + dt / 2 * q2,
                       rtol=0, atol=1e-15)
    assert abs(e[0] - (0.5 * (2.0 + 2.0 + dt * 0.7) + dt / 2 * -0.3)) < 1e-15
