"""Pins of the oracle's direct gravity (Eq. 4, Plummer-softened reading)
against closed forms: Newton's third law, the shell theorem, the softened
self-term, the Plummer sphere's potential energy -3 pi G M^2 / (32 a), and a
two-body circular orbit (run through the oracle's integrator)."""
import math

import numpy as np
import pytest

from paper_1807_08116_gb300 import ics


def _pos_m(r, m):
    pm = np.empty((r.shape[0], 4), np.float32)
    pm[:, :3] = r
    pm[:, 3] = m
    return pm


def test_momentum_conservation(orc):
    rng = np.random.default_rng(5)
    r = rng.normal(size=(700, 3))
    m = rng.uniform(0.5, 2.0, size=700)
    pm = _pos_m(r, m)
    acc, _ = orc.gravity(pm, G=1.0, eps=0.05)
    mf = pm[:, 3].astype(np.float64)
    tot = (mf[:, None] * acc).sum(axis=0)
    scale = (mf[:, None] * np.abs(acc)).sum()
    assert np.all(np.abs(tot) < 1e-13 * scale)


def _fibonacci_shell(n, radius):
    k = np.arange(n) + 0.5
    z = 1 - 2 * k / n
    phi = math.pi * (1 + 5 ** 0.5) * k
    s = np.sqrt(1 - z * z)
    return radius * np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def test_shell_theorem(orc):
    n = 20000
    shell = _fibonacci_shell(n, 1.0)
    probes = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.2], [3.0, 0.0, 0.0], [0.0, -2.0, 2.0]])
    r = np.concatenate([shell, probes])
    m = np.concatenate([np.full(n, 1.0 / n), np.zeros(len(probes))])
    pm = _pos_m(r, m)
    rows = np.arange(n, n + len(probes))
    acc, pot = orc.gravity(pm, G=1.0, eps=1e-4, rows=rows)
    # inside: no net force, constant potential -G M / R
    assert np.linalg.norm(acc[0]) < 1e-6 and np.linalg.norm(acc[1]) < 1e-3
    assert abs(pot[0] + 1.0) < 1e-5 and abs(pot[1] + 1.0) < 1e-3
    # outside: point mass at the centre
    for k, p in ((2, probes[2]), (3, probes[3])):
        d = np.linalg.norm(p)
        expect = -p / d ** 3
        assert np.linalg.norm(acc[k] - expect) < 1e-4 * np.linalg.norm(expect)
        assert abs(pot[k] + 1.0 / d) < 1e-4 / d


def test_softened_self_and_coincident_pair(orc):
    pm = np.array([[0.5, 0.5, 0.5, 2.0], [0.5, 0.5, 0.5, 3.0]], np.float32)
    acc, pot = orc.gravity(pm, G=1.0, eps=0.1)
    assert np.all(acc == 0.0)
    assert abs(pot[0] + 3.0 / 0.1) < 1e-12 and abs(pot[1] + 2.0 / 0.1) < 1e-12


def test_plummer_potential_energy(orc):
    d = ics.single_halo(8192, 8192, seed=0)
    pm = _pos_m(d["r"], d["m"])
    _, pot = orc.gravity(pm, G=1.0, eps=0.01)
    W = 0.5 * float(np.sum(pm[:, 3].astype(np.float64) * pot))
    exact = -3 * math.pi / 32
    # sampling noise of a 16384-particle realisation (~1%), the 0.999 mass
    # truncation and eps = 0.01 softening (both well below 1%) -> 2% band
    assert abs(W - exact) < 0.02 * abs(exact)


def test_two_body_circular_orbit(orc):
    # two equal masses on a circular orbit; relative angular frequency
    # omega^2 = G (m1 + m2) / (d^2 + eps^2)^(3/2) for the softened force
    G, m, d, eps = 1.0, 0.5, 1.0, 0.01
    w = math.sqrt(G * 2 * m / (d * d + eps * eps) ** 1.5)
    vrel = w * d
    r = np.array([[-d / 2, 0, 0], [d / 2, 0, 0]], np.float64)
    v = np.array([[0, -vrel / 2, 0], [0, vrel / 2, 0]], np.float64)
    period = 2 * math.pi / w
    errs = []
    for nstep in (1000, 2000):
        dt = period / nstep
        sim = orc.OracleSim(r.T, v.T, np.zeros(0), np.full(2, m, np.float32),
                            np.zeros(0, np.float32), n_gas=0, G=G, eps=eps)
        sim.initial_rhs()
        for _ in range(nstep):
            sim.step(dt)
        sep = sim.r[:, 1] - sim.r[:, 0]
        # after one period the separation vector returns to (d, 0, 0)
        errs.append(np.linalg.norm(sep - np.array([d, 0, 0])))
    # second-order scheme (Sect. 2.2): halving dt divides the phase error by 4
    assert errs[1] < 3e-5
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_thread_count_does_not_change_results(orc):
    # each target row is summed by one thread in source order, so the
    # single-thread timing row of the bench measures the same arithmetic
    d = ics.single_halo(300, 300, seed=9)
    pm = _pos_m(d["r"], d["m"])
    n0 = orc.threads()
    try:
        orc.set_threads(1)
        assert orc.threads() == 1
        a1, p1 = orc.gravity(pm, G=1.0, eps=0.01)
        orc.set_threads(max(2, n0))
        a2, p2 = orc.gravity(pm, G=1.0, eps=0.01)
    finally:
        orc.set_threads(n0)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
