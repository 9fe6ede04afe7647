"""Pins of the oracle's time-step condition (Eq. 17) against closed forms."""
import math

import numpy as np


def _lattice(n_side, dx):
    g = np.arange(n_side) * dx
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def _inputs(r, h, v, e, rho):
    ph = np.empty((len(r), 4), np.float32)
    ph[:, :3] = r
    ph[:, 3] = h
    ve = np.empty((len(r), 4), np.float32)
    ve[:, :3] = v
    ve[:, 3] = e
    return ph, ve, np.full(len(r), rho, np.float32)


def test_static_lattice_closed_form(orc):
    # gas at rest on a lattice of spacing dx, uniform e: s_min = dx,
    # c_max = c = sqrt(gamma (gamma-1) e), no approach (mu = 0), no force:
    # dt = C dx / (c (1 + 1.2 alpha))
    dx, e, gam, alpha, C = 0.125, 0.3, 5.0 / 3.0, 0.5, 0.6
    r = _lattice(7, dx)
    n = len(r)
    ph, ve, rho = _inputs(r, 1.25 * dx, np.zeros((n, 3)), np.full(n, e), 2.0)
    dt, rows = orc.cfl_dt(ph, ve, rho, np.zeros((n, 3)), np.zeros(n), C=C, gamma=gam, alpha=alpha)
    c = math.sqrt(gam * (gam - 1) * float(np.float32(e)))
    expect = C * dx / (c * (1 + 1.2 * alpha))
    assert abs(dt - expect) < 1e-12 * expect
    assert np.allclose(rows, expect, rtol=1e-12)


def test_force_and_heating_terms(orc):
    # one neighbour pair at rest with e = 0 (c = 0): dt = C s / sqrt(s (|Q| + |E|))
    ph = np.array([[0, 0, 0, 0.5], [0.375, 0.5, 0, 0.5]], np.float32)   # |dr| = 0.625 exactly
    ve = np.zeros((2, 4), np.float32)
    rho = np.ones(2, np.float32)
    Q = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 0.0]])
    E = np.array([1.0, 0.0])
    dt, rows = orc.cfl_dt(ph, ve, rho, Q, E, C=0.7)
    s = 0.625
    assert abs(rows[0] - 0.7 * s / math.sqrt(s * 6.0)) < 1e-12
    assert math.isinf(rows[1])         # no force, no sound speed: unbounded
    assert dt == rows[0]


def test_approach_tightens_the_step(orc):
    # approaching pair: mu = h dr.dv / (r^2 + eta h^2) < 0 adds 1.2 beta |mu|
    h = 0.5
    ph = np.array([[0, 0, 0, h], [0.375, 0, 0, h]], np.float32)
    rho = np.ones(2, np.float32)
    recede = np.array([[-1, 0, 0, 0], [1, 0, 0, 0]], np.float32)
    approach = np.array([[1, 0, 0, 0], [-1, 0, 0, 0]], np.float32)
    z3, z1 = np.zeros((2, 3)), np.zeros(2)
    d_r, _ = orc.cfl_dt(ph, recede, rho, z3, z1, C=1.0)
    d_a, rows = orc.cfl_dt(ph, approach, rho, z3, z1, C=1.0, beta=1.0)
    assert math.isinf(d_r)             # no sound speed, receding: no bound
    mu = h * (0.375 * -2.0) / (0.375 ** 2 + 0.1 * h * h)
    assert abs(rows[0] - 0.375 / (1.2 * abs(mu))) < 1e-12
