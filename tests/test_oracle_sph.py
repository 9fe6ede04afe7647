"""Pins of the oracle's SPH pieces: neighbour sets (support of Eqs. 8-9),
density (Eq. 7) and the hydrodynamic right-hand sides (Eqs. 10-11)."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree


def _lattice(n_side, spacing, jitter=0.0, seed=0):
    g = np.arange(n_side) * spacing
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    r = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    if jitter:
        r = r + np.random.default_rng(seed).uniform(-jitter, jitter, size=r.shape)
    return r


def _pos_h(r, h):
    ph = np.empty((r.shape[0], 4), np.float32)
    ph[:, :3] = r
    ph[:, 3] = h
    return ph


# -- neighbour sets -----------------------------------------------------------

def test_neighbors_equal_h_match_kdtree(orc):
    rng = np.random.default_rng(1)
    r = rng.uniform(0, 1, size=(3000, 3)).astype(np.float32)
    h = 0.04
    ph = _pos_h(r, h)
    starts, idx = orc.neighbors(ph)
    tree = cKDTree(r.astype(np.float64))
    ref = tree.query_ball_point(r.astype(np.float64), 2 * h)
    d2h = np.float64(np.float32(2 * h))
    for i in range(r.shape[0]):
        mine = set(idx[starts[i]:starts[i + 1]].tolist())
        theirs = set(ref[i]) - {i}
        diff = mine ^ theirs
        for j in diff:   # only exact-boundary ties may differ between FP32 and FP64
            d = np.linalg.norm(r[i].astype(np.float64) - r[j].astype(np.float64))
            assert abs(d - d2h) < 1e-6
    assert starts[-1] > 4 * r.shape[0]


def test_neighbors_variable_h_symmetric_and_exact(orc):
    rng = np.random.default_rng(2)
    n = 2500
    r = rng.normal(size=(n, 3)).astype(np.float32)
    h = (0.05 * (1 + np.sum(r.astype(np.float64) ** 2, axis=1)) ** 0.8).astype(np.float32)
    ph = _pos_h(r, h)
    starts, idx = orc.neighbors(ph)
    sets = [set(idx[starts[i]:starts[i + 1]].tolist()) for i in range(n)]
    for i in range(n):
        assert i not in sets[i]
        for j in sets[i]:
            assert i in sets[j]
    r64 = r.astype(np.float64)
    d = np.sqrt(((r64[:, None, :] - r64[None, :, :]) ** 2).sum(-1))
    s = h.astype(np.float64)[:, None] + h.astype(np.float64)[None, :]
    inside = d < s * (1 - 1e-6)
    outside = d > s * (1 + 1e-6)
    np.fill_diagonal(inside, False)
    for i in range(n):
        assert set(np.nonzero(inside[i])[0].tolist()) <= sets[i]
        assert not (set(np.nonzero(outside[i])[0].tolist()) & sets[i])


# -- sorting stage -------------------------------------------------------------

def test_counting_sort_matches_numpy(orc):
    rng = np.random.default_rng(3)
    M = 4096
    key = rng.integers(0, M, size=20000).astype(np.int32)
    key[:500] = 17   # a crowded bucket
    count, start, perm = orc.counting_sort(key, M)
    assert np.array_equal(count, np.bincount(key, minlength=M))
    assert np.array_equal(start, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=M))]))
    assert np.array_equal(perm, np.argsort(key, kind="stable"))


def test_binning_levels_cells_and_keys(orc):
    grid = dict(x0=-4.0, y0=-2.0, z0=0.0, log2_L0=-3, n_levels=6, log2_M=30)
    L0 = 2.0 ** -3
    cases = [
        # (x, y, z, h) -> expected (level, cx, cy, cz)
        ((-4.0, -2.0, 0.0, L0), (0, 0, 0, 0)),                        # h == L0: level 0
        ((-4.0, -2.0, 0.0, L0 * 0.3), (0, 0, 0, 0)),
        ((-4.0 + L0, -2.0, 0.0, L0), (0, 1, 0, 0)),                   # on a cell face
        ((np.nextafter(np.float32(-4.0 + L0), np.float32(-9)), -2.0, 0.0, L0), (0, 0, 0, 0)),  # below it
        ((-4.0, -2.0, 0.0, np.nextafter(np.float32(L0), np.float32(1))), (1, 0, 0, 0)),
        ((-4.0 + 3 * L0 * 2, -2.0 + 2 * L0 * 2, 5 * L0 * 2, 2 * L0), (1, 3, 2, 5)),
        ((-4.0, -2.0, 0.0, 8 * L0), (3, 0, 0, 0)),
        ((-4.0, -2.0, 0.0, 1000.0), (5, 0, 0, 0)),                    # clamped to the top
        ((-10.0, -2.0, 0.0, L0), (0, 0, 0, 0)),                       # below the origin
        ((1e9, -2.0, 0.0, L0), (0, 2097151, 0, 0)),                   # far outside
    ]
    ph = np.array([c[0] for c in cases], np.float32)
    level, cell, key = orc.bin_particles(ph, grid)
    for k, (_, (l, cx, cy, cz)) in enumerate(cases):
        assert level[k] == l, k
        assert tuple(cell[k]) == (cx, cy, cz), k
    # key = bit interleave of (cx, cy, cz) + level * golden-ratio constant, mod 2^log2_M
    salt = 0x9E3779B97F4A7C15
    mask = (1 << grid["log2_M"]) - 1
    assert key[0] == 0
    assert key[2] == 1                              # cx = 1 -> bit 0
    # (cx, cy, cz) = (3, 2, 5): bits x0=1 y0=0 z0=1 | x1=1 y1=1 z1=0 | x2=0 y2=0 z2=1
    m = (1 << 0) | (0 << 1) | (1 << 2) | (1 << 3) | (1 << 4) | (0 << 5) | (0 << 6) | (0 << 7) | (1 << 8)
    assert key[5] == (m + 1 * salt) & mask
    assert key[6] == (0 + 3 * salt) & mask
    m_far = 1 << 60 | 1 << 57 | 1 << 54 | 1 << 51 | 1 << 48 | 1 << 45 | 1 << 42 | 1 << 39 | 1 << 36 \
        | 1 << 33 | 1 << 30 | 1 << 27 | 1 << 24 | 1 << 21 | 1 << 18 | 1 << 15 | 1 << 12 | 1 << 9 \
        | 1 << 6 | 1 << 3 | 1
    assert key[9] == m_far & mask


# -- density (Eq. 7) -----------------------------------------------------------

@pytest.mark.parametrize("ratio,tol", [(1.25, 3e-3), (1.5, 3e-3), (2.0, 5e-4)])
def test_lattice_density(orc, ratio, tol):
    # uniform cubic lattice of spacing dx and equal masses m: every interior
    # particle sees the same neighbourhood, and the kernel sum reproduces the
    # continuum density m / dx^3 (normalisation condition of Sect. 2.2)
    dx, m = 0.125, 2.0e-3        # power-of-two spacing: lattice exact in FP32
    r = _lattice(13, dx)
    ph = _pos_h(r, ratio * dx)
    mass = np.full(r.shape[0], m, np.float32)
    centre = np.all(np.abs(r - 6 * dx) < 2.5 * dx, axis=1)
    rows = np.nonzero(centre)[0]
    rho, hn = orc.density(ph, mass, sigma=1.25, rows=rows)
    assert np.ptp(rho) < 1e-10 * rho.mean()
    assert abs(rho.mean() / (np.float32(m) / dx ** 3) - 1) < tol


def test_isolated_particle_density(orc):
    h, m = 0.3, 0.7
    ph = np.array([[0, 0, 0, h], [10, 0, 0, h]], np.float32)
    rho, hn = orc.density(ph, np.array([m, m], np.float32), sigma=1.25)
    m32, h32 = float(np.float32(m)), float(np.float32(h))
    assert abs(rho[0] - m32 / (math.pi * h32 ** 3)) < 1e-12 * rho[0]
    assert abs(hn[0] - 1.25 * math.pi ** (1 / 3) * h32) < 1e-12


# -- hydrodynamic right-hand sides (Eqs. 10-11) ---------------------------------

def _blob(seed, n=600):
    rng = np.random.default_rng(seed)
    r = rng.normal(scale=0.5, size=(n, 3))
    h = (0.12 * (1 + np.sum(r * r, axis=1)) ** 0.5).astype(np.float32)
    v = rng.normal(scale=0.3, size=(n, 3))
    e = rng.uniform(0.05, 0.3, size=n)
    m = rng.uniform(0.5, 1.5, size=n) / n
    return r, h, v, e, m


def _hydro_inputs(orc, r, h, v, e, m):
    ph = _pos_h(r, h)
    ve = np.empty((r.shape[0], 4), np.float32)
    ve[:, :3] = v
    ve[:, 3] = e
    mass = m.astype(np.float32)
    rho, _ = orc.density(ph, mass)
    return ph, ve, mass, rho.astype(np.float32)


def test_hydro_conserves_momentum_and_energy(orc):
    r, h, v, e, m = _blob(7)
    ph, ve, mass, rho = _hydro_inputs(orc, r, h, v, e, m)
    acc, de = orc.hydro(ph, ve, mass, rho)
    mf = mass.astype(np.float64)
    vf = ve[:, :3].astype(np.float64)
    # momentum: pairwise antisymmetry of m_i m_j Pi_ij grad W_p ("Newton's third law")
    p = (mf[:, None] * acc).sum(0)
    assert np.all(np.abs(p) < 1e-12 * (mf[:, None] * np.abs(acc)).sum())
    # total energy sum m (v.a + de/dt) vanishes pairwise
    dE = float((mf * ((vf * acc).sum(1) + de)).sum())
    scale = float((mf * (np.abs(vf * acc).sum(1) + np.abs(de))).sum())
    assert abs(dE) < 1e-12 * scale
    assert np.abs(acc).max() > 0


def test_hydro_pair_at_rest_matches_numerical_gradient(orc):
    # two particles at rest feel only the pressure term: a_1 = -m_2 Pi grad_1 W_p
    gam = 5.0 / 3.0
    h = np.float32(0.5)
    ph = np.array([[0.1, 0.2, 0.3, h], [0.35, 0.05, 0.4, h]], np.float32)
    ve = np.array([[0, 0, 0, 0.2], [0, 0, 0, 0.1]], np.float32)
    mass = np.array([0.3, 0.6], np.float32)
    rho = np.array([1.5, 2.5], np.float32)
    acc, de = orc.hydro(ph, ve, mass, rho, gamma=gam)
    P = sum((gam - 1) * float(rho[k]) * float(ve[k, 3]) / float(rho[k]) ** 2 for k in (0, 1))
    x1 = ph[0, :3].astype(np.float64)
    x2 = ph[1, :3].astype(np.float64)
    d = 1e-6
    grad = np.zeros(3)
    for ax in range(3):
        e_ = np.zeros(3)
        e_[ax] = d
        grad[ax] = (orc.Wp(np.linalg.norm(x1 + e_ - x2) / h, h)
                    - orc.Wp(np.linalg.norm(x1 - e_ - x2) / h, h)) / (2 * d)
    expect = -float(mass[1]) * P * grad
    assert np.allclose(acc[0], expect, rtol=1e-7, atol=0)
    assert np.allclose(acc[1] * float(mass[1]), -acc[0] * float(mass[0]), rtol=1e-12)
    assert np.all(de == 0.0)


def test_viscosity_only_for_approaching_pairs(orc):
    h = np.float32(0.5)
    ph = np.array([[0.0, 0, 0, h], [0.4, 0, 0, h]], np.float32)
    mass = np.array([1.0, 1.0], np.float32)
    rho = np.array([2.0, 2.0], np.float32)
    recede = np.array([[-1.0, 0, 0, 0.1], [1.0, 0, 0, 0.1]], np.float32)
    approach = np.array([[1.0, 0, 0, 0.1], [-1.0, 0, 0, 0.1]], np.float32)
    a_r, de_r = orc.hydro(ph, recede, mass, rho)
    a_r0, de_r0 = orc.hydro(ph, recede, mass, rho, alpha=0.0, beta=0.0)
    assert np.array_equal(a_r, a_r0) and np.array_equal(de_r, de_r0)
    a_a, de_a = orc.hydro(ph, approach, mass, rho)
    a_a0, de_a0 = orc.hydro(ph, approach, mass, rho, alpha=0.0, beta=0.0)
    # viscosity adds repulsion (particle 0 pushed to -x harder) and heats both
    assert a_a[0, 0] < a_a0[0, 0] < 0
    assert np.all(de_a > de_a0)
    # pressure-only compression heats, expansion cools (Eq. 3 sign)
    assert np.all(de_a0 > 0) and np.all(de_r0 < 0)


def test_hydro_galilean_invariance(orc):
    r, h, v, e, m = _blob(11, n=300)
    ph, ve, mass, rho = _hydro_inputs(orc, r, h, v, e, m)
    a0, d0 = orc.hydro(ph, ve, mass, rho)
    ve2 = ve.copy()
    ve2[:, :3] += np.float32(0.5)
    a1, d1 = orc.hydro(ph, ve2, mass, rho)
    assert np.allclose(a0, a1, rtol=1e-5, atol=1e-6 * np.abs(a0).max())
    assert np.allclose(d0, d1, rtol=1e-5, atol=1e-6 * np.abs(d0).max())
