"""Density (Eq. 7) and hydrodynamic forces (Eqs. 10-11) through the C ABI
against the FP64 oracle on the same FP32 inputs."""
import numpy as np
import pytest

from helpers import MAX_TOL, RMS_TOL, err, need_gpu, pos_h_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu

# density is a sum of positive terms in FP32 with compensation; every term
# carries a few roundings (1/h^3, the spline polynomial, sqrt) -> ~2e-7 each
RHO_RMS, RHO_MAX = 1e-6, 1e-5


def _setup(ph, cap_per=200):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    n = len(ph)
    ctx = nv.Ctx(n, max(1024, cap_per * n))
    x = torch.as_tensor(ph, device="cuda")
    nv.sph_bin_and_sort(ctx, x)
    nv.sph_build_neighbors(ctx, n)
    return torch, nv, ctx


def _density(ph, mass, lanes=4):
    torch, nv, ctx = _setup(ph)
    ctx.set_lanes(lanes)
    n = len(ph)
    m = torch.as_tensor(mass, device="cuda")
    rho = torch.empty(n, device="cuda")
    hn = torch.empty(n, device="cuda")
    nv.sph_density(ctx, m, rho, hn)
    torch.cuda.synchronize()
    return ctx, rho.cpu().numpy(), hn.cpu().numpy()


def _forces(ph, ve, mass, rho, lanes=4, **params):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    n = len(ph)
    ctx = nv.Ctx(n, max(1024, 200 * n), **params)
    ctx.set_lanes(lanes)
    nv.sph_bin_and_sort(ctx, torch.as_tensor(ph, device="cuda"))
    nv.sph_build_neighbors(ctx, n)
    out = torch.full((n, 4), float("nan"), device="cuda")
    nv.sph_forces(ctx, torch.as_tensor(ve, device="cuda"), torch.as_tensor(rho, device="cuda"),
                  torch.as_tensor(mass, device="cuda"), out)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    return out.cpu().numpy().astype(np.float64)


def _gas(d):
    ng = d["n_gas"]
    ph = pos_h_of(d["r"][:ng], d["h"])
    mass = d["m"][:ng].astype(np.float32)
    ve = np.empty((ng, 4), np.float32)
    ve[:, :3] = d["v"][:ng]
    ve[:, 3] = d["e"]
    return ph, mass, ve


def _stirred(d, seed=0):
    """Gas with a random velocity field (so viscosity and heating act) and a
    spread of internal energies."""
    ph, mass, ve = _gas(d)
    rng = np.random.default_rng(seed)
    ve[:, :3] = rng.normal(scale=0.3, size=(len(ve), 3))
    ve[:, 3] *= rng.uniform(0.5, 1.5, len(ve))
    return ph, mass, ve


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_density_single_halo(orc, lanes):
    d = ics.single_halo(8192, 8192, seed=0)
    ph, mass, _ = _gas(d)
    _, rho, hn = _density(ph, mass, lanes)
    orho, ohn = orc.density(ph, mass)
    r1, m1 = err(rho, orho)
    r2, m2 = err(hn, ohn)
    print(f"density rms {r1:.2e} max {m1:.2e}; h_next rms {r2:.2e} max {m2:.2e}")
    assert r1 <= RHO_RMS and m1 <= RHO_MAX
    assert r2 <= RHO_RMS and m2 <= RHO_MAX


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_forces_single_halo(orc, lanes):
    d = ics.single_halo(8192, 8192, seed=0)
    ph, mass, ve = _stirred(d)
    orho, _ = orc.density(ph, mass)
    rho = orho.astype(np.float32)
    a = _forces(ph, ve, mass, rho, lanes)
    oa, ode = orc.hydro(ph, ve, mass, rho)
    ra, ma = err(a[:, :3], oa)
    re, me = err(a[:, 3:], ode[:, None])
    print(f"hydro accel rms {ra:.2e} max {ma:.2e}; de/dt rms {re:.2e} max {me:.2e}")
    assert ra <= RMS_TOL and ma <= MAX_TOL
    assert re <= RMS_TOL and me <= MAX_TOL
    # pairwise antisymmetry: total hydro momentum change vanishes to FP32 rounding
    m = mass.astype(np.float64)
    assert np.abs((m[:, None] * a[:, :3]).sum(0)).max() < 1e-5 * (m[:, None] * np.abs(a[:, :3])).sum()


def test_equal_mass_density_loop_matches_the_general_one(orc):
    # with all gas masses equal, the density pass takes m_j from the row's own
    # particle and reads no mass array; one particle's mass one ulp off sends
    # it through the general loop.  Rows that do not have that particle as a
    # neighbour must come out bitwise the same either way (density, h_next and
    # the forces computed from the same densities), and both runs match the
    # oracle.
    d = ics.single_halo(8192, 8192, seed=0)
    ph, mass, ve = _stirred(d)
    assert np.all(mass == mass[0])
    k = int(np.argmin(ph[:, 3]))   # the smallest h: the fewest rows reach it
    off = mass.copy()
    off[k] = np.nextafter(off[k], np.float32(1.0))
    dist = np.linalg.norm(ph[:, :3].astype(np.float64) - ph[k, :3], axis=1)
    clear = dist >= 1.01 * (ph[:, 3].astype(np.float64) + ph[k, 3])
    assert clear.sum() > 8000
    res = {}
    rin = orc.density(ph, mass)[0].astype(np.float32)   # the same densities for both force passes
    for name, m in (("equal", mass), ("mixed", off)):
        _, rho, hn = _density(ph, m)
        orho, _ = orc.density(ph, m)
        r1, m1 = err(rho, orho)
        assert r1 <= RHO_RMS and m1 <= RHO_MAX, (name, r1, m1)
        a = _forces(ph, ve, m, rin)
        oa, ode = orc.hydro(ph, ve, m, rin)
        ra, ma = err(a[:, :3], oa)
        assert ra <= RMS_TOL and ma <= MAX_TOL, (name, ra, ma)
        res[name] = (rho, hn, a)
    for x, y in zip(res["equal"], res["mixed"]):
        assert np.array_equal(x[clear], y[clear])


def test_forces_at_rest_and_without_viscosity(orc):
    d = ics.single_halo(4096, 0, seed=2)
    ph, mass, ve = _gas(d)      # gas at rest: pressure only
    orho, _ = orc.density(ph, mass)
    rho = orho.astype(np.float32)
    a = _forces(ph, ve, mass, rho, alpha=0.0, beta=0.0)
    oa, ode = orc.hydro(ph, ve, mass, rho, alpha=0.0, beta=0.0)
    ra, ma = err(a[:, :3], oa)
    assert ra <= RMS_TOL and ma <= MAX_TOL
    assert np.all(a[:, 3] == 0.0)


@pytest.mark.parametrize("lanes", [1, 4])
def test_forces_head_on_pair_matches_hand_calculation(lanes):
    # the two-particle head-on case worked by hand from the definitions of
    # Pi_ij, nu_ij and mu_ij (Sect. 2.2), in FP32 on the device
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "viscosity_head_on.json")) as f:
        g = json.load(f)
    ph = np.array(g["pos_h"], np.float32)
    ve = np.array(g["vel_e"], np.float32)
    mass = np.array(g["mass"], np.float32)
    rho = np.array(g["rho"], np.float32)
    a = _forces(ph, ve, mass, rho, lanes, gamma=g["gamma"], alpha=g["alpha"], beta=g["beta"],
                eta=g["eta"])
    acc, de = np.array(g["acc"]), np.array(g["dedt"])
    assert np.abs(a[:, :3] - acc).max() < 2e-6 * np.abs(acc).max()
    assert np.abs(a[:, 3] - de).max() < 2e-6 * np.abs(de).max()


def test_two_halo_sampled_rows(orc):
    d = ics.two_halo(131072, 131072, seed=1)
    ph, mass, ve = _stirred(d, seed=1)
    n = len(ph)
    rows = np.random.default_rng(5).choice(n, 300, replace=False)
    # density on sampled rows
    _, rho, hn = _density(ph, mass)
    orho, ohn = orc.density(ph, mass, rows=rows)
    r1, m1 = err(rho[rows], orho)
    assert r1 <= RHO_RMS and m1 <= RHO_MAX
    # forces: the common density input comes from the oracle, evaluated on the
    # sampled rows and all their neighbours (the only densities they read)
    ostart, oidx = orc.neighbors(ph, rows=rows)
    need = np.unique(np.concatenate([rows, oidx]))
    rho_need, _ = orc.density(ph, mass, rows=need)
    rho_in = np.ones(n, np.float32)
    rho_in[need] = rho_need.astype(np.float32)
    a = _forces(ph, ve, mass, rho_in)
    oa, ode = orc.hydro(ph, ve, mass, rho_in, rows=rows)
    ra, ma = err(a[rows, :3], oa)
    re, me = err(a[rows, 3:], ode[:, None])
    print(f"two-halo hydro sample: accel rms {ra:.2e} max {ma:.2e}; de/dt rms {re:.2e} max {me:.2e}")
    assert ra <= RMS_TOL and ma <= MAX_TOL
    assert re <= RMS_TOL and me <= MAX_TOL


def test_large_collision_sampled_rows(orc):
    # the 2 x (1048576 + 1048576) collision, in the launch configuration of
    # its steps (2 lanes per row, the tuned choice at this size): density on
    # sampled rows against brute force; forces on sampled rows from a common
    # density input (the GPU densities, which both sides then read)
    d = ics.two_halo(1048576, 1048576, seed=2)
    ph, mass, ve = _stirred(d, seed=3)
    n = len(ph)
    rows = np.random.default_rng(7).choice(n, 48, replace=False)
    _, rho, _ = _density(ph, mass, lanes=2)
    orho, _ = orc.density(ph, mass, rows=rows)
    r1, m1 = err(rho[rows], orho)
    a = _forces(ph, ve, mass, rho, lanes=2)
    oa, ode = orc.hydro(ph, ve, mass, rho, rows=rows)
    ra, ma = err(a[rows, :3], oa)
    re, me = err(a[rows, 3:], ode[:, None])
    print(f"large-collision sample: rho rms {r1:.2e} max {m1:.2e}; accel rms {ra:.2e} "
          f"max {ma:.2e}; de/dt rms {re:.2e} max {me:.2e}")
    assert r1 <= RHO_RMS and m1 <= RHO_MAX
    assert ra <= RMS_TOL and ma <= MAX_TOL
    assert re <= RMS_TOL and me <= MAX_TOL


def test_isolated_and_empty():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    ph = np.array([[0, 0, 0, 0.3], [10, 0, 0, 0.3]], np.float32)
    _, rho, hn = _density(ph, np.array([0.7, 0.7], np.float32))
    m, h = float(np.float32(0.7)), float(np.float32(0.3))
    assert abs(rho[0] - m / (np.pi * h ** 3)) < 1e-6 * rho[0]
    ctx = nv.Ctx(4, 1024)
    z = torch.zeros((0, 4), device="cuda")
    nv.sph_bin_and_sort(ctx, z)
    nv.sph_build_neighbors(ctx, 0)
    e = torch.zeros(0, device="cuda")
    nv.sph_density(ctx, e, e.clone(), e.clone())
    nv.sph_forces(ctx, z, e, e.clone(), z.clone())
    torch.cuda.synchronize()


def test_cfl_time_step(orc):
    # Eq. 17 per particle and its minimum, on stirred gas with forces
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    d = ics.single_halo(6000, 0, seed=51)
    ph, mass, ve = _stirred(d, seed=3)
    n = len(ph)
    orho, _ = orc.density(ph, mass)
    rho = orho.astype(np.float32)
    rng = np.random.default_rng(4)
    acc = rng.normal(size=(n, 4)).astype(np.float32)
    grav = rng.normal(size=(n, 4)).astype(np.float32)
    ctx = nv.Ctx(n, 200 * n)
    nv.sph_bin_and_sort(ctx, torch.as_tensor(ph, device="cuda"))
    nv.sph_build_neighbors(ctx, n)
    dt_min = torch.empty(1, device="cuda")
    dt_p = torch.empty(n, device="cuda")
    cu = lambda a: torch.as_tensor(a, device="cuda")
    nv.sph_cfl_dt(ctx, cu(ve), cu(rho), cu(mass), cu(acc), cu(grav), 0.6, dt_min, dt_p)
    torch.cuda.synchronize()
    Q = acc[:, :3].astype(np.float64) + grav[:, :3].astype(np.float64)
    E = acc[:, 3].astype(np.float64)
    odt, orow = orc.cfl_dt(ph, ve, rho, Q, E, C=0.6)
    got = dt_p.cpu().numpy().astype(np.float64)
    fin = np.isfinite(orow)
    assert np.array_equal(np.isfinite(got), fin)
    rel = np.abs(got[fin] - orow[fin]) / orow[fin]
    print(f"cfl dt: max rel {rel.max():.2e}; min {odt:.4e}")
    assert rel.max() < 1e-5
    assert abs(float(dt_min.item()) - odt) < 1e-5 * odt
