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


def test_batched_sph_stages_match_the_oracle_per_simulation(orc):
    # Four gas-carrying simulations laid on top of one another (every halo is
    # centred on the origin, so their particles interleave in space and in the
    # shared hashed grid): the batch's sort, neighbour search, density and
    # forces, run as one launch per stage, against the oracle on each
    # simulation alone -- neighbour sets exact (no pair crosses simulations),
    # density and the hydro right-hand side within the stated tolerances.
    torch = need_gpu()
    from helpers import RMS_TOL, MAX_TOL, max_plain, pos_h_of
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.sim import assemble_batch
    lst = [ics.two_halo(1500, 500, seed=61), ics.single_halo(2500, 700, seed=62),
           ics.single_halo(900, 0, seed=63), ics.two_halo(350, 350, seed=64)]
    rng = np.random.default_rng(65)
    for d in lst:   # stir the gas so viscosity and heating act
        d["v"] = d["v"].copy()
        d["v"][:d["n_gas"]] = rng.normal(scale=0.3, size=(d["n_gas"], 3))
    ic, go, do, so = assemble_batch(lst)
    ng = int(ic["n_gas"])
    ph = pos_h_of(ic["r"][:ng], ic["h"])
    mass = ic["m"][:ng].astype(np.float32)
    ve = np.empty((ng, 4), np.float32)
    ve[:, :3] = ic["v"][:ng]
    ve[:, 3] = ic["e"]
    cu = lambda a: torch.as_tensor(a, device="cuda")
    batch = nv.Batch(go, do, cu(so))
    ctx = nv.Ctx(ng, 250 * ng)
    nv.sph_ctx_set_batch(ctx, batch)
    perm = torch.empty(ng, dtype=torch.int32, device="cuda")
    nv.sph_bin_and_sort(ctx, cu(ph), perm=perm)
    start = torch.empty(ng + 1, dtype=torch.int32, device="cuda")
    need = nv.sph_build_neighbors(ctx, ng, nb_start=start)
    idx = torch.empty(max(need, 1), dtype=torch.int32, device="cuda")
    nv.sph_build_neighbors(ctx, ng, nb_start=start, nb_idx=idx)
    rho = torch.empty(ng, device="cuda")
    hn = torch.empty(ng, device="cuda")
    nv.sph_density(ctx, cu(mass), rho, hn)
    torch.cuda.synchronize()
    rho_g = rho.cpu().numpy()
    # forces from a common density input: the oracle's, per simulation
    rho_in = np.empty(ng, np.float32)
    for s in range(len(lst)):
        a, b = go[s], go[s + 1]
        if b > a:
            rho_in[a:b], _ = orc.density(ph[a:b], mass[a:b])
    acc = torch.full((ng, 4), float("nan"), device="cuda")
    nv.sph_forces(ctx, cu(ve), cu(rho_in), cu(mass), acc)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    acc_g = acc.cpu().numpy().astype(np.float64)
    perm = perm.cpu().numpy()
    start = start.cpu().numpy()
    idx = idx.cpu().numpy()[:need]
    inv = np.empty_like(perm)
    inv[perm] = np.arange(ng, dtype=perm.dtype)
    for s in range(len(lst)):
        a, b = int(go[s]), int(go[s + 1])
        if b == a:
            continue
        # neighbour sets of every row of this simulation, against brute force
        # over this simulation's gas alone
        ost, oidx = orc.neighbors(ph[a:b])
        for i in range(a, b):
            k = inv[i]
            got = np.sort(perm[idx[start[k]:start[k + 1]]])
            ref = np.sort(oidx[ost[i - a]:ost[i - a + 1]] + a)
            assert np.array_equal(got, ref), (s, i)
        orho, _ = orc.density(ph[a:b], mass[a:b])
        r1, m1 = err(rho_g[a:b], orho)
        assert r1 <= 1e-6 and m1 <= 1e-5, (s, r1, m1)
        oa, ode = orc.hydro(ph[a:b], ve[a:b], mass[a:b], rho_in[a:b])
        ra, ma = err(acc_g[a:b, :3], oa)
        re_, me = err(acc_g[a:b, 3:], ode[:, None])
        print(f"batch sim {s} ({b - a} gas): rho rms {r1:.1e}; accel rms {ra:.1e} max {ma:.1e} "
              f"(plain {max_plain(acc_g[a:b, :3], oa):.1e}); de/dt rms {re_:.1e} max {me:.1e}")
        assert ra <= RMS_TOL and ma <= MAX_TOL, (s, ra, ma)
        assert re_ <= RMS_TOL and me <= MAX_TOL, (s, re_, me)
