"""One simulation resident in device memory, advanced by the library's
whole-step call (predictor-corrector of Sect. 2.2 of the paper).

Device memory is allocated with torch; every step runs in the CUDA kernels
behind sph_rhs_initial / sph_step.  The host side only sizes the context's
neighbour-list capacity (grown between steps when a step used > 70% of it).
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as nv


def assemble_batch(ic_list):
    """Lay several initial conditions out as one batched state: all gas
    (simulation by simulation), then all dark.  Returns (ic, gas_off,
    dark_off, sim_of_gas)."""
    gas_off = [0]
    dark_off = [0]
    rg, vg, rd, vd, e, h, mg, md, sim = [], [], [], [], [], [], [], [], []
    for s, d in enumerate(ic_list):
        ng = int(d["n_gas"])
        rg.append(d["r"][:ng]); vg.append(d["v"][:ng])
        rd.append(d["r"][ng:]); vd.append(d["v"][ng:])
        e.append(d["e"]); h.append(d["h"])
        mg.append(d["m"][:ng]); md.append(d["m"][ng:])
        sim.append(np.full(ng, s, np.int32))
        gas_off.append(gas_off[-1] + ng)
        dark_off.append(dark_off[-1] + int(d["n"]) - ng)
    r = np.concatenate(rg + rd)
    out = dict(r=r, v=np.concatenate(vg + vd), e=np.concatenate(e), h=np.concatenate(h),
               m=np.concatenate(mg + md), n_gas=gas_off[-1], n=r.shape[0])
    return out, np.array(gas_off, np.int32), np.array(dark_off, np.int32), np.concatenate(sim)


class Simulation:
    """One simulation, or a batch of independent ones (batch_offsets =
    (gas_off, dark_off, sim_of_gas) from assemble_batch), resident in device
    memory and advanced by sph_step."""

    def __init__(self, ic: dict, device=None, grav_flags=0, nb_per_particle=120,
                 batch_offsets=None, pairs=True, **params):
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.params = dict(nv.DEFAULT_PARAMS)
        self.params.update(params)
        self.n = int(ic["n"])
        self.n_gas = int(ic["n_gas"])
        n, ng, dev = self.n, self.n_gas, self.device
        f32 = dict(dtype=torch.float32, device=dev)
        f64 = dict(dtype=torch.float64, device=dev)
        t = {}
        t["r"] = torch.as_tensor(np.ascontiguousarray(np.asarray(ic["r"], np.float64).T).ravel(), **f64)
        t["v"] = torch.as_tensor(np.ascontiguousarray(np.asarray(ic["v"], np.float64).T).ravel(), **f64)
        t["e"] = torch.as_tensor(np.asarray(ic["e"], np.float64), **f64)
        t["v_save"] = torch.zeros(3 * n, **f64)
        t["e_save"] = torch.zeros(ng, **f64)
        t["mass"] = torch.as_tensor(np.asarray(ic["m"], np.float32), **f32)
        t["h"] = torch.as_tensor(np.asarray(ic["h"], np.float32), **f32)
        t["pos_m"] = torch.zeros((n, 4), **f32)
        t["pos_h"] = torch.zeros((ng, 4), **f32)
        t["vel_e"] = torch.zeros((ng, 4), **f32)
        t["rho"] = torch.zeros(ng, **f32)
        t["acc_hyd"] = torch.zeros((ng, 4), **f32)
        t["grav"] = torch.zeros((n, 4), **f32)
        self.grav_flags = int(grav_flags)
        # scratch of the pair-once gravity kernel (one simulation or a batch)
        if pairs and nv.pp_gravity_pairs_eligible(n, self.params["eps"], self.grav_flags):
            t["grav_work"] = nv.pp_gravity_pairs_workspace(n, device=dev)
        self.t = t
        self.state = nv.state_struct(t, n, ng, 0, self.grav_flags)
        self.ctx = None
        self.lanes = None
        self.grid_shift = 0
        self.nb_per_particle = nb_per_particle
        self.batch = None
        if batch_offsets is not None:
            gas_off, dark_off, sim_of_gas = batch_offsets
            self.sim_of_gas = torch.as_tensor(np.asarray(sim_of_gas, np.int32), device=dev)
            self.batch = nv.Batch(gas_off, dark_off, self.sim_of_gas)
            self.gas_off, self.dark_off = np.asarray(gas_off), np.asarray(dark_off)
        # the context also carries G and eps for collisionless runs
        self._make_ctx(max(1024, ng * nb_per_particle))
        self.graph = None
        self.diag_out = torch.zeros(8, **f64)

    # -- neighbour-list capacity -------------------------------------------
    def _make_ctx(self, capacity):
        old = self.ctx
        self.ctx = nv.Ctx(max(1, self.n_gas), capacity, device=self.device, **self.params)
        if self.lanes:
            self.ctx.set_lanes(self.lanes)
        if self.grid_shift:
            self.ctx.set_grid_shift(self.grid_shift)
        if self.batch is not None:
            nv.sph_ctx_set_batch(self.ctx, self.batch)
        if old is not None:
            old.close()
        self.graph = None   # a captured step refers to the old context

    def _resort_into_current_ctx(self):
        # the last sort is a pure function of pos_h: redo it in a new context
        nv.sph_bin_and_sort(self.ctx, self.t["pos_h"])
        nv.sph_build_neighbors(self.ctx, self.n_gas)

    def _check_capacity(self):
        if self.n_gas == 0:
            return
        flags = self.ctx.device_status()
        if flags & nv.SPH_FLAG_NB_OVERFLOW:
            raise nv.SphError("sph_step", nv.SPH_ERR_NB_OVERFLOW,
                              "(neighbour lists overflowed inside a step)")
        if flags:
            raise nv.SphError("sph_step", nv.SPH_ERR_DEVICE, f"(device flags {flags})")
        used = self.ctx.nb_total()
        if used > 0.7 * self.ctx.capacity:
            self._make_ctx(int(used * 1.6) + 1024)
            self._resort_into_current_ctx()

    def _size_initial(self):
        # one sort + count at the initial state to size the lists
        nv.integrate_step(nv.SPH_EMIT, 0.0, self.n, self.n_gas, self.t["r"], self.t["v"],
                          self.t["e"], None, None, None, None, self.t["mass"], self.t["h"],
                          self.t["pos_m"], self.t["pos_h"], self.t["vel_e"])
        while True:
            nv.sph_bin_and_sort(self.ctx, self.t["pos_h"])
            try:
                need = nv.sph_build_neighbors(self.ctx, self.n_gas)
            except nv.SphError as ex:
                if ex.code != nv.SPH_ERR_NB_OVERFLOW:
                    raise
                need = self.ctx.nb_total()
                self._make_ctx(int(need * 1.6) + 1024)
                continue
            if need > 0.7 * self.ctx.capacity:
                self._make_ctx(int(need * 1.6) + 1024)
                continue
            return

    # -- stepping -----------------------------------------------------------
    def initial_rhs(self, check=True):
        if self.n_gas > 0:
            self._size_initial()
        nv.sph_rhs_initial(self.ctx, self.state)
        if check:
            self._check_capacity()

    def step(self, dt, check=True):
        nv.sph_step(self.ctx, self.state, dt)
        if check:
            self._check_capacity()

    def step_cfl(self, C=0.5, dt_max=1e-2, check=True):
        """One step whose size min(dt_max, Eq. 17) is chosen on the device in
        the step's first force pass; returns the 1-element device tensor that
        holds it (no host round trip unless read)."""
        if not hasattr(self, "dt_used"):
            self.dt_used = torch.zeros(1, dtype=torch.float32, device=self.device)
        nv.sph_step_cfl(self.ctx, self.state, C, dt_max, self.dt_used)
        if check:
            self._check_capacity()
        return self.dt_used

    # -- CUDA graph of one step --------------------------------------------------
    def capture(self, dt):
        """Capture one step (launch sequence of sph_step) into a CUDA graph.
        Needs a previous step (so the step starts with the HFC at r_n)."""
        if self.state.fresh:
            raise RuntimeError("take one ordinary step before capturing")
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                if dt is None:   # adaptive: (C, dt_max) in self.graph_cfl
                    C, dt_max = self.graph_cfl
                    nv.sph_step_cfl(self.ctx, self.state, C, dt_max, self.dt_used, stream=side)
                else:
                    nv.sph_step(self.ctx, self.state, dt, stream=side)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = g
        self.graph_dt = dt
        return g

    def capture_cfl(self, C=0.5, dt_max=1e-2):
        """Capture one adaptive step (sph_step_cfl); each replay chooses its
        own step size on the device and leaves it in self.dt_used."""
        if not hasattr(self, "dt_used"):
            self.dt_used = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.graph_cfl = (C, dt_max)
        return self.capture(None)

    def replay(self, check=True):
        """One step by replaying the captured graph (re-captured if the
        context had to grow)."""
        if self.graph is None:
            self.capture(self.graph_dt)
        self.graph.replay()
        if check:
            self._check_capacity()

    def sim_slices(self, s):
        """Column indices of simulation s of a batch (gas, then dark)."""
        g0, g1 = int(self.gas_off[s]), int(self.gas_off[s + 1])
        d0, d1 = int(self.dark_off[s]), int(self.dark_off[s + 1])
        return np.concatenate([np.arange(g0, g1), self.n_gas + np.arange(d0, d1)])

    def set_grid_shift(self, shift):
        """Octaves added to the finest cell size of the sort's derived grid."""
        self.grid_shift = int(shift)
        self.ctx.set_grid_shift(self.grid_shift)
        self.graph = None

    def set_lanes(self, lanes):
        """Lanes per neighbour row in the density / force kernels."""
        self.lanes = int(lanes)
        self.ctx.set_lanes(self.lanes)

    def cfl_dt(self, C=0.5):
        """Next time step from the modified CFL condition (Eq. 17) at the
        current state (lists, density and forces of the last evaluation)."""
        if self.n_gas == 0:
            return float("inf")
        if not hasattr(self, "_dt_min"):
            self._dt_min = torch.empty(1, dtype=torch.float32, device=self.device)
        t = self.t
        nv.sph_cfl_dt(self.ctx, t["vel_e"], t["rho"], t["mass"][:self.n_gas], t["acc_hyd"],
                      t["grav"], C, self._dt_min)
        return float(self._dt_min.item())

    # -- host views -----------------------------------------------------------
    def positions(self):
        return self.t["r"].view(3, self.n).T.cpu().numpy()

    def velocities(self):
        return self.t["v"].view(3, self.n).T.cpu().numpy()

    def diagnostics(self):
        nv.sph_diagnostics(self.state, self.diag_out)
        d = self.diag_out.cpu().numpy()
        return dict(kinetic=d[0], thermal=d[1], potential=d[2], momentum=d[3:6], mass=d[6])
