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


class Simulation:
    def __init__(self, ic: dict, device=None, grav_flags=0, nb_per_particle=120, **params):
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
        self.t = t
        self.grav_flags = int(grav_flags)
        self.state = nv.state_struct(t, n, ng, 0, self.grav_flags)
        self.ctx = None
        self.nb_per_particle = nb_per_particle
        # the context also carries G and eps for collisionless runs
        self._make_ctx(max(1024, ng * nb_per_particle))
        self.diag_out = torch.zeros(8, **f64)

    # -- neighbour-list capacity -------------------------------------------
    def _make_ctx(self, capacity):
        old = self.ctx
        self.ctx = nv.Ctx(max(1, self.n_gas), capacity, device=self.device, **self.params)
        if old is not None:
            old.close()

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

    # -- host views -----------------------------------------------------------
    def positions(self):
        return self.t["r"].view(3, self.n).T.cpu().numpy()

    def velocities(self):
        return self.t["v"].view(3, self.n).T.cpu().numpy()

    def diagnostics(self):
        nv.sph_diagnostics(self.state, self.diag_out)
        d = self.diag_out.cpu().numpy()
        return dict(kinetic=d[0], thermal=d[1], potential=d[2], momentum=d[3:6], mass=d[6])
