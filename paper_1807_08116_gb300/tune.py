"""Autotuning of the gravity launch plan by timing candidates on the device.

The single-simulation kernel has two knobs (R targets per thread, S CTAs
per cluster sharing the source range); the batched kernel has R.  A built-in
cost model picks a plan without timing; these functions time the candidates
on the caller's own inputs instead and fix the fastest (sph_gravity_tune /
sph_batch_set_plan), returning the measurements.
"""
from __future__ import annotations

import torch

from . import native as nv

SINGLE_CANDIDATES = [(2, 1), (4, 1), (8, 1), (2, 2), (4, 2), (2, 4), (4, 4), (2, 8), (4, 8),
                     (2, 16)]


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_gravity(pos_m, G=1.0, eps=0.01, flags=0, candidates=None, reps=2, apply=True):
    """Time pp_gravity on pos_m for each (R, S); fix the fastest if apply."""
    out = torch.empty_like(pos_m)
    n = pos_m.shape[0]
    tiles = (n + 1023) // 1024
    res = {}
    for R, S in candidates or SINGLE_CANDIDATES:
        if S > max(1, tiles):
            continue
        nv.sph_gravity_tune(R, S)
        res[(R, S)] = _time(lambda: nv.pp_gravity(pos_m, out, G, eps, flags), reps)
    best = min(res, key=res.get)
    nv.sph_gravity_tune(*best) if apply else nv.sph_gravity_tune(0)
    return best, res


def tune_batch(batch, pos_m, G=1.0, eps=0.01, flags=0, reps=2):
    """Time pp_gravity_batched for R in {2, 4, 8}; keep the fastest."""
    out = torch.empty_like(pos_m)
    res = {}
    for R in (2, 4, 8):
        batch.set_plan(R)
        res[R] = _time(lambda: nv.pp_gravity_batched(batch, pos_m, out, G, eps, flags), reps)
    best = min(res, key=res.get)
    batch.set_plan(best)
    return best, res


def tune_lanes(sim, reps=3):
    """Time the force kernel of a Simulation (after its first evaluation) for
    1, 2, 4 and 8 lanes per neighbour row; keep the fastest."""
    t = sim.t
    res = {}
    for lanes in (1, 2, 4, 8):
        sim.set_lanes(lanes)
        res[lanes] = _time(lambda: nv.sph_forces(sim.ctx, t["vel_e"], t["rho"],
                                                 t["mass"][:sim.n_gas], t["acc_hyd"]), reps)
    best = min(res, key=res.get)
    sim.set_lanes(best)
    return best, res
