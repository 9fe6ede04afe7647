"""Autotuning by timing candidates on the device.

Gravity has two kernels: the one-sided one, with two knobs (R targets per
thread, S CTAs per cluster sharing the source range; the batched form has
R), and the pair-once one, with its block shape (threads per CTA, targets
per thread: the j-tile width is the block) and super-tile side, which wins
once a launch has enough tiles to fill the GPU.  A built-in cost model, a
default plan and a measured default crossover choose without timing; these
functions time the candidates instead and fix the fastest
(sph_gravity_tune / sph_batch_set_plan / pp_gravity_pairs_plan /
pp_gravity_pairs_min_n), returning the measurements.  tune_lanes does the
same for the lanes per neighbour row of the SPH sums, tune_grid for the cell
size of the neighbour search's grid.
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


def pairs_crossover(res):
    """The smallest size from which the pair-once time (res[n][1]) beats the
    one-sided time (res[n][0]) at that and every larger measured size, or
    None when it does not win at the largest."""
    threshold = None
    for n in sorted(res, reverse=True):
        if res[n][1] < res[n][0]:
            threshold = n
        else:
            break
    return threshold


def tune_pairs_threshold(make_pos_m, sizes=(8192, 12288, 16384, 24576, 32768, 49152, 65536),
                         G=1.0, eps=0.01, reps=5, apply=True):
    """Time the one-sided kernel (its cost-model plan) and the pair-once
    kernel on make_pos_m(n) for each n in sizes (ascending); the smallest n
    from which the pair-once kernel is faster at every larger size becomes
    the threshold of pp_gravity_pairs_min_n (if apply).  Returns (threshold,
    {n: (one_sided_ms, pairs_ms)}); threshold None if it never wins."""
    res = {}
    nv.pp_gravity_pairs_min_n(1)
    try:
        for n in sizes:
            x = make_pos_m(n)
            out = torch.empty_like(x)
            work = nv.pp_gravity_pairs_workspace(n, device=x.device)
            t1 = _time(lambda: nv.pp_gravity(x, out, G, eps), reps)
            t2 = _time(lambda: nv.pp_gravity_pairs(x, out, work, G, eps), reps)
            res[n] = (t1, t2)
    finally:
        nv.pp_gravity_pairs_min_n(0)
    threshold = pairs_crossover(res)
    if apply and threshold is not None:
        nv.pp_gravity_pairs_min_n(threshold)
    return threshold, res



# pair-once plans: (threads per CTA, targets per thread), i.e. blocks of
# 1024, 768, 1280 and 2048 bodies
PAIRS_SHAPES = [(128, 8), (128, 6), (128, 10), (256, 8)]


def tune_pairs_plan(pos_m, work, G=1.0, eps=0.01, shapes=None, super_offsets=(0, -1, 1), reps=2,
                    apply=True):
    """Time pp_gravity_pairs on pos_m for every block shape and super-tile
    side (the size-chosen side plus the offsets); fix the fastest if apply
    (else restore the default).  Returns ((threads, R, super_log2), {plan: ms})."""
    out = torch.empty_like(pos_m)
    n = pos_m.shape[0]
    res = {}
    try:
        for threads, R in shapes or PAIRS_SHAPES:
            nv.pp_gravity_pairs_plan(threads, R, -1)
            _, _, lg0 = nv.pp_gravity_pairs_get_plan(n)
            for off in super_offsets:
                lg = lg0 + off
                if lg < 0 or lg > 8:
                    continue
                nv.pp_gravity_pairs_plan(threads, R, lg)
                res[(threads, R, lg)] = _time(lambda: nv.pp_gravity_pairs(pos_m, out, work, G, eps), reps)
    finally:
        nv.pp_gravity_pairs_plan(0)
    best = min(res, key=res.get)
    if apply:
        nv.pp_gravity_pairs_plan(*best)
    return best, res


def tune_grid(sim, shifts=(-1, 0, 1), reps=3, apply=True):
    """Time the sort and the neighbour-list build of a Simulation (at its
    current working copies) for each octave shift of the derived grid's
    finest cell; keep the fastest if apply (else restore the shift it had).
    Returns (shift, {shift: ms})."""
    if sim.n_gas == 0:
        return 0, {}
    t = sim.t
    old = sim.grid_shift
    res = {}

    def build():
        nv.sph_bin_and_sort(sim.ctx, t["pos_h"])
        nv.sph_build_neighbors(sim.ctx, sim.n_gas, want_needed=False)
    try:
        for sh in shifts:
            sim.set_grid_shift(sh)
            res[sh] = _time(build, reps)
    finally:
        sim.set_grid_shift(old)
    best = min(res, key=res.get)
    if apply:
        sim.set_grid_shift(best)
    # leave the context's sort and lists as the step expects them
    build()
    return best, res


def tune_batch_pairs_plan(batch, pos_m, work, G=1.0, eps=0.01, shapes=None, reps=2, apply=True):
    """Time pp_gravity_pairs_batched on a batch for every block shape; fix the
    fastest plan if apply (else restore the default).  Returns ((threads, R),
    {shape: ms})."""
    out = torch.empty_like(pos_m)
    res = {}
    try:
        for threads, R in shapes or PAIRS_SHAPES:
            nv.pp_gravity_pairs_plan(threads, R, -1)
            res[(threads, R)] = _time(lambda: nv.pp_gravity_pairs_batched(batch, pos_m, out, work, G, eps),
                                      reps)
    finally:
        nv.pp_gravity_pairs_plan(0)
    best = min(res, key=res.get)
    if apply:
        nv.pp_gravity_pairs_plan(best[0], best[1], -1)
    return best, res
