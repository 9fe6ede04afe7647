"""Benchmark of the self-gravitating SPH step on GB300.

One "step" is one predictor-corrector step of the whole hot path (HFC, SU,
SP, neighbour lists, DC, GFC, HFC, SU) over the large two-halo collision,
2 x (1,048,576 gas + 1,048,576 dark) = 4,194,304 particles, FP32 forces with
FP64 leapfrog accumulators.  Metric: particle-steps per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank advances its own
independent replica of the workload (the step does not shard across GPUs
here: replicas only); value = particles x steps summed over ranks / the
slowest rank's time.

--impl reference times the FP64 CPU oracle on this host's cores on a bounded
sample of the same workload (target rows of every stage), extrapolated to a
whole step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (gas per halo, dark per halo, halos, seed, dt)
    "large": (1048576, 1048576, 2, 2, 1e-3),
    "two_halo": (131072, 131072, 2, 1, 1e-3),
    "single": (8192, 8192, 1, 0, 1e-3),
}
WORKLOAD_NAMES = {
    "large": "large two-halo collision 2x(1048576 gas + 1048576 dark), Plummer a=G=M=1",
    "two_halo": "two-halo collision 2x(131072 gas + 131072 dark), Plummer a=G=M=1",
    "single": "single Plummer halo 8192 gas + 8192 dark",
}
# DRAM bytes (read + write) of one gravity launch on the large two-halo
# workload, per kernel source, from an ncu capture of the source file with
# this SHA-256 (a figure is reported only while that file is unchanged).
GFC_TRAFFIC = {
    "pp_gravity_kernel": {"file": "gravity.cu", "n": 4194304, "bytes": 870.39e6,
                          "sha256": "84874065d5e239daf0a7be2711544d692b425dceaf2c41660785f2920f804721"},
    "pp_gravity_pairs_kernel": {"file": "gravity_pairs.cu", "n": 4194304, "bytes": 2.352522496e9,
                                "sha256": "7525917b0ee5448cdc0289209f2f206f9d20dd0cbbfbb30a4ca339e567265a02"},
}
FLOP_PER_INTERACTION = 20   # the usual direct-N-body convention
FP32_LANES_PER_SM = 128      # FP32 lanes per SM on Blackwell (4 partitions x 32)
SM_MAX_MHZ_FALLBACK = 2070.0


def sm_max_mhz(clk=None):
    """Maximum SM clock: the one nvidia-smi reported while the step ran, else
    the pool's measured record, else GB300's nominal 2070 MHz."""
    if clk and clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"])
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return SM_MAX_MHZ_FALLBACK


def fp32_lane_ops_per_s(sm_count, mhz):
    """FP32 pipe issue rate: SMs x 128 lanes x clock (one operation per lane
    per clock; an FMA counts as 2 flop)."""
    return sm_count * FP32_LANES_PER_SM * mhz * 1e6


def fp32_peak_tflops(sm_count, mhz):
    return 2.0 * fp32_lane_ops_per_s(sm_count, mhz) / 1e12


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over all ranks (x itself with one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, n, steps, ms):
    """Whole-job particle-steps/s: every rank advanced its own replica of n
    particles by `steps` steps; the job took the slowest rank's `ms`."""
    return world * n * steps / (ms / 1e3)


def gfc_traffic(n, kernel="pp_gravity_kernel"):
    """Per-launch DRAM bytes of a gravity kernel if its capture applies."""
    import hashlib
    rec = GFC_TRAFFIC.get(kernel)
    if rec is None or rec["bytes"] is None or n != rec["n"]:
        return None
    src = os.path.join(ROOT, "paper_1807_08116_gb300", "csrc", rec["file"])
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    return rec["bytes"] if digest == rec["sha256"] else None


# Algorithmic DRAM bytes of the SPH and sort stages per unit (the minimal
# traffic of each stage's data): sort (bin, scan, scatter, gather) 150 B and
# density 300 B per gas particle, each force pass 330 B per gas particle,
# each leapfrog phase 180 B per particle; the neighbour lists 4 B per entry
# plus 4 B per row start.
STAGE_BYTES = {"sp": ("gas", 150.0), "dc": ("gas", 300.0), "hfc_pred": ("gas", 330.0),
               "hfc_corr": ("gas", 330.0), "su_pred": ("all", 180.0), "su_corr": ("all", 180.0)}
HBM_FALLBACK_GBS = 6800.0


def hbm_peak():
    """Measured copy bandwidth of this GPU (GB/s) and where it came from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback 6.8 TB/s (no measured peak on this machine)"


def stage_roofline(stage_ms, n, ng, nb_entries):
    """Achieved GB/s of each HBM-bound stage: algorithmic bytes / stage time."""
    peak, note = hbm_peak()
    out = {"peak_gbs": peak, "peak_note": note}
    for k, (unit, b) in STAGE_BYTES.items():
        if k in stage_ms and stage_ms[k] > 0:
            byts = b * (ng if unit == "gas" else n)
            gbs = byts / (stage_ms[k] / 1e3) / 1e9
            out[k] = {"bytes": byts, "gbs": gbs, "frac": gbs / peak}
    if nb_entries is not None and stage_ms.get("nb", 0) > 0:
        byts = 4.0 * nb_entries + 4.0 * (ng + 1)
        gbs = byts / (stage_ms["nb"] / 1e3) / 1e9
        out["nb"] = {"bytes": byts, "gbs": gbs, "frac": gbs / peak}
    return out


# FP32-pipe operations per ordered interaction: the one-sided kernel does
# 3 FADD + 3 FFMA + 3 FMUL + 3 FFMA (+1 MUFU); the pair-once kernel does 16
# per unordered pair (3 FADD, 3 FFMA, 4 FMUL, 2 x 3 FFMA), i.e. 8 per
# ordered interaction, and 14 (7 per ordered interaction) in tiles whose
# bodies all have the same mass (the mass products leave the pair term).
FP32_OPS = {"pp_gravity_kernel": 12, "pp_gravity_pairs_kernel": 8}
FP32_OPS_EQUAL_MASS = {"pp_gravity_kernel": 12, "pp_gravity_pairs_kernel": 7}


def fp32_ops(kernel, masses):
    """FP32-pipe operations per ordered interaction of the kernel on these
    masses (every tile takes the equal-mass form when all masses are equal)."""
    m = np.asarray(masses)
    equal = m.size > 0 and bool(np.all(m == m.flat[0]))
    return (FP32_OPS_EQUAL_MASS if equal else FP32_OPS)[kernel]


def make_ic(name, rank=0):
    from paper_1807_08116_gb300 import ics
    g, d, halos, seed, _ = WORKLOADS[name]
    if halos == 1:
        return ics.single_halo(g, d, seed=seed + rank)
    return ics.two_halo(g, d, seed=seed + rank)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------

def oracle_sample(ic, rows_grav=256, rows_gas=256, seed=0):
    """Time the FP64 oracle on `rows_grav` gravity targets (over all N sources)
    and `rows_gas` gas targets (density + two hydro evaluations, brute force
    over all gas), then extrapolate to one full step (two HFC, one DC, one GFC
    per step; the O(N) integrator is timed in full).  Returns
    (particle-steps/s, seconds per extrapolated step, threads, description)."""
    import oracle
    n, ng = ic["n"], ic["n_gas"]
    rng = np.random.default_rng(seed)
    rg = np.sort(rng.choice(n, min(rows_grav, n), replace=False)).astype(np.int32)
    rh = np.sort(rng.choice(ng, min(rows_gas, ng), replace=False)).astype(np.int32)
    pm = np.empty((n, 4), np.float32)
    pm[:, :3] = ic["r"]
    pm[:, 3] = ic["m"]
    ph = np.empty((ng, 4), np.float32)
    ph[:, :3] = ic["r"][:ng]
    ph[:, 3] = ic["h"]
    ve = np.empty((ng, 4), np.float32)
    ve[:, :3] = ic["v"][:ng]
    ve[:, 3] = ic["e"]
    mass = ic["m"][:ng].astype(np.float32)
    oracle.density(ph[:8], mass[:8])   # load / build outside the timing
    t0 = time.perf_counter()
    oracle.gravity(pm, rows=rg)
    t_grav = time.perf_counter() - t0
    t0 = time.perf_counter()
    rho, _ = oracle.density(ph, mass, rows=rh)
    t_dc = time.perf_counter() - t0
    rho_all = np.ones(ng, np.float32)
    rho_all[rh] = rho
    t0 = time.perf_counter()
    oracle.hydro(ph, ve, mass, rho_all, rows=rh)
    t_hfc = time.perf_counter() - t0
    # integrator on the whole state (both phases)
    r = np.ascontiguousarray(ic["r"].T)
    v = np.ascontiguousarray(ic["v"].T)
    e = ic["e"].copy()
    vs, es = np.zeros_like(v), np.zeros_like(e)
    zeros_h = np.zeros((ng, 3))
    zeros_g = np.zeros((n, 3))
    t0 = time.perf_counter()
    oracle.predict(ng, 1e-3, r, v, e, vs, es, zeros_h, np.zeros(ng), zeros_g)
    oracle.correct(ng, 1e-3, v, e, vs, es, zeros_h, np.zeros(ng), zeros_g)
    t_su = time.perf_counter() - t0
    t_step = t_grav * n / len(rg) + (t_dc + 2 * t_hfc) * ng / len(rh) + t_su
    threads = oracle.threads()
    desc = (f"{len(rg)} of {n} gravity targets, {len(rh)} of {ng} gas targets (density + 2 hydro), "
            f"brute force FP64, extrapolated to one step; integrator over all particles; "
            f"sampled {t_grav + t_dc + t_hfc + t_su:.1f} s")
    return n / t_step, t_step, threads, desc


def gravity_parity(sim, n_rows=64, seed=11):
    """Accelerations of the last gravity evaluation on sampled rows against the
    FP64 oracle over all sources at the same FP32 positions: rms relative
    error, the maximum relative error with the 1% rms floor of the tests, and
    the plain maximum |da_i| / |a_i|."""
    import oracle
    pm = sim.t["pos_m"].cpu().numpy()
    g = sim.t["grav"][:, :3].cpu().numpy().astype(np.float64)
    n = pm.shape[0]
    rows = np.sort(np.random.default_rng(seed).choice(n, min(n_rows, n), replace=False)).astype(np.int32)
    ref, _ = oracle.gravity(pm, sim.params["G"], sim.params["eps"], rows=rows)
    d = np.linalg.norm(g[rows] - ref, axis=1)
    nr = np.linalg.norm(ref, axis=1)
    rms_ref = float(np.sqrt(np.mean(nr ** 2)))
    return {"rows": int(len(rows)), "rms_rel": float(np.sqrt((d ** 2).sum() / (nr ** 2).sum())),
            "max_rel_floored": float(np.max(d / (nr + 0.01 * rms_ref))),
            "max_rel_plain": float(np.max(d / nr)),
            "note": "gravity of the final timed state on sampled rows vs the FP64 oracle over all "
                    "sources; floor = 1% of the rms |a| (the tests' metric)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    ic = make_ic(args.workload)
    vals = []
    for k in range(args.warmup + args.steps):
        v, t_step, threads, desc = oracle_sample(ic, args.ref_rows, args.ref_rows, seed=k)
        if k >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": "particle-steps/s", "value": value,
        "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * ic["n"] / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload], "n": ic["n"], "n_gas": ic["n_gas"]},
        "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": threads,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def energy_momentum(sim):
    """Total energy (kinetic + thermal + potential, FP64 sums) and momentum of
    a simulation's current state; the potential comes from one extra gravity
    evaluation with the potential flag on the FP32 positions."""
    import torch

    from paper_1807_08116_gb300 import native as nv
    d = sim.diagnostics()
    phi = torch.empty_like(sim.t["pos_m"])
    nv.pp_gravity(sim.t["pos_m"], phi, G=sim.params["G"], eps=sim.params["eps"],
                  flags=nv.SPH_GRAV_POTENTIAL)
    pot = 0.5 * float((sim.t["mass"].double() * phi[:, 3].double()).sum())
    p = np.asarray(d["momentum"], dtype=np.float64)
    return {"E": float(d["kinetic"] + d["thermal"] + pot), "p": p,
            "p_scale": float(np.sqrt(2.0 * d["kinetic"] * d["mass"]))}


def run_ours(args):
    import torch

    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.sim import Simulation

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    nv.lib()
    ic = make_ic(args.workload, rank)
    n, ng = ic["n"], ic["n_gas"]
    dt = WORKLOADS[args.workload][4]
    sim = Simulation(ic)
    sim.initial_rhs()
    for _ in range(args.warmup):
        sim.step(dt)
    torch.cuda.synchronize()

    cons0 = energy_momentum(sim) if args.conservation else None

    # ---- device-resident timed region ------------------------------------
    evs = [nv.StageEvents() for _ in range(args.steps)]
    stream = torch.cuda.current_stream()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = nv.sph_launch_count()
    t_start.record(stream)
    for k in range(args.steps):
        sim.state.events = evs[k].ptr
        sim.step(dt, check=False)
    t_stop.record(stream)
    launches = nv.sph_launch_count() - launches0
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    sim.state.events = None
    flags = sim.ctx.device_status() if sim.ctx is not None else 0
    if flags:
        raise RuntimeError(f"device status flags {flags} during the timed steps")
    nb_entries = sim.ctx.nb_total() if (sim.ctx is not None and ng > 0) else None
    ms = t_start.elapsed_time(t_stop)
    stage = {name: float(np.mean([e.stage_ms()[name] for e in evs])) for name in nv.STAGES}
    for e in evs:
        e.close()
    ms = max_over_ranks(ms, dist, "cuda")
    value = aggregate_rate(world, n, args.steps, ms)
    conservation = None
    if cons0 is not None:
        cons1 = energy_momentum(sim)
        conservation = {
            "steps": args.steps, "dt": dt, "E0": cons0["E"], "E1": cons1["E"],
            "dE_over_E": abs(cons1["E"] - cons0["E"]) / abs(cons0["E"]),
            "dp_over_p_scale": float(np.abs(cons1["p"] - cons0["p"]).max() / cons0["p_scale"]),
            "note": "outside the timed region; potential from a separate gravity evaluation"}

    # ---- end to end through the C ABI with host buffers --------------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(sim, args, dt, barrier, dist, world, n, ng)

    # ---- roofline of the dominant kernel (gravity) -------------------------
    gfc_ms = stage["gfc"]
    achieved = FLOP_PER_INTERACTION * float(n) * float(n) / (gfc_ms / 1e3) / 1e12
    ips = float(n) * n / (gfc_ms / 1e3)
    if "grav_work" in sim.t and nv.pp_gravity_pairs_eligible(n, sim.params["eps"], sim.grav_flags):
        kernel = "pp_gravity_pairs_kernel"
        th, R, lg = nv.pp_gravity_pairs_get_plan(n)
        plan = {"scheme": "each unordered pair once (Newton's third law)", "block": th * R,
                "threads": th, "targets_per_thread": R, "super_tile_log2": lg}
    else:
        kernel = "pp_gravity_kernel"
        R, S = nv.sph_gravity_plan(n)
        plan = {"scheme": "one-sided", "targets_per_thread": R, "cluster_split": S}
    ops = fp32_ops(kernel, sim.t["mass"].cpu().numpy())
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz_max = sm_max_mhz(clk)
    mhz_run = float(clk["sm_mhz"]) if clk and clk.get("sm_mhz") else mhz_max
    peak = fp32_peak_tflops(sms, mhz_max)
    peak_run = fp32_peak_tflops(sms, mhz_run)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": args.gfc_traffic if args.gfc_traffic is not None else gfc_traffic(n, kernel),
            "kernel": kernel, "interactions_per_s": ips,
            "flop_per_interaction": FLOP_PER_INTERACTION,
            "fp32_ops_per_interaction": ops,
            "fp32_pipe_frac": ops * ips / fp32_lane_ops_per_s(sms, mhz_max),
            "sm_count": sms, "sm_max_mhz": mhz_max, "sm_mhz": mhz_run,
            "peak_at_sm_mhz": peak_run, "frac_at_sm_mhz": achieved / peak_run,
            "peak_note": f"FP32 pipe {sms} SM x {FP32_LANES_PER_SM} lanes x 2 flop x {mhz_max:.0f} MHz "
                         "(the device's SM count and maximum SM clock; derived, not measured); "
                         "achieved counts 20 flop per ordered interaction (N^2 per evaluation); "
                         "frac_at_sm_mhz takes the median SM clock sampled during the timed steps",
            "plan": plan}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, t_step, threads, desc = oracle_sample(ic, args.cpu_rows, args.cpu_rows)
        cpu = {"value": v, "unit": "particle-steps/s", "cores": threads, "kind": "oracle",
               "sample": desc}
        # the same oracle on one host thread, on a sample 1/16 the size
        import oracle
        oracle.set_threads(1)
        try:
            rows1 = max(64, args.cpu_rows // 16)
            v1, _, threads1, desc1 = oracle_sample(ic, rows1, rows1, seed=1)
        finally:
            oracle.set_threads(threads)
        cpu["single_thread"] = {"value": v1, "cores": threads1, "sample": desc1}
        # the sampled oracle rows double as a parity check of the timed state
        cpu["gravity_parity"] = gravity_parity(sim)

    if rank == 0:
        line = {
            "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES[args.workload], "n": n, "n_gas": ng, "dt": dt,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (state and lists > 129 MB)",
                       "precision": "FP32 forces (compensated sums), FP64 leapfrog state"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "stage_ms": stage, **({"conservation": conservation} if conservation else {}),
            "stage_roofline": stage_roofline(stage, n, ng, nb_entries),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_e2e(sim, args, dt, barrier, dist, world, n, ng):
    """Same metric through the C-ABI step with the state in pinned host
    memory: every step uploads r, v, e, h, runs sph_step and downloads r, v, e."""
    import torch

    from paper_1807_08116_gb300 import native as nv
    t = sim.t
    host = {k: torch.empty(t[k].shape, dtype=t[k].dtype, pin_memory=True)
            for k in ("r", "v", "e", "h")}
    for k in host:
        host[k].copy_(t[k])
    torch.cuda.synchronize()
    h2d = sum(host[k].numel() * host[k].element_size() for k in ("r", "v", "e", "h"))
    d2h = sum(host[k].numel() * host[k].element_size() for k in ("r", "v", "e"))
    steps = max(1, args.e2e_steps if args.e2e_steps is not None else args.steps)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for k in ("r", "v", "e", "h"):
            t[k].copy_(host[k], non_blocking=True)
        nv.sph_step(sim.ctx, sim.state, dt)
        for k in ("r", "v", "e"):
            host[k].copy_(t[k], non_blocking=True)
        torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    return {"value": aggregate_rate(world, n, steps, el * 1e3), "unit": "particle-steps/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": steps}


def run_ensemble(args):
    """Batched ensemble: 64 independent two-halo collisions (total particles
    per simulation log-uniform in [8192, 262144], impact parameter U[0, 4a],
    speed U[0.5, 2] x escape) advanced (a) as one batch -- one launch per
    stage (gravity: the pair-once kernel over the tiles of every simulation),
    the step captured as a CUDA graph --
    and (b) one simulation at a time with the single-simulation launches.
    Prints one JSON line with both aggregate particle-steps/s and the largest
    relative position difference between the two runs."""
    import torch

    from paper_1807_08116_gb300 import ics
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.sim import Simulation, assemble_batch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    nv.lib()
    params = ics.ensemble_params(args.n_sims, seed=3)
    lst = [ics.from_params(**p) for p in params]
    n_tot = sum(d["n"] for d in lst)
    dt = 1e-3
    ic, go, do, so = assemble_batch(lst)

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # (a) batched
    from paper_1807_08116_gb300.tune import tune_batch, tune_batch_pairs_plan, tune_grid, tune_lanes
    bsim = Simulation(ic, batch_offsets=(go, do, so))
    bsim.initial_rhs()
    pairs = "grav_work" in bsim.t   # pair-once gravity over all simulations' tiles
    best_R, tune = None, None
    if not pairs:
        best_R, tune = tune_batch(bsim.batch, bsim.t["pos_m"], reps=3)
    for _ in range(args.warmup):
        bsim.step(dt)
    # the SPH knobs of the batch, tuned after the warm-up steps (the initial
    # smoothing lengths give a few outlying rows with huge lists): grid cell
    # size and lanes per neighbour row
    best_shift, tune_shift = tune_grid(bsim, reps=3)
    best_lanes, tune_l = tune_lanes(bsim, reps=3)
    best_plan, tune_plan = None, None
    if pairs:   # the block shape of the pair-once launch over all simulations' tiles
        best_plan, tune_plan = tune_batch_pairs_plan(bsim.batch, bsim.t["pos_m"], bsim.t["grav_work"],
                                                     reps=2)
        tune_plan = {str(list(k)): v for k, v in tune_plan.items()}
    bsim.capture(dt)
    launches0 = nv.sph_launch_count()
    ms_b = timed(lambda: bsim.replay(check=False), args.steps)
    flags = bsim.ctx.device_status()
    if flags:
        raise RuntimeError(f"device flags {flags} in the batched run")

    # (b) one simulation at a time, each launch with the library's default
    # pair-once plan (the tuned plan was chosen for the batched launch)
    nv.pp_gravity_pairs_plan(0)
    sims = [Simulation(d) for d in lst]
    for sm in sims:
        sm.initial_rhs()
    for _ in range(args.warmup):
        for sm in sims:
            sm.step(dt)
    torch.cuda.synchronize()

    def seq_step():
        for sm in sims:
            sm.step(dt, check=False)
    ms_s = timed(seq_step, args.steps)

    rb = bsim.positions()
    worst = 0.0
    for k, sm in enumerate(sims):
        r = sm.positions()
        worst = max(worst, float(np.abs(rb[bsim.sim_slices(k)] - r).max() / max(np.abs(r).max(), 1e-30)))
    # stage breakdown of one more batched step (eager, outside the timed region,
    # after the comparison of positions)
    if best_plan:
        nv.pp_gravity_pairs_plan(best_plan[0], best_plan[1], -1)
    ev = nv.StageEvents()
    bsim.state.events = ev.ptr
    bsim.step(dt, check=False)
    torch.cuda.synchronize()
    bsim.state.events = None
    stage_b = ev.stage_ms()
    ev.close()
    v_b = n_tot * args.steps / (ms_b / 1e3)
    v_s = n_tot * args.steps / (ms_s / 1e3)
    line = {
        "metric": "ensemble aggregate particle-steps/s", "value": v_b, "unit": "particle-steps/s",
        "sequential_value": v_s, "speedup_vs_sequential": v_b / v_s, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b / args.steps,
        "sequential_ms_per_step": ms_s / args.steps, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"ensemble of {args.n_sims} two-halo collisions, "
                               "N log-uniform in [8192, 262144], b ~ U[0,4a], v ~ U[0.5,2] v_esc",
                   "n_total": n_tot, "n_sims": args.n_sims, "cuda_graph": True,
                   "gravity": ("pair-once, one launch over the tiles of every simulation" if pairs
                               else "one-sided persistent work queue"),
                   "gravity_units_R": best_R, "autotune_ms": tune,
                   "tuned": {"grid_shift": best_shift, "grid_shift_ms": tune_shift,
                             "lanes": best_lanes, "lanes_ms": tune_l,
                             "pairs_plan": list(best_plan) if best_plan else None,
                             "pairs_plan_ms": tune_plan}},
        "max_rel_position_diff_batched_vs_sequential": worst,
        "stage_ms_batched": stage_b,
        "interactions_per_step": float(sum(d["n"] ** 2 for d in lst)),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving stream: Poisson arrivals (20 req/s) of two-halo jobs, sizes
    log-uniform in [4096, 1048576], steps uniform in [10, 1000], admitted by a
    device-memory budget (150 GB) into a continuously batched server.  The
    offered load far exceeds one GPU, so the run is a bounded trace (the first
    --serve-jobs arrivals) over a bounded wall-clock window; the line reports
    offered against served load beside the latencies."""
    import torch

    from paper_1807_08116_gb300 import ics
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server, replay_trace

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    nv.lib()
    trace = ics.serving_trace(n_jobs=args.serve_jobs, rate=20.0, seed=4)
    made = {}
    t0 = time.perf_counter()
    for k, req in enumerate(trace):     # inputs prepared before the clock starts
        made[k] = ics.from_params(req["n"], req["b"], req["speed_factor"], req["seed"])
    prep_s = time.perf_counter() - t0
    for k, req in enumerate(trace):
        req["k"] = k
    server = Server(int(args.serve_budget_gb * (1 << 30)), max_resident=args.max_resident,
                    n_streams=8)
    server.set_policy(nv.SPH_SERVE_SHORTEST_FIRST if args.serve_policy == "sjf" else nv.SPH_SERVE_FIFO)
    jobs, steps, wall = replay_trace(server, trace, lambda req: made[req["k"]], args.serve_window)
    done = [j for j in jobs.values() if j["state"] == nv.SIM_DONE]
    lat = np.array([j["latency_s"] for j in done]) if done else np.zeros(0)
    # every simulation step's own latency (CUDA events on its stream)
    step_ms = server.step_times()
    call_ms = np.array([x["ms"] for x in steps if x["resident"] or x["ms"] > 0])
    served_ps = sum(j["steps_done"] * j["n"] for j in jobs.values())
    served_int = sum(j["steps_done"] * float(j["n"]) ** 2 for j in jobs.values())
    span = max(x["t"] for x in trace) - min(x["t"] for x in trace)
    offered_ps = sum(x["steps"] * x["n"] for x in trace) / max(span, 1e-9)
    offered_int = sum(x["steps"] * float(x["n"]) ** 2 for x in trace) / max(span, 1e-9)
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    line = {
        "metric": "serving aggregate particle-steps/s", "value": served_ps / wall,
        "unit": "particle-steps/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "serving stream: Poisson 20 req/s two-halo jobs, N log-uniform "
                               "[4096, 1048576], steps U{10..1000}",
                   "jobs_in_trace": len(trace), "window_s": args.serve_window,
                   "budget_gb": args.serve_budget_gb, "max_resident": args.max_resident,
                   "admission": args.serve_policy,
                   "input_prep_s": prep_s},
        "step_latency_ms": {"p50": pct(step_ms, 50), "p99": pct(step_ms, 99), "count": len(step_ms),
                            "note": "each simulation step's own CUDA-event time on its stream"},
        "server_call_ms": {"p50": pct(call_ms, 50), "p99": pct(call_ms, 99), "count": len(call_ms)},
        "request_latency_s": {"p50": pct(lat, 50), "p99": pct(lat, 99), "completed": len(done),
                              "completed_small": sum(1 for j in done if j["n"] < 131072)},
        "offered": {"particle_steps_per_s": offered_ps, "interactions_per_s": offered_int},
        "served": {"particle_steps_per_s": served_ps / wall, "interactions_per_s": served_int / wall},
        "submitted": len(jobs), "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sort(args):
    """The sorting stage alone on the gas of the two-halo construction with
    --n particles (half gas): sph_bin_and_sort as one cooperative launch and
    as its kernel sequence, --warmup untimed and --steps timed sorts each,
    CUDA events; the results of the two forms are bitwise equal (tested)."""
    import torch

    from paper_1807_08116_gb300 import ics
    from paper_1807_08116_gb300 import native as nv

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    nv.lib()
    q = args.n // 4
    d = ics.two_halo(q, q, seed=2)
    ng = d["n_gas"]
    ph = np.empty((ng, 4), np.float32)
    ph[:, :3] = d["r"][:ng]
    ph[:, 3] = d["h"]
    x = torch.as_tensor(ph, device="cuda")
    ctx = nv.Ctx(ng, 1024)
    res = {}
    for fused in (0, 1):
        ctx.set_sort_fused(fused)
        for _ in range(args.warmup):
            nv.sph_bin_and_sort(ctx, x)
        torch.cuda.synchronize()
        l0 = nv.sph_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            nv.sph_bin_and_sort(ctx, x)
        e1.record()
        torch.cuda.synchronize()
        res[fused] = (e0.elapsed_time(e1) / args.steps, (nv.sph_launch_count() - l0) / args.steps)
    peak, note = hbm_peak()
    byts = STAGE_BYTES["sp"][1] * ng
    print(json.dumps({"metric": "sort stage ms", "n_gas": ng, "steps": args.steps, "warmup": args.warmup,
                      "one_launch_ms": res[1][0], "sequence_ms": res[0][0],
                      "kernels_per_sort": {"one_launch": res[1][1], "sequence": res[0][1]},
                      "gbs_one_launch": byts / (res[1][0] / 1e3) / 1e9,
                      "frac_of_hbm": byts / (res[1][0] / 1e3) / 1e9 / peak, "peak_note": note}),
          flush=True)
    return 0


def run_gravity_sharded(args):
    """Gravity over --n particles split across the ranks by the paper's
    particle partition (Sect. 3): per launch, one all-gather of (x, y, z, m)
    (NCCL) and each rank's own rows over all sources (pp_gravity_rows, the
    one-sided kernel).  Total work is fixed (strong scaling); value = N^2
    interactions / the slowest rank's time per launch."""
    import torch

    from paper_1807_08116_gb300 import ics
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.shard import owned_rows, sharded_gravity

    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    nv.lib()
    q = args.n // 4
    d = ics.two_halo(q, q, seed=2)      # the same particles on every rank
    n = d["n"]
    i0, i1 = owned_rows(n)
    pm = np.empty((n, 4), np.float32)
    pm[:, :3] = d["r"]
    pm[:, 3] = d["m"]
    x = torch.as_tensor(pm[i0:i1].copy(), device="cuda")
    out = torch.empty((i1 - i0, 4), device="cuda")

    def launch():
        sharded_gravity(x, n, out)
    for _ in range(args.warmup):
        launch()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        launch()
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    if nv.pp_gravity_status():
        raise RuntimeError("gravity kernel reported a timeout")
    ips = float(n) * n / (ms / 1e3)
    if rank == 0:
        print(json.dumps({"metric": "PP interactions/s", "value": ips, "unit": "interactions/s",
                          "n": n, "n_gpus": world, "ms_per_launch": ms, "steps": args.steps,
                          "warmup": args.warmup, "scaling": "strong",
                          "config": {"workload": f"gravity of the two-halo construction, {n} bodies",
                                     "parallelism": f"particle partition over {world} rank(s): "
                                                    "all-gather of (x, y, z, m), own rows"},
                          "kernel": "pp_gravity_kernel (rows)",
                          "tflops_20flop": FLOP_PER_INTERACTION * ips / 1e12}), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_gravity(args):
    """Gravity kernel alone on the two-halo construction with --n particles
    (the same inputs the step uses): --warmup untimed and --steps timed
    launches, CUDA events on the launching stream."""
    import torch

    from paper_1807_08116_gb300 import ics
    from paper_1807_08116_gb300 import native as nv

    if args.shard:
        return run_gravity_sharded(args)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    nv.lib()
    q = args.n // 4
    d = ics.two_halo(q, q, seed=2)
    pm = np.empty((d["n"], 4), np.float32)
    pm[:, :3] = d["r"]
    pm[:, 3] = d["m"]
    x = torch.as_tensor(pm, device="cuda")
    out = torch.empty_like(x)
    n = d["n"]
    pairs = not args.one_sided and nv.pp_gravity_pairs_eligible(n, 0.01)
    work = nv.pp_gravity_pairs_workspace(n) if pairs else None
    tuned = None
    if pairs and args.tune:
        from paper_1807_08116_gb300.tune import tune_pairs_plan
        best, res = tune_pairs_plan(x, work, reps=2)
        tuned = {"best": list(best), "ms": {str(list(k)): v for k, v in sorted(res.items())}}

    def launch():
        if pairs:
            nv.pp_gravity_pairs(x, out, work)
        else:
            nv.pp_gravity(x, out)
    for _ in range(args.warmup):
        launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        launch()
    e1.record()
    torch.cuda.synchronize()
    if nv.pp_gravity_status():
        raise RuntimeError("gravity kernel reported a timeout")
    ms = e0.elapsed_time(e1) / args.steps
    ips = float(n) * n / (ms / 1e3)
    kernel = "pp_gravity_pairs_kernel" if pairs else "pp_gravity_kernel"
    if pairs:
        th, R, lg = nv.pp_gravity_pairs_get_plan(n)
        plan = {"scheme": "each unordered pair once", "block": th * R, "threads": th,
                "targets_per_thread": R, "super_tile_log2": lg, "tuned": tuned}
    else:
        R, S = nv.sph_gravity_plan(n)
        plan = {"scheme": "one-sided", "targets_per_thread": R, "cluster_split": S}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_max_mhz()
    print(json.dumps({"metric": "PP interactions/s", "value": ips, "unit": "interactions/s",
                      "n": n, "ms_per_launch": ms, "steps": args.steps, "warmup": args.warmup,
                      "kernel": kernel, "tflops_20flop": FLOP_PER_INTERACTION * ips / 1e12,
                      "frac_of_fp32_peak": FLOP_PER_INTERACTION * ips / 1e12 / fp32_peak_tflops(sms, mhz),
                      "fp32_pipe_frac": fp32_ops(kernel, x[:, 3].cpu().numpy()) * ips /
                      fp32_lane_ops_per_s(sms, mhz),
                      "sm_count": sms, "sm_max_mhz": mhz, "plan": plan}), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["ensemble", "serve", "gravity", "sort"],
                    default="large")
    ap.add_argument("--n", type=int, default=4194304, help="particles of --workload gravity / sort")
    ap.add_argument("--one-sided", action="store_true",
                    help="--workload gravity: time the one-sided kernel instead of the pair-once one")
    ap.add_argument("--tune", action="store_true",
                    help="--workload gravity: time every pair-once plan first and keep the fastest")
    ap.add_argument("--shard", action="store_true",
                    help="--workload gravity: split the rows over the ranks (particle partition, "
                         "one all-gather of the sources per launch)")
    ap.add_argument("--n-sims", type=int, default=64)
    ap.add_argument("--serve-jobs", type=int, default=120)
    ap.add_argument("--serve-window", type=float, default=90.0)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--max-resident", type=int, default=16)
    ap.add_argument("--serve-policy", choices=["fifo", "sjf"], default="fifo",
                    help="admission order of queued requests (sjf: least estimated work first)")
    ap.add_argument("--conservation", action="store_true",
                    help="report the energy and momentum change over the timed steps")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end measurement (default: --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-rows", type=int, default=512,
                    help="target rows per stage of each reference-arm step sample")
    ap.add_argument("--cpu-rows", type=int, default=8192,
                    help="target rows per stage of the cpu_baseline sample")
    ap.add_argument("--gfc-traffic", type=float, default=None,
                    help="DRAM bytes per gravity launch from an ncu capture of this workload")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "gravity":
        return run_gravity(args)
    if args.workload == "sort":
        return run_sort(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
