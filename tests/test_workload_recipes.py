"""The seeded draws behind the batched-ensemble and serving workloads follow
the distributions their configurations state, and bench.py's roofline and
traffic bookkeeping does the arithmetic it documents (host logic only)."""
import math
import os

import numpy as np
from scipy import stats

from paper_1807_08116_gb300 import ics


def _ks_uniform(x, lo, hi):
    return stats.kstest((np.asarray(x, float) - lo) / (hi - lo), "uniform").pvalue


def test_ensemble_draws():
    # 64 collisions: total N log-uniform in [8192, 262144] (to a multiple of 4),
    # impact parameter U[0, 4a], speed U[0.5, 2] x escape; a larger draw of the
    # same generator checks the shapes
    ps = ics.ensemble_params(4096, seed=3)
    n = np.array([p["n"] for p in ps])
    assert n.min() >= 8192 and n.max() <= 262144 and np.all(n % 4 == 0)
    assert _ks_uniform(np.log(n), math.log(8192), math.log(262144)) > 1e-3
    assert _ks_uniform([p["b"] for p in ps], 0.0, 4.0) > 1e-3
    assert _ks_uniform([p["speed_factor"] for p in ps], 0.5, 2.0) > 1e-3


def test_serving_trace_draws():
    # Poisson arrivals at 20 requests/s, N log-uniform in [4096, 1048576],
    # step counts uniform on {10, ..., 1000}
    tr = ics.serving_trace(n_jobs=5000, rate=20.0, seed=4)
    t = np.array([x["t"] for x in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert stats.kstest(gaps, "expon", args=(0, 1 / 20.0)).pvalue > 1e-3
    assert abs(len(t) / t[-1] - 20.0) < 1.0
    n = np.array([x["n"] for x in tr])
    assert n.min() >= 4096 and n.max() <= 1048576 and np.all(n % 4 == 0)
    assert _ks_uniform(np.log(n), math.log(4096), math.log(1048576)) > 1e-3
    steps = np.array([x["steps"] for x in tr])
    assert steps.min() >= 10 and steps.max() <= 1000
    assert abs(steps.mean() - 505.0) < 10.0


def test_from_params_particle_counts():
    d = ics.from_params(8192, 1.0, 1.0, 11)
    assert d["n"] == 8192 and d["n_gas"] == 4096


def test_stage_roofline_arithmetic(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "hbm_peak", lambda: (1000.0, "test"))
    ms = {"sp": 1.0, "dc": 2.0, "hfc_pred": 1.0, "hfc_corr": 1.0, "su_pred": 0.5,
          "su_corr": 0.5, "nb": 4.0}
    out = bench.stage_roofline(ms, n=2000, ng=1000, nb_entries=50000)
    # sort 150 B per gas particle over 1 ms: 150e3 B / 1e-3 s = 0.15 GB/s
    assert math.isclose(out["sp"]["gbs"], 0.15) and math.isclose(out["sp"]["frac"], 0.15 / 1000)
    # density 300 B per gas particle over 2 ms
    assert math.isclose(out["dc"]["bytes"], 300e3) and math.isclose(out["dc"]["gbs"], 0.15)
    # each leapfrog phase 180 B per particle (all 2000) over 0.5 ms
    assert math.isclose(out["su_pred"]["bytes"], 360e3) and math.isclose(out["su_pred"]["gbs"], 0.72)
    # lists: 4 B per entry plus 4 B per row start
    assert math.isclose(out["nb"]["bytes"], 4.0 * 50000 + 4.0 * 1001)
    assert out["peak_gbs"] == 1000.0


def test_gravity_traffic_only_while_the_kernel_source_is_unchanged(monkeypatch):
    import hashlib

    import bench
    # the recorded figure applies to the recorded size and source digest only
    rec = bench.GFC_TRAFFIC["pp_gravity_pairs_kernel"]
    src = os.path.join(bench.ROOT, "paper_1807_08116_gb300", "csrc", rec["file"])
    same = hashlib.sha256(open(src, "rb").read()).hexdigest() == rec["sha256"]
    got = bench.gfc_traffic(rec["n"], "pp_gravity_pairs_kernel")
    assert got == (rec["bytes"] if same else None)
    assert bench.gfc_traffic(rec["n"] // 2, "pp_gravity_pairs_kernel") is None
    assert bench.gfc_traffic(rec["n"], "no_such_kernel") is None
    # a changed source drops the figure
    fake = dict(bench.GFC_TRAFFIC)
    fake["pp_gravity_pairs_kernel"] = dict(rec, sha256="0" * 64)
    monkeypatch.setattr(bench, "GFC_TRAFFIC", fake)
    assert bench.gfc_traffic(rec["n"], "pp_gravity_pairs_kernel") is None


def test_fp32_operations_follow_the_masses():
    import bench
    # the pair-once kernel issues 7 FP32-pipe operations per ordered
    # interaction when every tile takes the equal-mass form, 8 otherwise; the
    # one-sided kernel 12 either way
    eq = np.full(1000, 1e-3, np.float32)
    mixed = eq.copy()
    mixed[17] = np.nextafter(mixed[17], np.float32(1.0))
    assert bench.fp32_ops("pp_gravity_pairs_kernel", eq) == 7
    assert bench.fp32_ops("pp_gravity_pairs_kernel", mixed) == 8
    assert bench.fp32_ops("pp_gravity_kernel", eq) == 12
    assert bench.fp32_ops("pp_gravity_kernel", mixed) == 12


def test_pairs_crossover_choice():
    from paper_1807_08116_gb300.tune import pairs_crossover
    # (one-sided ms, pair-once ms) per size
    assert pairs_crossover({8192: (0.07, 0.15), 16384: (0.25, 0.21), 32768: (0.51, 0.38)}) == 16384
    # a win below a loss does not count: the threshold is where the wins stay
    assert pairs_crossover({8192: (0.2, 0.1), 16384: (0.2, 0.3), 32768: (0.5, 0.4)}) == 32768
    assert pairs_crossover({8192: (0.1, 0.2), 16384: (0.2, 0.3)}) is None
    assert pairs_crossover({}) is None
