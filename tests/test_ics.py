"""The synthetic Plummer inputs have the distribution they claim."""
import math

import numpy as np
from scipy import stats

from paper_1807_08116_gb300 import ics


def test_plummer_mass_profile():
    d = ics.single_halo(4096, 4096, seed=0)
    rr = np.linalg.norm(d["r"], axis=1)
    # cumulative mass fraction r^3/(1+r^2)^1.5, truncated at 0.999
    cdf = lambda x: np.minimum(1.0, (x ** 3 / (1 + x * x) ** 1.5) / ics.MFRAC_MAX)
    assert stats.kstest(rr, cdf).pvalue > 1e-3


def test_dark_particles_are_virialised():
    d = ics.single_halo(0, 20000, seed=1)
    v2 = np.sum(d["v"] ** 2, axis=1)
    K = 0.5 * float(np.sum(d["m"].astype(np.float64) * v2))
    # Plummer kinetic energy 3 pi G M^2 / (64 a) (half of |W|)
    assert abs(K / (3 * math.pi / 64) - 1) < 0.03


def test_two_halo_layout():
    d = ics.two_halo(1000, 1000, seed=5)
    n_gas = d["n_gas"]
    assert n_gas == 2000 and d["n"] == 4000
    m = d["m"].astype(np.float64)
    com = (m[:, None] * d["r"]).sum(0) / m.sum()
    vcm = (m[:, None] * d["v"]).sum(0) / m.sum()
    assert np.all(np.abs(vcm) < 0.05)
    gasA = d["r"][:1000].mean(0)
    gasB = d["r"][1000:2000].mean(0)
    assert abs((gasB - gasA)[0] - 10) < 1.0 and abs((gasB - gasA)[1] - 2) < 1.0
    v_rel = 1.5 * math.sqrt(4.0 / math.sqrt(104.0))
    assert abs(d["v"][1000, 0] - d["v"][0, 0] + v_rel) < 1e-12
    assert np.all(d["h"] > 0) and np.all(d["e"] > 0)
    assert abs(d["e"][0] - math.pi / 32 / (2.0 / 3.0)) < 1e-12


def test_determinism_and_param_draws():
    a = ics.two_halo(100, 100, seed=7)
    b = ics.two_halo(100, 100, seed=7)
    assert np.array_equal(a["r"], b["r"]) and np.array_equal(a["v"], b["v"])
    ps = ics.ensemble_params(64, seed=3)
    ns = np.array([p["n"] for p in ps])
    assert ns.min() >= 8192 and ns.max() <= 262144 and np.all(ns % 4 == 0)
    tr = ics.serving_trace(50)
    assert all(tr[i]["t"] < tr[i + 1]["t"] for i in range(49))
