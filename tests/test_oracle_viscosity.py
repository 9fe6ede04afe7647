"""Pins of the artificial viscosity of the oracle's hydro right-hand side
(Sect. 2.2: nu_ij and mu_ij after Eq. 11, inside Pi_ij of Eqs. 10-11).

- A two-particle head-on case worked by hand from the printed definitions
  (tests/golden/viscosity_head_on.json) fixes the magnitude of nu_ij.
- The viscous part of the force (defaults minus alpha = beta = 0) is
  dissipative: it takes kinetic energy out of a converging flow and puts the
  same amount into heat.
- Copies of the oracle with a plausible mistake planted in the viscosity
  (alpha and beta swapped, the division by rho_ij dropped, c_i in place of
  c_ij, eta squared, h_ij left out of mu_ij) are compiled on the CPU and each
  one fails the head-on pin.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "viscosity_head_on.json")
ORACLE_C = os.path.join(os.path.dirname(HERE), "oracle", "sph_oracle.c")

# FP64 oracle on FP32-exact inputs against a hand calculation carried to 17
# digits: the only difference is FP64 rounding of a few dozen operations
TOL = 1e-12


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _inputs(g):
    ph = np.array(g["pos_h"], np.float32)
    ve = np.array(g["vel_e"], np.float32)
    mass = np.array(g["mass"], np.float32)
    rho = np.array(g["rho"], np.float32)
    return ph, ve, mass, rho


def _rel(a, ref):
    a = np.asarray(a, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def test_golden_inputs_are_exact_in_fp32():
    g = _golden()
    for k in ("pos_h", "vel_e", "mass", "rho"):
        a = np.array(g[k], np.float64)
        assert np.array_equal(a.astype(np.float32).astype(np.float64), a), k


def test_head_on_pair_matches_hand_calculation(orc):
    g = _golden()
    ph, ve, mass, rho = _inputs(g)
    acc, de = orc.hydro(ph, ve, mass, rho, gamma=g["gamma"], alpha=g["alpha"], beta=g["beta"],
                        eta=g["eta"])
    assert _rel(acc, g["acc"]) < TOL
    assert _rel(de, g["dedt"]) < TOL
    # the pressure part alone (alpha = beta = 0 switches the viscosity off)
    acc0, _ = orc.hydro(ph, ve, mass, rho, gamma=g["gamma"], alpha=0.0, beta=0.0, eta=g["eta"])
    assert _rel(acc0, g["acc_without_viscosity"]) < TOL
    # Newton's third law on the pair
    m = mass.astype(np.float64)
    assert abs(m[0] * acc[0, 0] + m[1] * acc[1, 0]) < 1e-14 * abs(m[0] * acc[0, 0])


def test_receding_pair_feels_no_viscosity(orc):
    g = _golden()
    ph, ve, mass, rho = _inputs(g)
    ve[:, :3] *= -1.0    # same speeds, moving apart: mu_ij = 0
    acc, _ = orc.hydro(ph, ve, mass, rho, gamma=g["gamma"], alpha=g["alpha"], beta=g["beta"],
                       eta=g["eta"])
    assert _rel(acc, g["acc_without_viscosity"]) < TOL


def _converging_blob(seed=5, n=400):
    rng = np.random.default_rng(seed)
    r = rng.normal(scale=0.5, size=(n, 3))
    h = (0.12 * (1 + np.sum(r * r, axis=1)) ** 0.5).astype(np.float32)
    v = -0.8 * r + rng.normal(scale=0.05, size=(n, 3))     # collapsing flow
    e = rng.uniform(0.05, 0.3, size=n)
    m = rng.uniform(0.5, 1.5, size=n) / n
    ph = np.empty((n, 4), np.float32)
    ph[:, :3] = r
    ph[:, 3] = h
    ve = np.empty((n, 4), np.float32)
    ve[:, :3] = v
    ve[:, 3] = e
    return ph, ve, m.astype(np.float32)


def test_viscous_part_dissipates_kinetic_into_thermal_energy(orc):
    ph, ve, mass = _converging_blob()
    rho, _ = orc.density(ph, mass)
    rho = rho.astype(np.float32)
    a1, d1 = orc.hydro(ph, ve, mass, rho)
    a0, d0 = orc.hydro(ph, ve, mass, rho, alpha=0.0, beta=0.0)
    av, dv = a1 - a0, d1 - d0
    m = mass.astype(np.float64)
    v = ve[:, :3].astype(np.float64)
    kin = float((m * (v * av).sum(1)).sum())     # d/dt of kinetic energy, viscous part
    th = float((m * dv).sum())                    # d/dt of thermal energy, viscous part
    assert kin < 0.0 and th > 0.0
    # what the viscosity takes from the motion it gives to heat, pair by pair
    assert abs(kin + th) < 1e-10 * th
    # and every particle is heated (or left alone) by it
    assert np.all(dv >= -1e-12 * np.abs(dv).max())


# -- planted mistakes ----------------------------------------------------------

# (name, text in oracle_hydro, replacement): each is a plausible slip in
# writing nu_ij or mu_ij
MUTATIONS = [
    ("alpha and beta swapped", "nu = mu * (beta * mu - alpha * c_ij) / rho_ij;",
     "nu = mu * (alpha * mu - beta * c_ij) / rho_ij;"),
    ("division by rho_ij dropped", "nu = mu * (beta * mu - alpha * c_ij) / rho_ij;",
     "nu = mu * (beta * mu - alpha * c_ij);"),
    ("c_i in place of c_ij", "double c_ij = 0.5 * (c_i + c_j);", "double c_ij = c_i;"),
    ("eta squared", "double mu = hij * rv / (r2 + eta * hij * hij);",
     "double mu = hij * rv / (r2 + eta * eta * hij * hij);"),
    ("h_ij left out of mu", "double mu = hij * rv / (r2 + eta * hij * hij);",
     "double mu = rv / (r2 + eta * hij * hij);"),
]


def _hydro_fn_bounds(src):
    b = src.index("void oracle_hydro(")
    e = src.index("\n}\n", b)
    return b, e


def _build_variant(tmp_path, name, src):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", str(c), "-o",
                    str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    f = lib.oracle_hydro
    P, I = ctypes.c_void_p, ctypes.c_int
    f.argtypes = [I, P, P, P, P, P, P, I, P, P]
    f.restype = None
    return lib, f


def _run_variant(f, g):
    ph, ve, mass, rho = _inputs(g)
    par = np.array([g["gamma"], g["alpha"], g["beta"], g["eta"]], np.float64)
    rows = np.arange(2, dtype=np.int32)
    acc = np.empty((2, 3))
    de = np.empty(2)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    f(2, p(ph), p(ve), p(mass), p(rho), p(par), p(rows), 2, p(acc), p(de))
    return acc, de


def test_each_planted_viscosity_mistake_fails_the_pin(tmp_path):
    g = _golden()
    with open(ORACLE_C) as fh:
        src = fh.read()
    b, e = _hydro_fn_bounds(src)
    # the harness itself: the unmodified source passes
    _, f = _build_variant(tmp_path, "unmodified", src)
    acc, de = _run_variant(f, g)
    assert _rel(acc, g["acc"]) < TOL and _rel(de, g["dedt"]) < TOL
    for k, (name, old, new) in enumerate(MUTATIONS):
        body = src[b:e]
        assert body.count(old) == 1, name
        mutant = src[:b] + body.replace(old, new) + src[e:]
        _, f = _build_variant(tmp_path, f"mutant{k}", mutant)
        acc, de = _run_variant(f, g)
        # every mistake moves both outputs far outside the pin's tolerance
        assert _rel(acc, g["acc"]) > 1e-3, name
        assert _rel(de, g["dedt"]) > 1e-3, name
