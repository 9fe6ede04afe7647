"""Seeded synthetic initial conditions: Plummer halos of gas + dark particles.

This module is an input generator only.  It holds none of the SPH method's
arithmetic (no kernels, forces or integrator); the CUDA path and the CPU
oracle both read the arrays it returns.

The paper's own galaxy models (a quasi-isothermal dark halo and a King bulge,
Sect. 2.1) are not specified in enough detail to rebuild, so Plummer spheres
stand in for them, with the particle counts and the gas / dark split of the
paper's runs (Sect. 4: N_g = N_h = N/2, N from 2^18 to 2^23; galaxy
collisions, Sect. 2.1).

Units: G = M = a = 1 per halo unless overridden.

Recipe (one halo of total mass M, scale a, n_gas gas + n_dark dark particles):
  * radius by inverse transform of the Plummer cumulative mass
    M(<r)/M = r^3 / (r^2 + a^2)^(3/2), the uniform variate truncated at 0.999
    so no particle is drawn beyond r ~ 38.7 a (Aarseth, Henon & Wielen 1974);
  * isotropic direction;
  * dark particles: speed q * v_esc(r), v_esc = sqrt(2 G M) (r^2 + a^2)^(-1/4),
    q drawn by rejection from g(q) = q^2 (1 - q^2)^(7/2) (same reference);
  * gas particles: at rest in the halo frame, with the uniform specific
    internal energy of an isothermal gas in virial equilibrium in the total
    Plummer potential, p/rho = pi G M / (32 a), e = (p/rho) / (gamma - 1);
  * initial smoothing length h = sigma (m / rho_gas(r))^(1/3) from the
    analytic gas density rho_gas = (M_gas/M) 3M/(4 pi a^3) (1 + r^2/a^2)^(-5/2);
  * equal masses m = M / (n_gas + n_dark).

Two-halo collision: centres offset by (10 a, 2 a, 0) (10 a along the motion,
impact parameter 2 a), closing speed v_rel = 1.5 * sqrt(2 G (2M) / d0),
d0 = |offset|, split equally in the centre-of-mass frame.

Particle order in every returned array: all gas first (halo A then halo B),
then all dark (halo A then halo B).  Random streams: numpy PCG64 seeded from
SeedSequence(seed).spawn(#halos), one stream per halo.
"""
from __future__ import annotations

import math

import numpy as np

MFRAC_MAX = 0.999


def _plummer_radii(rng, n, a):
    x = rng.uniform(0.0, MFRAC_MAX, size=n)
    x = np.maximum(x, 1e-300)
    return a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)


def _isotropic(rng, n):
    cth = rng.uniform(-1.0, 1.0, size=n)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def _speed_fraction(rng, n):
    out = np.empty(n)
    filled = 0
    while filled < n:
        m = 2 * (n - filled) + 64
        q = rng.uniform(0.0, 1.0, size=m)
        y = rng.uniform(0.0, 0.1, size=m)
        ok = y < q * q * (1.0 - q * q) ** 3.5
        take = q[ok][: n - filled]
        out[filled:filled + take.shape[0]] = take
        filled += take.shape[0]
    return out


def plummer_halo(rng, n_gas, n_dark, M=1.0, a=1.0, G=1.0, gamma=5.0 / 3.0, sigma=1.25):
    """One Plummer halo at the origin, at rest.  Returns a dict of FP64 arrays
    (r [n,3], v [n,3], e [n_gas], h [n_gas]) and FP32 masses m [n]."""
    n = n_gas + n_dark
    m = M / n
    r_gas = _plummer_radii(rng, n_gas, a)
    x_gas = _isotropic(rng, n_gas) * r_gas[:, None]
    r_dark = _plummer_radii(rng, n_dark, a)
    x_dark = _isotropic(rng, n_dark) * r_dark[:, None]
    vesc = math.sqrt(2.0 * G * M) * (r_dark * r_dark + a * a) ** -0.25
    v_dark = _isotropic(rng, n_dark) * (_speed_fraction(rng, n_dark) * vesc)[:, None]

    p_over_rho = math.pi * G * M / (32.0 * a)
    e = np.full(n_gas, p_over_rho / (gamma - 1.0))
    m_gas_frac = n_gas / n if n else 0.0
    rho_gas = m_gas_frac * 3.0 * M / (4.0 * math.pi * a ** 3) * (1.0 + (r_gas / a) ** 2) ** -2.5
    h = sigma * np.cbrt(m / rho_gas) if n_gas else np.zeros(0)

    return dict(
        r_gas=x_gas, v_gas=np.zeros_like(x_gas), r_dark=x_dark, v_dark=v_dark,
        e=e, h=h, m=m,
    )


def _assemble(halos, offsets, velocities):
    rg, vg, rd, vd, e, h, mg, md = [], [], [], [], [], [], [], []
    for hl, off, vel in zip(halos, offsets, velocities):
        rg.append(hl["r_gas"] + off)
        vg.append(hl["v_gas"] + vel)
        rd.append(hl["r_dark"] + off)
        vd.append(hl["v_dark"] + vel)
        e.append(hl["e"])
        h.append(hl["h"])
        mg.append(np.full(hl["r_gas"].shape[0], hl["m"]))
        md.append(np.full(hl["r_dark"].shape[0], hl["m"]))
    r = np.concatenate(rg + rd, axis=0)
    v = np.concatenate(vg + vd, axis=0)
    n_gas = sum(x.shape[0] for x in rg)
    return dict(
        r=np.ascontiguousarray(r, np.float64),
        v=np.ascontiguousarray(v, np.float64),
        e=np.concatenate(e).astype(np.float64),
        h=np.concatenate(h).astype(np.float32),
        m=np.concatenate(mg + md).astype(np.float32),
        n_gas=n_gas,
        n=r.shape[0],
    )


def single_halo(n_gas, n_dark, seed=0, **kw):
    """One halo at rest at the origin (the 8192 + 8192 single-halo workload)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed).spawn(1)[0]))
    hl = plummer_halo(rng, n_gas, n_dark, **kw)
    return _assemble([hl], [np.zeros(3)], [np.zeros(3)])


def two_halo(n_gas_each, n_dark_each, seed=1, dx=10.0, b=2.0, speed_factor=1.5,
             M=1.0, a=1.0, G=1.0, **kw):
    """Two equal Plummer halos on a collision course (see module docstring)."""
    ss = np.random.SeedSequence(seed).spawn(2)
    halos = [plummer_halo(np.random.Generator(np.random.PCG64(s)), n_gas_each, n_dark_each,
                          M=M, a=a, G=G, **kw) for s in ss]
    off = np.array([dx * a, b * a, 0.0])
    d0 = float(np.linalg.norm(off))
    v_rel = speed_factor * math.sqrt(2.0 * G * (2.0 * M) / d0)
    offsets = [-0.5 * off, 0.5 * off]
    velocities = [np.array([0.5 * v_rel, 0.0, 0.0]), np.array([-0.5 * v_rel, 0.0, 0.0])]
    return _assemble(halos, offsets, velocities)


def ensemble_params(n_sims=64, seed=3, n_min=8192, n_max=262144):
    """Per-simulation (n_total, impact parameter b, speed factor, seed) of the
    batched ensemble: sizes log-uniform in [n_min, n_max] (rounded to a
    multiple of 4 so each halo has equal gas and dark counts), b ~ U[0, 4a],
    speed ~ U[0.5, 2] x escape."""
    rng = np.random.Generator(np.random.PCG64(seed))
    logn = rng.uniform(math.log(n_min), math.log(n_max), size=n_sims)
    n = (np.exp(logn) / 4.0).round().astype(np.int64) * 4
    b = rng.uniform(0.0, 4.0, size=n_sims)
    sp = rng.uniform(0.5, 2.0, size=n_sims)
    seeds = rng.integers(0, 2 ** 31 - 1, size=n_sims)
    return [dict(n=int(n[i]), b=float(b[i]), speed_factor=float(sp[i]), seed=int(seeds[i]))
            for i in range(n_sims)]


def from_params(n, b, speed_factor, seed):
    """Two-halo IC of total particle count n (n/4 gas + n/4 dark per halo)."""
    q = n // 4
    return two_halo(q, q, seed=seed, b=b, speed_factor=speed_factor)


def serving_trace(n_jobs=200, rate=20.0, seed=4, n_min=4096, n_max=1048576,
                  steps_min=10, steps_max=1000):
    """Poisson arrivals (rate per second) of two-halo jobs; sizes log-uniform,
    step counts uniform in [steps_min, steps_max]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n_jobs)
    t = np.cumsum(gaps)
    logn = rng.uniform(math.log(n_min), math.log(n_max), size=n_jobs)
    n = (np.exp(logn) / 4.0).round().astype(np.int64) * 4
    steps = rng.integers(steps_min, steps_max + 1, size=n_jobs)
    b = rng.uniform(0.0, 4.0, size=n_jobs)
    sp = rng.uniform(0.5, 2.0, size=n_jobs)
    seeds = rng.integers(0, 2 ** 31 - 1, size=n_jobs)
    return [dict(t=float(t[i]), n=int(n[i]), steps=int(steps[i]), b=float(b[i]),
                 speed_factor=float(sp[i]), seed=int(seeds[i])) for i in range(n_jobs)]
