"""FP64 CPU oracle for the self-gravitating SPH right-hand side of
Khrapov & Khoperskov, arXiv:1807.08116.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_1807_08116_gb300``)
and imports nothing from it.

The arithmetic lives in ``sph_oracle.c`` (plain brute-force loops, FP64); this
module compiles it with gcc, loads it through ctypes and strings the calls
together in the order of the paper's predictor-corrector scheme (Sect. 2.2,
Eqs. 12-16).  Every function takes the FP32 working copies the GPU path
consumes, promotes them exactly to FP64 and returns FP64 results.

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: kernel normalisation and C^2 continuity (Eqs. 8-9), uniform-lattice
density (Eq. 7), two-body and Plummer closed forms (Eq. 4), momentum and
energy conservation of the pairwise forms (Eqs. 10-11), a hand-worked
two-particle head-on case for the artificial viscosity (after Eq. 11),
velocity-Verlet equivalence of the scheme for dark-only runs (Eqs. 12-16),
and numpy's stable argsort / scipy's k-d tree for the binning and the
neighbour sets.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_SO = os.path.join(_HERE, "_sph_oracle.so")
_lock = threading.Lock()
_lib = None

# Physical constants of the paper's model (Sect. 2): viscosity alpha, beta,
# eta (after Eq. 11); smoothing-length factor sigma ~ 1.2-1.3 (after Eq. 8).
DEFAULTS = dict(G=1.0, eps=0.01, gamma=5.0 / 3.0, alpha=0.5, beta=1.0, eta=0.1,
                sigma=1.25)


def build(force: bool = False) -> str:
    """Compile sph_oracle.c into _sph_oracle.so (gcc, FP contraction off)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", _SO + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.oracle_threads.restype = I
            lib.oracle_threads.argtypes = []
            lib.oracle_set_threads.restype = I
            lib.oracle_set_threads.argtypes = [I]
            lib.oracle_W.restype = D
            lib.oracle_W.argtypes = [D, D]
            lib.oracle_Wp.restype = D
            lib.oracle_Wp.argtypes = [D, D]
            lib.oracle_dWp_dxi.restype = D
            lib.oracle_dWp_dxi.argtypes = [D, D]
            lib.oracle_neighbor_counts.argtypes = [I, P, P, I, P]
            lib.oracle_neighbor_lists.argtypes = [I, P, P, I, P, P]
            lib.oracle_bin.argtypes = [I, P, P, P, P, P, P]
            lib.oracle_counting_sort.argtypes = [I, P, I, P, P, P]
            lib.oracle_density.argtypes = [I, P, P, D, P, I, P, P]
            lib.oracle_hydro.argtypes = [I, P, P, P, P, P, P, I, P, P]
            lib.oracle_gravity.argtypes = [I, P, D, D, P, I, P, P]
            lib.oracle_predict.argtypes = [I, I, D, P, P, P, P, P, P, P, P]
            lib.oracle_correct.argtypes = [I, I, D, P, P, P, P, P, P, P]
            lib.oracle_cfl.restype = D
            lib.oracle_cfl.argtypes = [I, P, P, P, P, P, P, P, I, P]
            for f in ("oracle_neighbor_counts", "oracle_neighbor_lists", "oracle_bin",
                      "oracle_counting_sort", "oracle_density", "oracle_hydro",
                      "oracle_gravity", "oracle_predict", "oracle_correct"):
                getattr(lib, f).restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _rows(rows, n):
    if rows is None:
        return np.arange(n, dtype=np.int32)
    return _c(rows, np.int32)


def threads() -> int:
    """Number of host threads the oracle's parallel loops use."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> int:
    """Use n host threads in the parallel loops; returns the count in effect."""
    return int(_load().oracle_set_threads(int(n)))


# -- kernels (Eqs. 8, 9) ------------------------------------------------------

def W(xi: float, h: float) -> float:
    return _load().oracle_W(float(xi), float(h))


def Wp(xi: float, h: float) -> float:
    return _load().oracle_Wp(float(xi), float(h))


def dWp_dxi(xi: float, h: float) -> float:
    return _load().oracle_dWp_dxi(float(xi), float(h))


# -- sorting stage (Sect. 3) -------------------------------------------------

def bin_particles(pos_h, grid):
    """Level, integer cell (3) and bucket key per particle.

    grid: dict(x0, y0, z0, log2_L0, n_levels, log2_M)."""
    pos_h = _c(pos_h, np.float32)
    n = pos_h.shape[0]
    g = np.array([grid["x0"], grid["y0"], grid["z0"]], dtype=np.float32)
    ig = np.array([grid["log2_L0"], grid["n_levels"], grid["log2_M"]], dtype=np.int32)
    level = np.empty(n, np.int32)
    cell = np.empty((n, 3), np.int32)
    key = np.empty(n, np.int32)
    _load().oracle_bin(n, _p(pos_h), _p(g), _p(ig), _p(level), _p(cell), _p(key))
    return level, cell, key


def counting_sort(key, M):
    """(count[M], cell_start[M+1] exclusive, perm[n]) of a stable counting sort."""
    key = _c(key, np.int32)
    n = key.shape[0]
    count = np.empty(M, np.int32)
    start = np.empty(M + 1, np.int32)
    perm = np.empty(n, np.int32)
    _load().oracle_counting_sort(n, _p(key), int(M), _p(count), _p(start), _p(perm))
    return count, start, perm


# -- neighbour sets ----------------------------------------------------------

def neighbors(pos_h, rows=None):
    """Brute-force neighbour lists (ascending j) of the given rows: (starts, idx)."""
    pos_h = _c(pos_h, np.float32)
    n = pos_h.shape[0]
    rows = _rows(rows, n)
    counts = np.empty(rows.shape[0], np.int32)
    lib = _load()
    lib.oracle_neighbor_counts(n, _p(pos_h), _p(rows), rows.shape[0], _p(counts))
    starts = np.zeros(rows.shape[0] + 1, np.int64)
    np.cumsum(counts, out=starts[1:])
    idx = np.empty(int(starts[-1]), np.int32)
    lib.oracle_neighbor_lists(n, _p(pos_h), _p(rows), rows.shape[0], _p(starts), _p(idx))
    return starts, idx


# -- density, hydro forces, gravity ------------------------------------------

def density(pos_h, mass, sigma=DEFAULTS["sigma"], rows=None):
    pos_h = _c(pos_h, np.float32)
    mass = _c(mass, np.float32)
    n = pos_h.shape[0]
    rows = _rows(rows, n)
    rho = np.empty(rows.shape[0], np.float64)
    hn = np.empty(rows.shape[0], np.float64)
    _load().oracle_density(n, _p(pos_h), _p(mass), float(sigma), _p(rows), rows.shape[0],
                           _p(rho), _p(hn))
    return rho, hn


def hydro(pos_h, vel_e, mass, rho, gamma=DEFAULTS["gamma"], alpha=DEFAULTS["alpha"],
          beta=DEFAULTS["beta"], eta=DEFAULTS["eta"], rows=None):
    pos_h = _c(pos_h, np.float32)
    vel_e = _c(vel_e, np.float32)
    mass = _c(mass, np.float32)
    rho = _c(rho, np.float32)
    n = pos_h.shape[0]
    rows = _rows(rows, n)
    par = np.array([gamma, alpha, beta, eta], np.float64)
    acc = np.empty((rows.shape[0], 3), np.float64)
    de = np.empty(rows.shape[0], np.float64)
    _load().oracle_hydro(n, _p(pos_h), _p(vel_e), _p(mass), _p(rho), _p(par), _p(rows),
                         rows.shape[0], _p(acc), _p(de))
    return acc, de


def gravity(pos_m, G=DEFAULTS["G"], eps=DEFAULTS["eps"], rows=None):
    pos_m = _c(pos_m, np.float32)
    n = pos_m.shape[0]
    rows = _rows(rows, n)
    acc = np.empty((rows.shape[0], 3), np.float64)
    pot = np.empty(rows.shape[0], np.float64)
    _load().oracle_gravity(n, _p(pos_m), float(G), float(eps), _p(rows), rows.shape[0],
                           _p(acc), _p(pot))
    return acc, pot


def cfl_dt(pos_h, vel_e, rho, Q, E, C=0.5, gamma=DEFAULTS["gamma"], alpha=DEFAULTS["alpha"],
           beta=DEFAULTS["beta"], eta=DEFAULTS["eta"], rows=None):
    """Time step of Eq. 17: (min over rows, per-row bound).  Q: total
    acceleration [n, 3]; E: de/dt [n]."""
    pos_h = _c(pos_h, np.float32)
    vel_e = _c(vel_e, np.float32)
    rho = _c(rho, np.float32)
    n = pos_h.shape[0]
    rows = _rows(rows, n)
    par = np.array([gamma, alpha, beta, eta, C], np.float64)
    dt_row = np.empty(rows.shape[0], np.float64)
    dt = _load().oracle_cfl(n, _p(pos_h), _p(vel_e), _p(rho), _p(_c(Q, np.float64)),
                            _p(_c(E, np.float64)), _p(par), _p(rows), rows.shape[0], _p(dt_row))
    return dt, dt_row


# -- integrator ---------------------------------------------------------------

def predict(n_gas, dt, r, v, e, v_save, e_save, a_hyd, dedt, grav):
    """In-place predictor (Eqs. 12-14) on SoA FP64 arrays r[3,n], v[3,n], e[n_gas]."""
    n = r.shape[1]
    _load().oracle_predict(n, n_gas, float(dt), _p(r), _p(v), _p(e), _p(v_save), _p(e_save),
                           _p(_c(a_hyd, np.float64)), _p(_c(dedt, np.float64)),
                           _p(_c(grav, np.float64)))


def correct(n_gas, dt, v, e, v_save, e_save, a_hyd, dedt, grav):
    """In-place corrector (Eqs. 15-16)."""
    n = v.shape[1]
    _load().oracle_correct(n, n_gas, float(dt), _p(v), _p(e), _p(v_save), _p(e_save),
                           _p(_c(a_hyd, np.float64)), _p(_c(dedt, np.float64)),
                           _p(_c(grav, np.float64)))


# -- the whole scheme -----------------------------------------------------------

class OracleSim:
    """The predictor-corrector scheme of Sect. 2.2 on one simulation, FP64.

    State: r, v (FP64 [3, n]), e (FP64 [n_gas]), masses (FP32), smoothing
    lengths (FP32, gas).  Each right-hand-side evaluation reads FP32 working
    copies of r, h, v, e and rho, the precision the GPU path stores them in,
    and computes in FP64.  Gas particles are indices [0, n_gas).

    Order of one step (Eqs. 12-16; gravity once per step, reading R8; the
    smoothing length of the previous density evaluation, reading R7):
      hydro at (r_n, v_n, e_n)          [skipped right after the first RHS]
      predictor -> v~, e~, r_{n+1}
      density at r_{n+1} -> rho, next h
      gravity at r_{n+1}
      hydro at (r_{n+1}, v~, e~)
      corrector -> v_{n+1}, e_{n+1}
    """

    def __init__(self, r, v, e, mass, h, n_gas, **params):
        self.p = dict(DEFAULTS)
        self.p.update(params)
        self.r = np.array(r, np.float64, order="C").reshape(3, -1).copy()
        self.v = np.array(v, np.float64, order="C").reshape(3, -1).copy()
        self.n = self.r.shape[1]
        self.n_gas = int(n_gas)
        self.e = np.array(e, np.float64).copy()
        self.m = np.array(mass, np.float32).copy()
        self.h_eval = np.array(h, np.float32).copy()
        self.h_state = self.h_eval.copy()
        self.v_save = np.zeros_like(self.v)
        self.e_save = np.zeros_like(self.e)
        self.rho = None
        self.grav = None
        self.pot = None
        self.a_hyd = np.zeros((self.n_gas, 3))
        self.dedt = np.zeros(self.n_gas)
        self.fresh = False

    # FP32 working copies
    def pos_h(self):
        ph = np.empty((self.n_gas, 4), np.float32)
        ph[:, :3] = self.r[:, :self.n_gas].T
        ph[:, 3] = self.h_eval
        return ph

    def pos_m(self):
        pm = np.empty((self.n, 4), np.float32)
        pm[:, :3] = self.r.T
        pm[:, 3] = self.m
        return pm

    def vel_e(self):
        ve = np.empty((self.n_gas, 4), np.float32)
        ve[:, :3] = self.v[:, :self.n_gas].T
        ve[:, 3] = self.e
        return ve

    def _density(self):
        if self.n_gas == 0:
            self.rho = np.zeros(0)
            return
        rho, hn = density(self.pos_h(), self.m[:self.n_gas], self.p["sigma"])
        self.rho = rho
        self.h_state = hn.astype(np.float32)

    def _gravity(self):
        acc, pot = gravity(self.pos_m(), self.p["G"], self.p["eps"])
        self.grav = acc
        self.pot = pot

    def _hydro(self):
        if self.n_gas == 0:
            return
        acc, de = hydro(self.pos_h(), self.vel_e(), self.m[:self.n_gas],
                        self.rho.astype(np.float32), self.p["gamma"], self.p["alpha"],
                        self.p["beta"], self.p["eta"])
        self.a_hyd = acc
        self.dedt = de

    def initial_rhs(self):
        """First right-hand-side evaluation at t = 0."""
        self._density()
        self._gravity()
        self._hydro()
        self.fresh = True

    def step(self, dt):
        if self.rho is None:
            self.initial_rhs()
        if not self.fresh:
            self._hydro()
        predict(self.n_gas, dt, self.r, self.v, self.e, self.v_save, self.e_save,
                self.a_hyd, self.dedt, self.grav)
        self.h_eval = self.h_state.copy()
        self._density()
        self._gravity()
        self._hydro()
        correct(self.n_gas, dt, self.v, self.e, self.v_save, self.e_save,
                self.a_hyd, self.dedt, self.grav)
        self.fresh = False

    def energies(self):
        """(kinetic, thermal, potential) in FP64; potential from the last gravity."""
        m = self.m.astype(np.float64)
        kin = 0.5 * float(np.sum(m * np.sum(self.v * self.v, axis=0)))
        th = float(np.sum(m[:self.n_gas] * self.e))
        pot = 0.5 * float(np.sum(m * self.pot)) if self.pot is not None else float("nan")
        return kin, th, pot
