"""ctypes binding of libsphgb.so (C ABI in include/sphgb.h).

Argument marshalling only: every function takes torch CUDA tensors (or
None), checks dtype / shape / contiguity, and forwards raw device pointers and
the current CUDA stream to the C function of the same name.  All arithmetic
runs in the library's kernels; there is no fallback path: if the library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsphgb.so")

SPH_OK = 0
SPH_ERR_INVALID_ARG = 1
SPH_ERR_CUDA = 2
SPH_ERR_NB_OVERFLOW = 3
SPH_ERR_BUDGET = 4
SPH_ERR_TIMEOUT = 5
SPH_ERR_NOT_FOUND = 6
SPH_ERR_DEVICE = 7

SPH_FLAG_NB_OVERFLOW = 1
SPH_FLAG_SEARCH_WIDE = 2
SPH_FLAG_TIMEOUT = 4
SPH_FLAG_ROW_UNSORTED = 8
SPH_FLAG_GRAV_RANGE = 16

SPH_GRAV_POTENTIAL = 1
SPH_GRAV_NO_KAHAN = 2

SPH_PREDICT, SPH_CORRECT, SPH_EMIT = 0, 1, 2
SPH_SERVE_FIFO, SPH_SERVE_SHORTEST_FIRST = 0, 1

_ERR_NAMES = {1: "INVALID_ARG", 2: "CUDA_ERROR", 3: "NB_OVERFLOW", 4: "BUDGET", 5: "TIMEOUT",
              6: "NOT_FOUND", 7: "DEVICE_ERROR"}


class SphError(RuntimeError):
    def __init__(self, fn, code, extra=""):
        super().__init__(f"{fn} failed: {_ERR_NAMES.get(code, code)} {extra}".strip())
        self.code = code


class SphParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("G", "eps", "gamma", "alpha", "beta", "eta", "sigma")]


class SphGrid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_float), ("y0", ctypes.c_float), ("z0", ctypes.c_float),
                ("log2_L0", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("log2_M", ctypes.c_int32)]


class SphState(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_gas", ctypes.c_int32)] + [
        (k, ctypes.c_void_p) for k in ("r", "v", "e", "v_save", "e_save", "mass", "h", "pos_m",
                                       "pos_h", "vel_e", "rho", "acc_hyd", "grav")] + [
        ("fresh", ctypes.c_int32), ("grav_flags", ctypes.c_int32), ("events", ctypes.c_void_p),
        ("grav_work", ctypes.c_void_p), ("grav_work_bytes", ctypes.c_size_t)]

class SimRequest(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_gas", ctypes.c_int32), ("n_steps", ctypes.c_int32),
                ("dt", ctypes.c_double)] + [(k, ctypes.c_void_p) for k in
                                            ("h_r", "h_v", "h_e", "h_m", "h_h")]


class SimStatus(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("state", "error", "n", "n_gas", "n_steps",
                                              "steps_done")] + [
        (k, ctypes.c_double) for k in ("submit_s", "admit_s", "done_s", "step_ms_p50",
                                       "step_ms_p99")] + [
        (k, ctypes.c_void_p) for k in ("h_r", "h_v", "h_e")]


class SphServerInfo(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int32), ("resident", ctypes.c_int32),
                ("arena_bytes", ctypes.c_size_t), ("arena_free_bytes", ctypes.c_size_t)]


SIM_QUEUED, SIM_RUNNING, SIM_DONE, SIM_FAILED = 0, 1, 2, 3

STAGES = ("hfc_pred", "su_pred", "sp", "nb", "dc", "gfc", "hfc_corr", "su_corr")


DEFAULT_PARAMS = dict(G=1.0, eps=0.01, gamma=5.0 / 3.0, alpha=0.5, beta=1.0, eta=0.1, sigma=1.25)

_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I = ctypes.c_int32
_I64 = ctypes.c_int64


def lib():
    """Load libsphgb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                               "(or python -m paper_1807_08116_gb300.build) first")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "sph_version": (_I, []),
            "sph_ctx_workspace_bytes": (ctypes.c_size_t, [_I, _I, _I64]),
            "sph_ctx_create": (_I, [ctypes.POINTER(SphParams), _I, _I, _I64, _P, ctypes.c_size_t, _P,
                                    ctypes.POINTER(_P)]),
            "sph_ctx_destroy": (_I, [_P]),
            "sph_ctx_set_params": (_I, [_P, ctypes.POINTER(SphParams)]),
            "sph_ctx_set_lanes": (_I, [_P, _I]),
            "sph_ctx_set_sort_fused": (_I, [_P, _I]),
            "sph_ctx_set_grid_shift": (_I, [_P, _I]),
            "pp_gravity_pairs_plan": (_I, [_I, _I, _I]),
            "pp_gravity_pairs_get_plan": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                               ctypes.POINTER(_I)]),
            "sph_ctx_device_status": (_I, [_P, _P, ctypes.POINTER(_I)]),
            "sph_ctx_get_grid": (_I, [_P, _P, ctypes.POINTER(SphGrid)]),
            "sph_ctx_nb_total": (_I, [_P, _P, ctypes.POINTER(_I64)]),
            "sph_bin_and_sort": (_I, [_P, _P, _I, ctypes.POINTER(SphGrid), _P, _P, _P, _P]),
            "sph_build_neighbors": (_I, [_P, _I, _P, _P, _I64, ctypes.POINTER(_I64), _P]),
            "sph_density": (_I, [_P, _I, _P, _P, _P, _P]),
            "sph_forces": (_I, [_P, _I, _P, _P, _P, _P, _P]),
            "sph_cfl_dt": (_I, [_P, _I, _P, _P, _P, _P, _P, ctypes.c_float, _P, _P, _P]),
            "pp_gravity": (_I, [_P, _I, ctypes.c_float, ctypes.c_float, _P, _I, _P]),
            "pp_gravity_status": (_I, [_P, ctypes.POINTER(_I)]),
            "pp_gravity_rows": (_I, [_P, _I, _I, _I, ctypes.c_float, ctypes.c_float, _P, _I, _P]),
            "sph_set_wait_limit_ns": (_I, [_I64]),
            "sph_wait_probe": (_I, [_P]),
            "pp_gravity_pairs": (_I, [_P, _I, ctypes.c_float, ctypes.c_float, _P, _I, _P,
                                      ctypes.c_size_t, _P]),
            "pp_gravity_pairs_workspace_bytes": (ctypes.c_size_t, [_I]),
            "pp_gravity_pairs_eligible": (_I, [_I, ctypes.c_float, _I]),
            "pp_gravity_pairs_min_n": (_I, [_I]),
            "pp_gravity_pairs_batched": (_I, [_P, _P, ctypes.c_float, ctypes.c_float, _P, _I, _P,
                                              ctypes.c_size_t, _P]),
            "sph_gravity_plan": (_I, [_I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
            "sph_gravity_tune": (_I, [_I, _I]),
            "integrate_step": (_I, [_I, ctypes.c_double, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                    _P, _P, _P, _P]),
            "sph_rhs_initial": (_I, [_P, ctypes.POINTER(SphState), _P]),
            "sph_step": (_I, [_P, ctypes.POINTER(SphState), ctypes.c_double, _P]),
            "sph_step_cfl": (_I, [_P, ctypes.POINTER(SphState), ctypes.c_float, ctypes.c_float, _P,
                                  _P]),
            "sph_forces_cfl": (_I, [_P, _I, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float, _P,
                                    _P, _P]),
            "sph_diagnostics": (_I, [ctypes.POINTER(SphState), _P, _P]),
            "sph_events_create": (_I, [_I, _P]),
            "sph_events_destroy": (_I, [_I, _P]),
            "sph_event_elapsed_ms": (_I, [_P, _P, ctypes.POINTER(ctypes.c_float)]),
            "sph_launch_count": (ctypes.c_int64, []),
            "sph_batch_workspace_bytes": (ctypes.c_size_t, [_I, _P, _P]),
            "sph_batch_create": (_I, [_I, _P, _P, _P, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
            "sph_batch_destroy": (_I, [_P]),
            "sph_batch_set_plan": (_I, [_P, _I, _P]),
            "pp_gravity_batched": (_I, [_P, _P, ctypes.c_float, ctypes.c_float, _P, _I, _P]),
            "sph_ctx_set_batch": (_I, [_P, _P]),
            "sph_server_create": (_I, [ctypes.POINTER(SphParams), _P, ctypes.c_size_t, _I, _I,
                                       ctypes.POINTER(_P)]),
            "sph_server_destroy": (_I, [_P]),
            "sim_submit": (_I, [_P, ctypes.POINTER(SimRequest), ctypes.POINTER(ctypes.c_uint64)]),
            "sph_server_step": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]),
            "sim_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(SimStatus)]),
            "sim_release": (_I, [_P, ctypes.c_uint64]),
            "sph_server_info": (_I, [_P, ctypes.POINTER(SphServerInfo)]),
            "sph_server_step_times": (_I, [_P, _P, _I, ctypes.POINTER(_I)]),
            "sph_server_set_policy": (_I, [_P, _I]),
            "sim_checkpoint": (_I, [_P, ctypes.c_uint64, _P, _P, _P, _P, ctypes.POINTER(_I)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


def _check(fn, rc, extra=""):
    if rc != SPH_OK:
        raise SphError(fn, rc, extra)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype, shape=None, name="tensor", allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def params_struct(**kw):
    p = dict(DEFAULT_PARAMS)
    p.update({k: v for k, v in kw.items() if k in DEFAULT_PARAMS})
    return SphParams(**{k: float(v) for k, v in p.items()})


# ---------------------------------------------------------------------------
# Context
# ---------------------------------------------------------------------------

def sph_ctx_workspace_bytes(n_gas_max, log2_M, nb_capacity):
    return int(lib().sph_ctx_workspace_bytes(int(n_gas_max), int(log2_M), int(nb_capacity)))


def default_log2_M(n_gas):
    """2^log2_M >= 2 n_gas buckets (at least 2^10)."""
    m = 10
    while (1 << m) < 2 * max(1, n_gas):
        m += 1
    return m


class Ctx:
    """A context: host handle plus its device workspace (a torch uint8 tensor)."""

    def __init__(self, n_gas_max, nb_capacity, log2_M=None, device=None, stream=None, **params):
        self.n_gas_max = int(n_gas_max)
        self.log2_M = int(log2_M if log2_M is not None else default_log2_M(n_gas_max))
        self.capacity = int(nb_capacity)
        self.params = params_struct(**params)
        nbytes = sph_ctx_workspace_bytes(self.n_gas_max, self.log2_M, self.capacity)
        if nbytes == 0:
            raise SphError("sph_ctx_workspace_bytes", SPH_ERR_INVALID_ARG)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_ptr = self.workspace.data_ptr() + off
        h = ctypes.c_void_p()
        rc = lib().sph_ctx_create(ctypes.byref(self.params), self.n_gas_max, self.log2_M,
                                  self.capacity, ctypes.c_void_p(self._ws_ptr), nbytes,
                                  _stream(stream), ctypes.byref(h))
        _check("sph_ctx_create", rc)
        self.handle = h

    @property
    def M(self):
        return 1 << self.log2_M

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().sph_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_lanes(self, lanes):
        """Lanes per neighbour row in the density / force kernels (1, 2, 4, 8)."""
        _check("sph_ctx_set_lanes", lib().sph_ctx_set_lanes(self.handle, int(lanes)))
        self.lanes = int(lanes)

    def set_sort_fused(self, fused):
        """1: the sorting stage as one cooperative launch (default); 0: as a
        sequence of kernels (the same results)."""
        _check("sph_ctx_set_sort_fused", lib().sph_ctx_set_sort_fused(self.handle, int(fused)))

    def set_grid_shift(self, shift):
        """Octaves added to the finest cell size of the derived grid."""
        _check("sph_ctx_set_grid_shift", lib().sph_ctx_set_grid_shift(self.handle, int(shift)))
        self.grid_shift = int(shift)

    def device_status(self, stream=None):
        f = _I()
        rc = lib().sph_ctx_device_status(self.handle, _stream(stream), ctypes.byref(f))
        if rc not in (SPH_OK, SPH_ERR_DEVICE):
            _check("sph_ctx_device_status", rc)
        return int(f.value)

    def grid(self, stream=None):
        g = SphGrid()
        _check("sph_ctx_get_grid", lib().sph_ctx_get_grid(self.handle, _stream(stream), ctypes.byref(g)))
        return dict(x0=g.x0, y0=g.y0, z0=g.z0, log2_L0=g.log2_L0, n_levels=g.n_levels,
                    log2_M=g.log2_M)

    def nb_total(self, stream=None):
        t = _I64()
        _check("sph_ctx_nb_total", lib().sph_ctx_nb_total(self.handle, _stream(stream), ctypes.byref(t)))
        return int(t.value)


def _grid_struct(grid):
    if grid is None:
        return None
    return ctypes.byref(SphGrid(float(grid["x0"]), float(grid["y0"]), float(grid["z0"]),
                                int(grid["log2_L0"]), int(grid["n_levels"]), int(grid["log2_M"])))


# ---------------------------------------------------------------------------
# Stage calls
# ---------------------------------------------------------------------------

def sph_bin_and_sort(ctx, pos_h, grid=None, key=None, cell_start=None, perm=None, stream=None):
    n = pos_h.shape[0]
    rc = lib().sph_bin_and_sort(
        ctx.handle, _ptr(pos_h, torch.float32, (n, 4), "pos_h"), n, _grid_struct(grid),
        _ptr(key, torch.int32, (n,), "key", True), _ptr(cell_start, torch.int32, (ctx.M + 1,),
                                                          "cell_start", True),
        _ptr(perm, torch.int32, (n,), "perm", True), _stream(stream))
    _check("sph_bin_and_sort", rc)


def sph_build_neighbors(ctx, n_gas, nb_start=None, nb_idx=None, want_needed=True, stream=None):
    """Returns the total list length (if want_needed) or None."""
    needed = _I64(-1)
    cap = 0 if nb_idx is None else nb_idx.numel()
    rc = lib().sph_build_neighbors(
        ctx.handle, int(n_gas), _ptr(nb_start, torch.int32, (n_gas + 1,), "nb_start", True),
        _ptr(nb_idx, torch.int32, None, "nb_idx", True), cap,
        ctypes.byref(needed) if want_needed else None, _stream(stream))
    _check("sph_build_neighbors", rc, f"(needed {needed.value}, capacity {ctx.capacity})")
    return int(needed.value) if want_needed else None


def sph_density(ctx, mass, rho, h_next, stream=None):
    n = mass.shape[0]
    rc = lib().sph_density(ctx.handle, n, _ptr(mass, torch.float32, (n,), "mass"),
                           _ptr(rho, torch.float32, (n,), "rho"),
                           _ptr(h_next, torch.float32, (n,), "h_next"), _stream(stream))
    _check("sph_density", rc)


def sph_forces(ctx, vel_e, rho, mass, acc_dedt, stream=None):
    n = vel_e.shape[0]
    rc = lib().sph_forces(ctx.handle, n, _ptr(vel_e, torch.float32, (n, 4), "vel_e"),
                          _ptr(rho, torch.float32, (n,), "rho"),
                          _ptr(mass, torch.float32, (n,), "mass"),
                          _ptr(acc_dedt, torch.float32, (n, 4), "acc_dedt"), _stream(stream))
    _check("sph_forces", rc)


def sph_cfl_dt(ctx, vel_e, rho, mass, acc_hyd, grav, C, dt_min, dt_particle=None, stream=None):
    """Eq. 17 time step; grav may hold more rows than the gas (a state's grav)."""
    n = vel_e.shape[0]
    if grav.shape[0] < n or tuple(grav.shape[1:]) != (4,):
        raise ValueError("grav must have at least n_gas rows of 4")
    rc = lib().sph_cfl_dt(ctx.handle, n, _ptr(vel_e, torch.float32, (n, 4), "vel_e"),
                          _ptr(rho, torch.float32, (n,), "rho"),
                          _ptr(mass, torch.float32, (n,), "mass"),
                          _ptr(acc_hyd, torch.float32, (n, 4), "acc_hyd"),
                          _ptr(grav, torch.float32, None, "grav"), float(C),
                          _ptr(dt_particle, torch.float32, (n,), "dt_particle", True),
                          _ptr(dt_min, torch.float32, (1,), "dt_min"), _stream(stream))
    _check("sph_cfl_dt", rc)


def pp_gravity(pos_m, acc_pot, G=1.0, eps=0.01, flags=0, stream=None):
    n = pos_m.shape[0]
    rc = lib().pp_gravity(_ptr(pos_m, torch.float32, (n, 4), "pos_m"), n, float(G), float(eps),
                          _ptr(acc_pot, torch.float32, (n, 4), "acc_pot"), int(flags),
                          _stream(stream))
    _check("pp_gravity", rc)


def pp_gravity_rows(pos_m, i0, i1, acc_pot, G=1.0, eps=0.01, flags=0, stream=None):
    """Gravity of the targets [i0, i1) over all sources of pos_m [n, 4] into
    acc_pot [i1 - i0, 4]."""
    n = pos_m.shape[0]
    _check("pp_gravity_rows", lib().pp_gravity_rows(
        _ptr(pos_m, torch.float32, (n, 4), "pos_m"), n, int(i0), int(i1), float(G), float(eps),
        _ptr(acc_pot, torch.float32, (int(i1) - int(i0), 4), "acc_pot"), int(flags), _stream(stream)))


def pp_gravity_pairs_workspace_bytes(n):
    return int(lib().pp_gravity_pairs_workspace_bytes(int(n)))


def pp_gravity_pairs_workspace(n, device="cuda"):
    """A scratch tensor for pp_gravity_pairs over n bodies (256-byte aligned)."""
    nbytes = pp_gravity_pairs_workspace_bytes(n)
    return torch.empty((nbytes + 255) // 256 * 256, dtype=torch.uint8, device=device)


def pp_gravity_pairs(pos_m, acc_pot, work, G=1.0, eps=0.01, flags=0, stream=None):
    """Gravity with every pair evaluated once (falls back to pp_gravity when not
    eligible or `work` is None / too small)."""
    n = pos_m.shape[0]
    wp, wb = (None, 0) if work is None else (work.data_ptr(), work.numel() * work.element_size())
    if work is not None and (not work.is_cuda or not work.is_contiguous()):
        raise ValueError("work: contiguous CUDA tensor expected")
    rc = lib().pp_gravity_pairs(_ptr(pos_m, torch.float32, (n, 4), "pos_m"), n, float(G),
                                float(eps), _ptr(acc_pot, torch.float32, (n, 4), "acc_pot"),
                                int(flags), wp, wb, _stream(stream))
    _check("pp_gravity_pairs", rc)


def pp_gravity_pairs_plan(threads=0, R=8, super_log2=-1):
    """Fix the launch plan of the single-simulation pair-once kernel
    (threads=0: the default)."""
    _check("pp_gravity_pairs_plan", lib().pp_gravity_pairs_plan(int(threads), int(R), int(super_log2)))


def pp_gravity_pairs_get_plan(n):
    """(threads, R, super_log2) pp_gravity_pairs uses for n bodies."""
    t, r, lg = _I(), _I(), _I()
    _check("pp_gravity_pairs_get_plan", lib().pp_gravity_pairs_get_plan(int(n), ctypes.byref(t),
                                                                        ctypes.byref(r), ctypes.byref(lg)))
    return int(t.value), int(r.value), int(lg.value)


def pp_gravity_pairs_eligible(n, eps=0.01, flags=0):
    return bool(lib().pp_gravity_pairs_eligible(int(n), float(eps), int(flags)))


def pp_gravity_pairs_min_n(n_min=0):
    """Smallest n for the pair-once kernel (0: default)."""
    _check("pp_gravity_pairs_min_n", lib().pp_gravity_pairs_min_n(int(n_min)))


def pp_gravity_status(stream=None):
    f = _I()
    rc = lib().pp_gravity_status(_stream(stream), ctypes.byref(f))
    if rc not in (SPH_OK, SPH_ERR_DEVICE):
        _check("pp_gravity_status", rc)
    return int(f.value)


def sph_set_wait_limit_ns(limit_ns=0):
    """Time limit of the gravity kernels' bounded waits (0: the default 2 s)."""
    _check("sph_set_wait_limit_ns", lib().sph_set_wait_limit_ns(int(limit_ns)))


def sph_wait_probe(stream=None):
    """Launch the probe whose bounded wait runs out (sets SPH_FLAG_TIMEOUT)."""
    _check("sph_wait_probe", lib().sph_wait_probe(_stream(stream)))


def sph_gravity_plan(n, flags=0):
    R, S = _I(), _I()
    _check("sph_gravity_plan", lib().sph_gravity_plan(int(n), int(flags), ctypes.byref(R),
                                                      ctypes.byref(S)))
    return int(R.value), int(S.value)


def sph_gravity_tune(R=0, S=1):
    """Force the gravity launch plan (R targets per thread, S-CTA clusters); R=0: automatic."""
    _check("sph_gravity_tune", lib().sph_gravity_tune(int(R), int(S)))


def integrate_step(phase, dt, n, n_gas, r, v, e, v_save, e_save, acc_hyd, grav, mass, h,
                   pos_m=None, pos_h=None, vel_e=None, stream=None):
    f64, f32 = torch.float64, torch.float32
    emit = phase == SPH_EMIT
    rc = lib().integrate_step(
        int(phase), float(dt), int(n), int(n_gas),
        _ptr(r, f64, (3 * n,), "r"), _ptr(v, f64, (3 * n,), "v"),
        _ptr(e, f64, (n_gas,), "e", n_gas == 0),
        _ptr(v_save, f64, (3 * n,), "v_save", emit),
        _ptr(e_save, f64, (n_gas,), "e_save", emit or n_gas == 0),
        _ptr(acc_hyd, f32, (n_gas, 4), "acc_hyd", emit or n_gas == 0),
        _ptr(grav, f32, (n, 4), "grav", emit),
        _ptr(mass, f32, (n,), "mass", pos_m is None),
        _ptr(h, f32, (n_gas,), "h", pos_h is None or n_gas == 0),
        _ptr(pos_m, f32, (n, 4), "pos_m", True), _ptr(pos_h, f32, (n_gas, 4), "pos_h", True),
        _ptr(vel_e, f32, (n_gas, 4), "vel_e", True), _stream(stream))
    _check("integrate_step", rc)


def state_struct(t: dict, n, n_gas, fresh=0, grav_flags=0):
    def p(k):
        x = t.get(k)
        return None if x is None else x.data_ptr()
    gw = t.get("grav_work")
    return SphState(n, n_gas, p("r"), p("v"), p("e"), p("v_save"), p("e_save"), p("mass"),
                    p("h"), p("pos_m"), p("pos_h"), p("vel_e"), p("rho"), p("acc_hyd"),
                    p("grav"), int(fresh), int(grav_flags), None, p("grav_work"),
                    0 if gw is None else gw.numel() * gw.element_size())


class StageEvents:
    """2 * len(STAGES) CUDA events for one sph_step (created by the library)."""

    def __init__(self):
        self.count = 2 * len(STAGES)
        self.arr = (ctypes.c_void_p * self.count)()
        _check("sph_events_create", lib().sph_events_create(self.count, self.arr))

    @property
    def ptr(self):
        return ctypes.cast(self.arr, ctypes.c_void_p).value

    def stage_ms(self):
        out = {}
        for k, name in enumerate(STAGES):
            ms = ctypes.c_float()
            _check("sph_event_elapsed_ms", lib().sph_event_elapsed_ms(
                self.arr[2 * k], self.arr[2 * k + 1], ctypes.byref(ms)))
            out[name] = float(ms.value)
        return out

    def total_ms(self):
        ms = ctypes.c_float()
        _check("sph_event_elapsed_ms", lib().sph_event_elapsed_ms(
            self.arr[0], self.arr[self.count - 1], ctypes.byref(ms)))
        return float(ms.value)

    def close(self):
        if self.arr is not None:
            lib().sph_events_destroy(self.count, self.arr)
            self.arr = None


def sph_launch_count():
    return int(lib().sph_launch_count())


def sph_rhs_initial(ctx, state: SphState, stream=None):
    _check("sph_rhs_initial", lib().sph_rhs_initial(ctx.handle if ctx else None,
                                                    ctypes.byref(state), _stream(stream)))


def sph_step(ctx, state: SphState, dt, stream=None):
    _check("sph_step", lib().sph_step(ctx.handle if ctx else None, ctypes.byref(state), float(dt),
                                      _stream(stream)))


def sph_step_cfl(ctx, state: SphState, C, dt_max, dt_out, stream=None):
    """One step whose size (Eq. 17, capped at dt_max) is chosen on the device
    and written to dt_out (a 1-element float32 CUDA tensor)."""
    _check("sph_step_cfl", lib().sph_step_cfl(ctx.handle if ctx else None, ctypes.byref(state),
                                              float(C), float(dt_max),
                                              _ptr(dt_out, torch.float32, (1,), "dt_out"),
                                              _stream(stream)))


def sph_forces_cfl(ctx, n_gas, vel_e, rho, mass, acc_dedt, grav, C, dt_max, dt_min,
                   dt_particle=None, stream=None):
    """sph_forces plus the Eq. 17 time step in the same pass."""
    f32 = torch.float32
    rc = lib().sph_forces_cfl(ctx.handle, int(n_gas), _ptr(vel_e, f32, (n_gas, 4), "vel_e"),
                              _ptr(rho, f32, (n_gas,), "rho"), _ptr(mass, f32, (n_gas,), "mass"),
                              _ptr(acc_dedt, f32, (n_gas, 4), "acc_dedt"),
                              _ptr(grav, f32, None, "grav"), float(C), float(dt_max),
                              _ptr(dt_particle, f32, (n_gas,), "dt_particle", True),
                              _ptr(dt_min, f32, (1,), "dt_min"), _stream(stream))
    _check("sph_forces_cfl", rc)


def sph_diagnostics(state: SphState, out, stream=None):
    _check("sph_diagnostics", lib().sph_diagnostics(ctypes.byref(state),
                                                    _ptr(out, torch.float64, (8,), "out"),
                                                    _stream(stream)))


# ---------------------------------------------------------------------------
# Batches of independent simulations
# ---------------------------------------------------------------------------

class Batch:
    """A batch descriptor: per-simulation gas / dark offsets (host) and the
    simulation index of every gas particle (device), plus its workspace."""

    def __init__(self, gas_off, dark_off, sim_of_gas, stream=None):
        import numpy as np
        self.gas_off = np.ascontiguousarray(gas_off, np.int32)
        self.dark_off = np.ascontiguousarray(dark_off, np.int32)
        self.n_sims = len(self.gas_off) - 1
        self.sim_of_gas = sim_of_gas
        gp = self.gas_off.ctypes.data_as(ctypes.c_void_p)
        dp = self.dark_off.ctypes.data_as(ctypes.c_void_p)
        nbytes = int(lib().sph_batch_workspace_bytes(self.n_sims, gp, dp))
        if nbytes == 0:
            raise SphError("sph_batch_workspace_bytes", SPH_ERR_INVALID_ARG)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=sim_of_gas.device)
        ptr = self.workspace.data_ptr() + ((-self.workspace.data_ptr()) % 256)
        h = ctypes.c_void_p()
        n_gas = int(self.gas_off[-1])
        rc = lib().sph_batch_create(self.n_sims, gp, dp,
                                    _ptr(sim_of_gas, torch.int32, (n_gas,), "sim_of_gas", n_gas == 0),
                                    ctypes.c_void_p(ptr), nbytes, _stream(stream), ctypes.byref(h))
        _check("sph_batch_create", rc)
        self.handle = h

    def set_plan(self, R, stream=None):
        _check("sph_batch_set_plan", lib().sph_batch_set_plan(self.handle, int(R), _stream(stream)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().sph_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pp_gravity_batched(batch, pos_m, acc_pot, G=1.0, eps=0.01, flags=0, stream=None):
    n = pos_m.shape[0]
    rc = lib().pp_gravity_batched(batch.handle, _ptr(pos_m, torch.float32, (n, 4), "pos_m"),
                                  float(G), float(eps),
                                  _ptr(acc_pot, torch.float32, (n, 4), "acc_pot"), int(flags),
                                  _stream(stream))
    _check("pp_gravity_batched", rc)


def pp_gravity_pairs_batched(batch, pos_m, acc_pot, work, G=1.0, eps=0.01, flags=0, stream=None):
    """Pair-once gravity over every simulation of a batch (falls back to
    pp_gravity_batched when not eligible or `work` is None / too small)."""
    n = pos_m.shape[0]
    wp, wb = (None, 0) if work is None else (work.data_ptr(), work.numel() * work.element_size())
    rc = lib().pp_gravity_pairs_batched(batch.handle, _ptr(pos_m, torch.float32, (n, 4), "pos_m"),
                                        float(G), float(eps),
                                        _ptr(acc_pot, torch.float32, (n, 4), "acc_pot"), int(flags),
                                        wp, wb, _stream(stream))
    _check("pp_gravity_pairs_batched", rc)


def sph_ctx_set_batch(ctx, batch):
    _check("sph_ctx_set_batch", lib().sph_ctx_set_batch(ctx.handle, batch.handle if batch else None))
