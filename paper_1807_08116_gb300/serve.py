"""Serving: a thin Python face of the library's request server (sim_submit,
sph_server_step, sim_poll, sph_server_step_times) and a driver that replays
a timed request trace.

All scheduling, admission against the memory budget and stepping happen in
the C++ server (csrc/serve.cu); this module marshals arrays and keeps time.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import torch

from . import native as nv


class Server:
    def __init__(self, budget_bytes, max_resident=16, n_streams=8, device=None, **params):
        lib = nv.lib()
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.arena = torch.empty(int(budget_bytes) + 256, dtype=torch.uint8, device=dev)
        base = self.arena.data_ptr() + ((-self.arena.data_ptr()) % 256)
        self.params = nv.params_struct(**params)
        h = ctypes.c_void_p()
        nv._check("sph_server_create", lib.sph_server_create(
            ctypes.byref(self.params), ctypes.c_void_p(base), int(budget_bytes), int(max_resident),
            int(n_streams), ctypes.byref(h)))
        self.handle = h

    def submit(self, ic, n_steps, dt=1e-3):
        n, ng = int(ic["n"]), int(ic["n_gas"])
        r = np.ascontiguousarray(np.asarray(ic["r"], np.float64).T)
        v = np.ascontiguousarray(np.asarray(ic["v"], np.float64).T)
        e = np.ascontiguousarray(ic["e"], np.float64)
        m = np.ascontiguousarray(ic["m"], np.float32)
        h = np.ascontiguousarray(ic["h"], np.float32)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        req = nv.SimRequest(n, ng, int(n_steps), float(dt), P(r), P(v), P(e), P(m), P(h))
        jid = ctypes.c_uint64()
        nv._check("sim_submit", nv.lib().sim_submit(self.handle, ctypes.byref(req), ctypes.byref(jid)))
        return int(jid.value)

    def step(self):
        res = ctypes.c_int32()
        ms = ctypes.c_double()
        nv._check("sph_server_step", nv.lib().sph_server_step(self.handle, ctypes.byref(res),
                                                              ctypes.byref(ms)))
        return int(res.value), float(ms.value)

    def poll(self, jid, with_result=False):
        st = nv.SimStatus()
        nv._check("sim_poll", nv.lib().sim_poll(self.handle, int(jid), ctypes.byref(st)))
        out = {k: getattr(st, k) for k, _ in nv.SimStatus._fields_ if not k.startswith("h_")}
        if with_result and st.state == nv.SIM_DONE:
            n, ng = st.n, st.n_gas
            def arr(ptr, count):
                buf = (ctypes.c_double * count).from_address(ptr)
                return np.frombuffer(buf, np.float64).copy()
            out["r"] = arr(st.h_r, 3 * n).reshape(3, n).T
            out["v"] = arr(st.h_v, 3 * n).reshape(3, n).T
            out["e"] = arr(st.h_e, ng) if ng else np.zeros(0)
        return out

    def set_policy(self, policy):
        """nv.SPH_SERVE_FIFO or nv.SPH_SERVE_SHORTEST_FIRST admission order."""
        nv._check("sph_server_set_policy", nv.lib().sph_server_set_policy(self.handle, int(policy)))

    def step_times(self):
        """Latencies (ms) of every simulation step completed so far."""
        cnt = ctypes.c_int32()
        nv._check("sph_server_step_times", nv.lib().sph_server_step_times(self.handle, None, 0,
                                                                          ctypes.byref(cnt)))
        buf = np.zeros(max(cnt.value, 1), np.float32)
        nv._check("sph_server_step_times", nv.lib().sph_server_step_times(
            self.handle, buf.ctypes.data_as(ctypes.c_void_p), buf.size, ctypes.byref(cnt)))
        return buf[:min(cnt.value, buf.size)].copy()

    def checkpoint(self, jid):
        """State of a resident job as an initial condition (r, v, e, h, m) and
        the steps it has taken; submit it with the remaining steps to resume."""
        st = self.poll(jid)
        n, ng = st["n"], st["n_gas"]
        r = np.empty(3 * n)
        v = np.empty(3 * n)
        e = np.empty(max(ng, 1))
        h = np.empty(max(ng, 1), np.float32)
        done = ctypes.c_int32()
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        nv._check("sim_checkpoint", nv.lib().sim_checkpoint(self.handle, int(jid), P(r), P(v), P(e), P(h),
                                                            ctypes.byref(done)))
        return dict(r=r.reshape(3, n).T.copy(), v=v.reshape(3, n).T.copy(), e=e[:ng].copy(),
                    h=h[:ng].copy(), n=n, n_gas=ng), int(done.value)

    def release(self, jid):
        nv._check("sim_release", nv.lib().sim_release(self.handle, int(jid)))

    def info(self):
        i = nv.SphServerInfo()
        nv._check("sph_server_info", nv.lib().sph_server_info(self.handle, ctypes.byref(i)))
        return dict(queued=i.queued, resident=i.resident, arena_bytes=i.arena_bytes,
                    arena_free_bytes=i.arena_free_bytes)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            nv.lib().sph_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def replay_trace(server, trace, make_ic, window_s, dt=1e-3):
    """Submit the requests of `trace` (dicts with arrival time t in seconds,
    n, steps and IC parameters) at their arrival times and step the server
    until every request finished or `window_s` seconds passed.  Returns
    per-request records and per-step wall times."""
    pending = sorted(trace, key=lambda x: x["t"])
    ics_ready = {}
    t0 = time.perf_counter()
    jobs = {}
    steps = []
    k = 0
    while True:
        now = time.perf_counter() - t0
        while k < len(pending) and pending[k]["t"] <= now:
            req = pending[k]
            ic = ics_ready.pop(k, None) or make_ic(req)
            jid = server.submit(ic, req["steps"], dt)
            jobs[jid] = dict(req=req, submitted=time.perf_counter() - t0, n=ic["n"])
            k += 1
        if k < len(pending) and k not in ics_ready:
            ics_ready[k] = make_ic(pending[k])   # prepare the next arrival while waiting
        resident, ms = server.step()
        if resident or ms > 0:
            steps.append(dict(t=time.perf_counter() - t0, resident=resident, ms=ms))
        done = all(server.poll(j)["state"] >= nv.SIM_DONE for j in jobs)
        if (k == len(pending) and done) or time.perf_counter() - t0 > window_s:
            break
        if resident == 0 and k < len(pending):
            time.sleep(max(0.0, min(0.05, pending[k]["t"] - (time.perf_counter() - t0))))
    for jid, rec in jobs.items():
        st = server.poll(jid)
        rec.update(state=st["state"], steps_done=st["steps_done"], n_steps=st["n_steps"],
                   latency_s=(st["done_s"] - st["submit_s"]) if st["state"] == nv.SIM_DONE else None,
                   step_ms_p50=st["step_ms_p50"], step_ms_p99=st["step_ms_p99"])
    return jobs, steps, time.perf_counter() - t0
