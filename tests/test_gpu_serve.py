"""The request server (sim_submit / sph_server_step / sim_poll) through the C
ABI: a job's result does not depend on what else is resident, equals a lone
Simulation run, and admission respects the memory budget."""
import numpy as np
import pytest

from helpers import need_gpu
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def _run_all(server, timeout_steps=10000):
    from paper_1807_08116_gb300 import native as nv
    for _ in range(timeout_steps):
        res, _ = server.step()
        info = server.info()
        if info["resident"] == 0 and info["queued"] == 0:
            return
    raise AssertionError("server did not finish")


def test_result_alone_equals_result_in_the_mix():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server
    x = ics.two_halo(1500, 1500, seed=41)
    others = [ics.single_halo(3000, 1000, seed=42), ics.two_halo(600, 900, seed=43),
              ics.single_halo(0, 2500, seed=44)]
    alone = Server(2 << 30, max_resident=4, n_streams=4)
    jx = alone.submit(x, 6)
    _run_all(alone)
    ref = alone.poll(jx, with_result=True)
    assert ref["state"] == nv.SIM_DONE and ref["steps_done"] == 6

    mix = Server(2 << 30, max_resident=3, n_streams=2)
    ids = [mix.submit(others[0], 9), mix.submit(others[1], 3)]
    mix.step()                                   # x arrives while others run
    ids.append(mix.submit(x, 6))
    ids.append(mix.submit(others[2], 4))
    _run_all(mix)
    got = mix.poll(ids[2], with_result=True)
    assert got["state"] == nv.SIM_DONE
    for k in ("r", "v", "e"):
        assert np.array_equal(got[k], ref[k]), k
    for j in ids:
        assert mix.poll(j)["state"] == nv.SIM_DONE


def test_server_equals_simulation():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server
    from paper_1807_08116_gb300.sim import Simulation
    d = ics.single_halo(2048, 2048, seed=45)
    srv = Server(1 << 30, max_resident=2, n_streams=1)
    j = srv.submit(d, 4)
    _run_all(srv)
    got = srv.poll(j, with_result=True)
    sim = Simulation(d)
    sim.initial_rhs()
    for _ in range(4):
        sim.step(1e-3)
    assert np.array_equal(got["r"], sim.positions())
    assert np.array_equal(got["v"], sim.velocities())


def test_budget_admission_and_errors():
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server
    small = ics.single_halo(4000, 4000, seed=46)
    srv = Server(24 << 20, max_resident=8, n_streams=2)
    with pytest.raises(nv.SphError) as ex:
        srv.submit(ics.two_halo(131072, 131072, seed=47), 2)     # can never fit
    assert ex.value.code == nv.SPH_ERR_BUDGET
    ids = [srv.submit(small, 2) for _ in range(8)]
    srv.step()
    info = srv.info()
    assert info["resident"] >= 1 and info["queued"] >= 1      # memory, not slots, binds
    _run_all(srv)
    for j in ids:
        assert srv.poll(j)["state"] == nv.SIM_DONE
    assert srv.info()["arena_free_bytes"] == srv.info()["arena_bytes"]
    with pytest.raises(nv.SphError) as ex:
        srv.poll(987654321)
    assert ex.value.code == nv.SPH_ERR_NOT_FOUND
    srv.release(ids[0])
    with pytest.raises(nv.SphError):
        srv.poll(ids[0])


def test_job_admitted_mid_stream_matches_the_oracle(orc):
    # a collision submitted while another job is already running, advanced in
    # the mix, against the FP64 oracle stepping the same initial condition
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server
    from helpers import err
    x = ics.two_halo(1024, 1024, seed=48)
    busy = ics.single_halo(3000, 1500, seed=49)
    srv = Server(1 << 30, max_resident=4, n_streams=2)
    jb = srv.submit(busy, 8)
    srv.step()
    srv.step()
    jx = srv.submit(x, 5)
    _run_all(srv)
    got = srv.poll(jx, with_result=True)
    assert got["state"] == nv.SIM_DONE and got["steps_done"] == 5
    assert srv.poll(jb)["state"] == nv.SIM_DONE
    ref = orc.OracleSim(x["r"].T, x["v"].T, x["e"], x["m"], x["h"], x["n_gas"])
    ref.initial_rhs()
    for _ in range(5):
        ref.step(1e-3)
    dr = np.abs(got["r"] - ref.r.T).max()
    rv, mv = err(got["v"], ref.v.T)
    re_, _ = err(got["e"][:, None], ref.e[:, None])
    print(f"served job vs oracle: |dr| {dr:.2e}, v rms {rv:.2e} max {mv:.2e}, e rms {re_:.2e}")
    assert dr < 1e-9
    assert rv < 1e-6
    assert re_ < 1e-6


def _scaled_h_job(orc, n_gas, lo, hi, seed):
    """A gas sphere whose smoothing lengths are scaled so that its neighbour
    lists need between lo and hi entries per particle (brute-force count)."""
    from helpers import pos_h_of
    d = ics.single_halo(n_gas, 0, seed=seed)
    for f in np.linspace(1.0, 1.6, 25):
        h = (d["h"] * f).astype(np.float32)
        starts, _ = orc.neighbors(pos_h_of(d["r"], h))
        per = starts[-1] / n_gas
        if lo < per < hi:
            d = dict(d)
            d["h"] = h
            return d, per
    raise AssertionError("no scale puts the list length in range")


def test_admission_that_fails_after_sizing_lists_leaves_the_next_job_intact(orc):
    # The first job's lists need 88-115 entries per particle: admission builds
    # them in its first context (120 per particle), finds them more than 70%
    # full, and asks the arena for a larger context, which the budget refuses.
    # Its memory goes back to the arena while its list kernels may still be
    # queued; the next job is admitted into the same bytes on another stream
    # and must still give exactly its lone result.
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server
    big, per = _scaled_h_job(orc, 6000, 88.0, 115.0, seed=50)
    small = ics.single_halo(1500, 500, seed=51)
    alone = Server(256 << 20, max_resident=2, n_streams=2)
    js = alone.submit(small, 3)
    _run_all(alone)
    ref = alone.poll(js, with_result=True)
    assert ref["state"] == nv.SIM_DONE
    # an arena that holds the big job's state and first context, not a second one
    ws1 = nv.sph_ctx_workspace_bytes(6000, nv.default_log2_M(6000), 120 * 6000)
    budget = int(1.3 * ws1) + (4 << 20)
    srv = Server(budget, max_resident=2, n_streams=2)
    jf = srv.submit(big, 3)
    jn = srv.submit(small, 3)
    _run_all(srv)
    st = srv.poll(jf)
    assert st["state"] == nv.SIM_FAILED and st["error"] == nv.SPH_ERR_BUDGET, (st, per)
    got = srv.poll(jn, with_result=True)
    assert got["state"] == nv.SIM_DONE
    for k in ("r", "v", "e"):
        assert np.array_equal(got[k], ref[k]), k
    assert srv.info()["arena_free_bytes"] == srv.info()["arena_bytes"]


def test_small_job_is_not_held_to_the_pace_of_a_large_one():
    # No lockstep: a small job with twice the steps of a large resident one
    # finishes first, each step timed on its own stream, and its result is
    # still exactly its lone result.
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server
    big = ics.two_halo(65536, 65536, seed=52)
    small = ics.single_halo(2048, 2048, seed=53)
    alone = Server(2 << 30, max_resident=2, n_streams=2)
    js = alone.submit(small, 16)
    _run_all(alone)
    ref = alone.poll(js, with_result=True)
    srv = Server(4 << 30, max_resident=4, n_streams=4)
    jb = srv.submit(big, 8)
    js = srv.submit(small, 16)
    for _ in range(100000):
        srv.step()
        if srv.poll(js)["state"] == nv.SIM_DONE:
            break
    sb = srv.poll(jb)
    assert sb["steps_done"] < sb["n_steps"], sb     # the large job is still running
    got = srv.poll(js, with_result=True)
    for k in ("r", "v", "e"):
        assert np.array_equal(got[k], ref[k]), k
    _run_all(srv)
    assert srv.poll(jb)["state"] == nv.SIM_DONE
    times = srv.step_times()
    assert len(times) == 8 + 16 and np.all(times > 0)
    print(f"step ms: small p50 {got['step_ms_p50']:.2f}, large p50 {srv.poll(jb)['step_ms_p50']:.2f}")
    assert got["step_ms_p50"] < srv.poll(jb)["step_ms_p50"]


def test_shortest_first_admission():
    # one slot: under FIFO the first request is admitted first; under
    # shortest-first the request with the least work left is, whatever its
    # place in the queue
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server
    big = ics.two_halo(8192, 8192, seed=54)
    small = ics.single_halo(1024, 1024, seed=55)
    for policy, first in ((nv.SPH_SERVE_FIFO, "big"), (nv.SPH_SERVE_SHORTEST_FIRST, "small")):
        srv = Server(1 << 30, max_resident=1, n_streams=1)
        srv.set_policy(policy)
        ids = {"big": srv.submit(big, 3), "small": srv.submit(small, 3)}
        _run_all(srv)
        st = {k: srv.poll(v) for k, v in ids.items()}
        assert all(x["state"] == nv.SIM_DONE for x in st.values())
        other = "small" if first == "big" else "big"
        assert st[first]["done_s"] <= st[other]["admit_s"], (policy, st)


def test_checkpoint_resumes_bitwise():
    # a checkpoint of a running job, submitted as a new request with the
    # remaining steps, ends in exactly the state of the uninterrupted job
    need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.serve import Server
    d = ics.two_halo(1200, 800, seed=56)
    total = 9
    srv = Server(1 << 30, max_resident=2, n_streams=2)
    j = srv.submit(d, total)
    while srv.poll(j)["steps_done"] < 4:
        srv.step()
    ck, done = srv.checkpoint(j)
    assert 4 <= done < total
    _run_all(srv)
    full = srv.poll(j, with_result=True)
    ic = dict(ck)
    ic["m"] = d["m"]
    srv2 = Server(1 << 30, max_resident=2, n_streams=2)
    j2 = srv2.submit(ic, total - done)
    _run_all(srv2)
    res = srv2.poll(j2, with_result=True)
    assert res["state"] == nv.SIM_DONE
    for k in ("r", "v", "e"):
        assert np.array_equal(res[k], full[k]), k
