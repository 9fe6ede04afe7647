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
