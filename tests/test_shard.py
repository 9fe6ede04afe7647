"""The particle partition of the gravity stage (the paper's N/k particles per
GPU, Sect. 3) as gloo ranks on the CPU: the row split, the all-gather of
(x, y, z, m) with unequal blocks, and each rank's own rows assembled back
into the full result, which equals the oracle's gravity over all particles.
On the CPU the rows are computed by the oracle; on a GPU the same module
calls the library's pp_gravity_rows (tests/test_gpu_shard.py)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_row_ranges_cover_every_row_once():
    from paper_1807_08116_gb300.shard import row_ranges
    for n in (0, 1, 7, 1000, 1001, 4194304):
        for world in (1, 2, 3, 4, 8):
            rr = row_ranges(n, world)
            assert len(rr) == world and rr[0][0] == 0 and rr[-1][1] == n
            sizes = [b - a for a, b in rr]
            assert all(rr[k][1] == rr[k + 1][0] for k in range(world - 1))
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        row_ranges(10, 0)


def _oracle_rows(pos_m, i0, i1, out, G, eps, flags):
    import torch

    import oracle
    acc, pot = oracle.gravity(pos_m.numpy(), G, eps, rows=np.arange(i0, i1, dtype=np.int32))
    out[:, :3] = torch.as_tensor(acc, dtype=out.dtype)
    out[:, 3] = torch.as_tensor(pot, dtype=out.dtype)


def _worker(rank, world, port, n, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1807_08116_gb300 import ics
        from paper_1807_08116_gb300.shard import gather_positions, owned_rows, sharded_gravity
        d = ics.single_halo(n // 2, n - n // 2, seed=77)   # the same particles on every rank
        pm = np.empty((d["n"], 4), np.float32)
        pm[:, :3] = d["r"]
        pm[:, 3] = d["m"]
        i0, i1 = owned_rows(d["n"])
        local = torch.as_tensor(pm[i0:i1].copy())
        out = torch.empty((i1 - i0, 4), dtype=torch.float32)
        full = sharded_gravity(local, d["n"], out, rows_fn=_oracle_rows)
        gathered_ok = bool(np.array_equal(full.numpy(), pm))
        # assemble every rank's own rows on every rank (the same padded gather)
        res = gather_positions(out, d["n"])
        q.put((rank, i0, i1, gathered_ok, res.numpy() if rank == 0 else None))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 2003), (3, 1000)])
def test_gloo_ranks_assemble_the_oracle_gravity(orc, world, n):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ranges = [(a, b) for _, a, b, _, _ in res]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(ok for _, _, _, ok, _ in res)
    got = res[0][4]
    from paper_1807_08116_gb300 import ics
    d = ics.single_halo(n // 2, n - n // 2, seed=77)
    pm = np.empty((d["n"], 4), np.float32)
    pm[:, :3] = d["r"]
    pm[:, 3] = d["m"]
    acc, pot = orc.gravity(pm)
    # FP32 storage of FP64 rows: equal to rounding
    assert np.allclose(got[:, :3], acc, rtol=1e-6, atol=1e-7 * np.abs(acc).max())
    assert np.allclose(got[:, 3], pot, rtol=1e-6, atol=0)
