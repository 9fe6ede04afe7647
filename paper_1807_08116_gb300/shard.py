"""The particle partition of the paper's multi-GPU design for the gravity
stage (Sect. 3: with k GPUs, each GPU computes the dynamics of N/k particles).

Each rank owns one contiguous range of particle rows.  Per gravity evaluation
it contributes the (x, y, z, m) of its own rows to one all-gather of 16 bytes
per particle, which leaves every rank with the whole set of sources, and then
computes the gravity of its own rows over all N sources with the library's
pp_gravity_rows kernel.  The integrator and the SPH stages of a rank touch
only its own rows (SPH would also need the gas within reach of the partition
boundary; the gravity exchange is the one this module carries).

torch.distributed carries the all-gather (NCCL between GPUs, gloo on CPU);
every row's arithmetic runs in the CUDA kernel.  With no process group the
module degenerates to one rank that owns every row.
"""
from __future__ import annotations

import torch

from . import native as nv


def row_ranges(n: int, world: int):
    """Contiguous, balanced rows [i0, i1) of each of `world` ranks; the first
    n % world ranks take one row more."""
    if n < 0 or world < 1:
        raise ValueError("n >= 0 and world >= 1 required")
    base, extra = divmod(n, world)
    out, i0 = [], 0
    for r in range(world):
        i1 = i0 + base + (1 if r < extra else 0)
        out.append((i0, i1))
        i0 = i1
    return out


def _world(group=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def owned_rows(n: int, group=None):
    """Rows [i0, i1) this rank owns."""
    world, rank = _world(group)
    return row_ranges(n, world)[rank]


def gather_positions(local_pos_m: torch.Tensor, n: int, group=None) -> torch.Tensor:
    """All-gather of every rank's (x, y, z, m) rows into one [n, 4] array in
    row order.  local_pos_m holds this rank's rows (its owned_rows range).
    Ranges may differ by one row, so each block travels padded to the
    largest one and the padding is dropped on arrival."""
    world, rank = _world(group)
    ranges = row_ranges(n, world)
    i0, i1 = ranges[rank]
    if tuple(local_pos_m.shape) != (i1 - i0, 4):
        raise ValueError(f"local_pos_m must have shape {(i1 - i0, 4)}, got {tuple(local_pos_m.shape)}")
    if world == 1:
        return local_pos_m.contiguous()
    import torch.distributed as dist
    m = max(b - a for a, b in ranges)
    send = torch.zeros((m, 4), dtype=local_pos_m.dtype, device=local_pos_m.device)
    send[: i1 - i0] = local_pos_m
    recv = torch.empty((world * m, 4), dtype=local_pos_m.dtype, device=local_pos_m.device)
    dist.all_gather_into_tensor(recv, send, group=group)
    parts = [recv[r * m: r * m + (b - a)] for r, (a, b) in enumerate(ranges)]
    return torch.cat(parts, 0).contiguous()


def _kernel_rows(pos_m, i0, i1, out, G, eps, flags):
    nv.pp_gravity_rows(pos_m, i0, i1, out, G=G, eps=eps, flags=flags)


def sharded_gravity(local_pos_m: torch.Tensor, n: int, out_local: torch.Tensor, G=1.0, eps=0.01,
                    flags=0, group=None, rows_fn=None):
    """Gravity (Eq. 4) of this rank's own rows: one all-gather of the sources,
    then the rows [i0, i1) over all n of them into out_local [i1 - i0, 4].
    rows_fn(pos_m, i0, i1, out, G, eps, flags) computes the rows; it defaults
    to the library's pp_gravity_rows (device tensors)."""
    full = gather_positions(local_pos_m, n, group)
    i0, i1 = owned_rows(n, group)
    if tuple(out_local.shape) != (i1 - i0, 4):
        raise ValueError(f"out_local must have shape {(i1 - i0, 4)}, got {tuple(out_local.shape)}")
    (rows_fn or _kernel_rows)(full, i0, i1, out_local, G, eps, flags)
    return full
