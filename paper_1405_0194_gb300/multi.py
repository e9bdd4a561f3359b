"""Pole-parallel DM / EDM / FDM and shift-parallel inertia counts over several
GPUs, one process per GPU.

The poles of the expansion are independent (Sec. II.B): rank r evaluates a
contiguous share of them, accumulating its partial DM, EDM and FDM on the
pattern in its own device memory, and the pole sum is completed by one
sum-allreduce of the three nnz arrays. Inertia shifts are independent as
well (Sec. II.C); each rank counts a share and the counts are all-gathered
in shift order. Nothing else crosses ranks: every rank holds the same plan
(the symbolic analysis is deterministic, so all ranks build the identical
ordering and supernode partition).

The per-rank work goes through the C ABI (``pexsi_dm_device``,
``pexsi_inertia_device``); ``torch.distributed`` supplies the collective
(NCCL between GPUs). The orchestration takes the per-rank work as a callable,
so that its sharding and reduction can be exercised by CPU ranks (gloo).
"""
from __future__ import annotations

from typing import Callable

import numpy as np


def shard(count: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block [begin, end) of `count` items owned by `rank`; block
    sizes differ by at most one, lower ranks take the larger blocks."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(max(0, count), world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def dm_allreduce(compute_range: Callable[..., None], out, n_poles: int, batch: int, group=None):
    """Pole sum over all ranks of `group`.

    compute_range(begin, end, accumulate, last) evaluates poles [begin, end)
    into `out` (a 3 x nnz float64 tensor on this rank's device: DM, EDM, FDM),
    overwriting it when accumulate == 0 and adding otherwise; `last` marks
    the rank's final batch, where the status of all its batches is checked
    (a failure raises there, before the collective). Each rank runs its share
    in batches of at most `batch` poles, then one sum-allreduce leaves the
    full result in `out` on every rank."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    begin, end = shard(n_poles, world, rank)
    step = max(1, batch)
    starts = list(range(begin, end, step))
    for k, p in enumerate(starts):
        compute_range(p, min(end, p + step), 0 if k == 0 else 1, k == len(starts) - 1)
    if not starts:  # no poles on this rank: contribute zeros
        out.zero_()
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out


def inertia_allgather(count_shifts: Callable[[np.ndarray], np.ndarray], shifts, group=None, device=None):
    """Inertia counts of all shifts: each rank counts its share with
    count_shifts (returns int64 counts) and the shares are all-gathered in
    shift order."""
    import torch
    import torch.distributed as dist

    shifts = np.asarray(shifts, dtype=np.float64).ravel()
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    begin, end = shard(shifts.shape[0], world, rank)
    width = shard(shifts.shape[0], world, 0)[1]  # the largest share
    local = np.zeros(width, dtype=np.int64)
    if end > begin:
        local[:end - begin] = np.asarray(count_shifts(shifts[begin:end]), dtype=np.int64)
    t = torch.from_numpy(local)
    if device is not None:
        t = t.to(device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    counts = []
    for r in range(world):
        b, e = shard(shifts.shape[0], world, r)
        counts.append(parts[r].cpu().numpy()[:e - b])
    return np.concatenate(counts) if counts else np.zeros(0, dtype=np.int64)


def dm_sharded(plan, dH: int, dS: int, mu: float, beta: float, n_poles: int, delta_e: float, out, stream: int,
               batch: int, group=None):
    """DM / EDM / FDM of all n_poles poles with the poles shared among the
    ranks of `group`. dH, dS: device addresses of H and S on this rank's
    GPU; out: 3 x nnz float64 CUDA tensor (rows DM, EDM, FDM); stream: the
    CUDA stream of the calls (the current torch stream, so that the
    collective is ordered after them)."""
    from . import capi

    def compute_range(b: int, e: int, acc: int, last: bool) -> None:
        # the last batch reads the chain's status: a breakdown or a timed-out
        # wait in any batch of this rank raises PexsiError here
        capi.pexsi_dm_device(plan, dH, dS, mu, beta, n_poles, delta_e, b, e, acc, out[0].data_ptr(),
                             out[1].data_ptr(), out[2].data_ptr(), stream, want_info=last)

    return dm_allreduce(compute_range, out, n_poles, batch, group)


def inertia_sharded(plan, dH: int, dS: int, shifts, stream: int, group=None, device=None):
    """Inertia counts at all shifts, shifts shared among the ranks."""
    from . import capi

    return inertia_allgather(lambda sh: capi.pexsi_inertia_device(plan, dH, dS, sh, stream), shifts, group, device)
