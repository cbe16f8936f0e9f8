"""Multi-rank layout of the two phases (one process per GPU).

The paper distributes the two outer loops over series (Sec. III-C): phase 1
by series, then a broadcast of optE, then phase 2 by library series, each
worker writing its own rows of the causal map.  Here every rank takes a
contiguous shard of series for phase 1 and of library rows for phase 2; the
only exchange is an all-gather of the N optimal-E values between the
phases.  Nothing is reduced: each rank owns its rho rows.

The compute steps are passed in (the CUDA entry points on GPUs), so the
rank logic is the same whatever runs the kernels.
"""

from __future__ import annotations

from typing import Callable

import torch


def shard_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced [begin, end) of n items for `rank` of `world`."""
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def all_gather_optE(local: torch.Tensor, N: int, world: int, rank: int, group=None) -> torch.Tensor:
    """Concatenate every rank's optE shard (int32) into the full [N] vector."""
    import torch.distributed as dist

    sizes = [shard_range(N, world, r)[1] - shard_range(N, world, r)[0] for r in range(world)]
    width = max(sizes)
    buf = torch.zeros(width, dtype=torch.int32, device=local.device)
    buf[: local.numel()] = local
    out = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(out, buf, group=group)
    return torch.cat([o[:s] for o, s in zip(out, sizes)])


def run_sharded(Y, compute_optE: Callable, compute_rows: Callable, world: int, rank: int, group=None):
    """Phase 1 on this rank's series, all-gather optE, phase 2 on this
    rank's library rows.  Returns (optE [N], (row_begin, row_end), rows)."""
    N = Y.shape[0]
    b, e = shard_range(N, world, rank)
    local = compute_optE(Y[b:e])
    optE = all_gather_optE(torch.as_tensor(local, dtype=torch.int32), N, world, rank, group)
    rows = compute_rows(Y, optE, b, e)
    return optE, (b, e), rows
