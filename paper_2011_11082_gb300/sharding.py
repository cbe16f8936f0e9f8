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


def _wait_count(store, key: str, target: int, timeout_s: float):
    """Block until the store counter `key` reaches `target` (bounded)."""
    import time

    t0 = time.monotonic()
    while int(store.add(key, 0)) < target:
        if time.monotonic() - t0 > timeout_s:
            raise TimeoutError(f"{key}: {int(store.add(key, 0))} of {target} after {timeout_s:.0f} s")
        time.sleep(0.002)


def run_self_scheduled(Y, compute_optE: Callable, compute_rows: Callable, store, block: int = 64,
                       phase1_block: int = 256, timeout_s: float = 600.0, tag: str = "edm"):
    """Self-scheduling form of the paper's master-worker runtime (Sec. III-C):
    every rank repeatedly takes the next unclaimed block from a shared atomic
    counter in `store` (a torch.distributed Store: TCPStore, FileStore, ...)
    until none are left, so fast ranks take more blocks.  Phase 1 runs over
    blocks of series; each finished block publishes its optE in the store;
    once all blocks are in, every rank reads the full optE (the paper's
    broadcast) and phase 2 runs over blocks of library rows.  Returns
    (optE [N] int32, [(row_begin, row_end, rows), ...] for the blocks this
    rank computed).  `tag` separates independent runs on one store; the
    store's server must outlive every rank's last call (synchronise the
    ranks before the process hosting it exits)."""
    import numpy as np

    N = Y.shape[0]
    n1 = (N + phase1_block - 1) // phase1_block
    while True:
        b = int(store.add(f"{tag}/p1/next", 1)) - 1
        if b >= n1:
            break
        lo, hi = b * phase1_block, min(N, (b + 1) * phase1_block)
        e = np.ascontiguousarray(np.asarray(compute_optE(Y[lo:hi]), dtype=np.int32))
        store.set(f"{tag}/p1/optE/{b}", e.tobytes())
        store.add(f"{tag}/p1/done", 1)
    _wait_count(store, f"{tag}/p1/done", n1, timeout_s)
    optE = np.concatenate([np.frombuffer(store.get(f"{tag}/p1/optE/{b}"), dtype=np.int32) for b in range(n1)])
    optE_t = torch.from_numpy(optE.copy())
    n2 = (N + block - 1) // block
    mine = []
    while True:
        b = int(store.add(f"{tag}/p2/next", 1)) - 1
        if b >= n2:
            break
        lo, hi = b * block, min(N, (b + 1) * block)
        mine.append((lo, hi, compute_rows(Y, optE_t, lo, hi)))
    return optE_t, mine
