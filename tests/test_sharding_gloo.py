"""Multi-rank path on CPU: two gloo ranks shard phase 1 by series and phase 2
by library rows, exchange optE once, and together reproduce the
single-process result exactly (the compute steps here are the oracle)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import edm_synth as synth
from paper_2011_11082_gb300.sharding import run_sharded, shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, Y, E_max, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as orc

    def opt(Ys):
        return orc.optimal_E(Ys, E_max, nthreads=1)[0]

    def rows(Yf, optE, b, e):
        return orc.ccm_rho_rows(Yf, optE.numpy(), rows=np.arange(b, e), nthreads=1)

    optE, (b, e), R = run_sharded(Y, opt, rows, world, rank)
    np.save(os.path.join(out_dir, f"rows_{rank}.npy"), R)
    np.save(os.path.join(out_dir, f"optE_{rank}.npy"), optE.numpy())
    np.save(os.path.join(out_dir, f"range_{rank}.npy"), np.array([b, e]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_covers_exactly():
    for n in (1, 7, 64, 101):
        for w in (1, 2, 3, 8):
            seen = []
            for r in range(w):
                b, e = shard_range(n, w, r)
                seen.extend(range(b, e))
            assert seen == list(range(n))


def test_two_ranks_match_single_process(tmp_path):
    from oracle import oracle as orc

    Y = synth.coupled_logistic(13, 160, 0.1, 0.05, seed_data=21, seed_noise=22)
    E_max = 5
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, Y, E_max, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    oE, _ = orc.optimal_E(Y, E_max)
    R = orc.ccm_rho_rows(Y, oE)
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"optE_{r}.npy"), oE)
    parts = [np.load(tmp_path / f"rows_{r}.npy") for r in range(2)]
    ranges = [tuple(np.load(tmp_path / f"range_{r}.npy")) for r in range(2)]
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == 13
    assert np.array_equal(np.concatenate(parts), R)


def _ss_worker(rank, world, port, Y, E_max, out_dir):
    from oracle import oracle as orc
    from paper_2011_11082_gb300.sharding import run_self_scheduled

    store = dist.TCPStore("127.0.0.1", port, world, is_master=(rank == 0), timeout=__import__("datetime").timedelta(seconds=120))

    def opt(Ys):
        return orc.optimal_E(Ys, E_max, nthreads=1)[0]

    def rows(Yf, optE, b, e):
        if rank == 0:  # a slow rank: the other one should take more blocks
            __import__("time").sleep(0.05)
        return orc.ccm_rho_rows(Yf, optE.numpy(), rows=np.arange(b, e), nthreads=1)

    optE, blocks = run_self_scheduled(Y, opt, rows, store, block=2, phase1_block=3, timeout_s=120)
    np.save(os.path.join(out_dir, f"ss_optE_{rank}.npy"), optE.numpy())
    for lo, hi, R in blocks:
        np.save(os.path.join(out_dir, f"ss_rows_{lo}_{hi}_{rank}.npy"), R)
    # keep the master's store alive until every other rank has stopped using it
    store.add("ss/finished", 1)
    while int(store.add("ss/finished", 0)) < world:
        __import__("time").sleep(0.01)
    if rank != 0:
        store.add("ss/left", 1)
    else:
        while int(store.add("ss/left", 0)) < world - 1:
            __import__("time").sleep(0.01)


def test_self_scheduled_ranks_cover_every_block_once(tmp_path):
    """Three ranks pull phase-1 and phase-2 blocks from a shared counter:
    every block is computed exactly once, the union equals the single-process
    result, and a slower rank ends up with fewer blocks."""
    from oracle import oracle as orc

    Y = synth.coupled_logistic(14, 150, 0.1, 0.05, seed_data=23, seed_noise=24)
    E_max = 4
    port = _free_port()
    mp.start_processes(_ss_worker, args=(3, port, Y, E_max, str(tmp_path)), nprocs=3, join=True, start_method="spawn")
    oE, _ = orc.optimal_E(Y, E_max)
    R = orc.ccm_rho_rows(Y, oE)
    for r in range(3):
        assert np.array_equal(np.load(tmp_path / f"ss_optE_{r}.npy"), oE)
    got = np.full_like(R, np.nan)
    owners = {}
    for f in os.listdir(tmp_path):
        if f.startswith("ss_rows_"):
            lo, hi, r = (int(v) for v in f[len("ss_rows_"):-4].split("_"))
            assert (lo, hi) not in owners
            owners[(lo, hi)] = r
            got[lo:hi] = np.load(tmp_path / f)
    assert sorted(owners) == [(b, min(14, b + 2)) for b in range(0, 14, 2)]
    assert np.array_equal(got, R)
    counts = [sum(1 for v in owners.values() if v == r) for r in range(3)]
    assert counts[0] <= max(counts[1], counts[2]), counts


def _steps_worker(rank, world, port, Y, E_max, out_dir):
    """The strong-scaling bench mode's use of the runtime: the default store of
    a gloo process group, one tag per step, several steps in a row."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as orc
    from paper_2011_11082_gb300.sharding import run_self_scheduled

    store = dist.distributed_c10d._get_default_store()
    N = Y.shape[0]
    for k in range(2):
        rho = np.full((N, N), np.nan)  # this rank's columns of a target-major map

        def opt(Ys):
            return orc.optimal_E(Ys, E_max, nthreads=1)[0]

        def rows(Yf, optE, b, e):
            rho[:, b:e] = orc.ccm_rho_rows(Yf, optE.numpy(), rows=np.arange(b, e), nthreads=1).T
            return e - b

        optE, blocks = run_self_scheduled(Y, opt, rows, store, block=3, phase1_block=4, tag=f"bench/{k}")
        np.save(os.path.join(out_dir, f"st{k}_rho_{rank}.npy"), rho)
        np.save(os.path.join(out_dir, f"st{k}_optE_{rank}.npy"), optE.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_self_scheduled_steps_on_the_process_group_store(tmp_path):
    """Two ranks, two consecutive steps on the process group's own store:
    in each step the ranks' columns together form the single-process
    target-major map, every column exactly once."""
    from oracle import oracle as orc

    Y = synth.coupled_logistic(11, 140, 0.1, 0.05, seed_data=25, seed_noise=26)
    E_max = 4
    port = _free_port()
    mp.start_processes(_steps_worker, args=(2, port, Y, E_max, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    oE, _ = orc.optimal_E(Y, E_max)
    R = orc.ccm_rho_rows(Y, oE).T  # target-major
    for k in range(2):
        parts = [np.load(tmp_path / f"st{k}_rho_{r}.npy") for r in range(2)]
        have = [~np.isnan(p).all(axis=0) for p in parts]
        assert not np.any(have[0] & have[1]) and np.all(have[0] | have[1])
        got = np.where(have[0][None, :], parts[0], parts[1])
        assert np.array_equal(got, R)
        for r in range(2):
            assert np.array_equal(np.load(tmp_path / f"st{k}_optE_{r}.npy"), oE)
