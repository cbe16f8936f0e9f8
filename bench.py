"""All-pairs CCM benchmark: cross-map pairs per second on one GB300.

A step is one pass of the whole hot path over the synthetic workload:
phase 1 (optimal E of every series) + phase 2 (kNN tables, lookup and rho
for every library x target pair), with the N x N rho written to device
memory.  Default workload: N = 101,729 coupled logistic maps, T = 1,500.

    python bench.py --gpus N --steps K --warmup W [--impl reference]

Prints one JSON line on rank 0.  `value` is whole-job pairs/s from CUDA
events on the launching stream (max over ranks); `roofline` is for the
dominant kernel (lookup) from per-launch events taken live in the timed
region; `e2e` is the same metric through the public API with host buffers
(H2D of the series and D2H of rho inside the timed region);
`cpu_baseline` is the FP64 oracle on a bounded sample on this host's cores.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (N, T, density, b_max, E_max)
    "n101729_t1500": (101729, 1500, 0.0001, 0.02, 20),
    "n16384_t1500": (16384, 1500, 0.001, 0.02, 20),
    "n2048_t1500": (2048, 1500, 0.01, 0.02, 20),
    "n64_t500": (64, 500, 0.05, 0.05, 10),
}
# the batched form: 256 independent datasets, N ~ U[32, 1024], T ~ U[200, 3000]
BATCHED = "batched256"
METRIC = "cross-map pairs/s at N=101,729,T=1500 (1 GB300) + % HBM roofline vs plain FP32"
UNIT = "pairs/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# shared-memory bandwidth per SM and clock (bytes / cycle): 32 banks x 4 B
SMEM_BYTES_PER_CLK = 128.0


def _lookup_sources_hash():
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2011_11082_gb300", "csrc")
    # the kernels and the planner (which shapes every launch)
    for f in ("lookup_chunked.cuh", "lookup_multi_impl.cuh", "lookup_chunked128.cu", "lookup_chunked64.cu", "edm_api.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def _measured_traffic(workload, precision, pairs_per_launch):
    """DRAM bytes per lookup launch (read + write) from the committed ncu
    capture, if it was taken on the lookup kernels and planner as they are
    now (else None).  The capture stores bytes per pair of the captured
    launches; launches differ in size, so the figure is scaled to the mean
    launch of this run (traffic grows with the pairs a launch processes)."""
    p = os.path.join(ROOT, "profiles", "lookup_dram_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(f"{workload}/{precision}")
    if not e or e.get("sources") != _lookup_sources_hash():
        return None
    return float(e["bytes_per_pair"]) * pairs_per_launch


def _smem_gather_bytes(hist, T, Tp, s_y, N):
    """Shared-memory bytes the lookup must read per step: for every (library,
    target) pair, every query row reads E+1 gathered values and one
    observation, s_y bytes each."""
    tot = 0.0
    for e0, cnt in enumerate(hist):
        E = e0 + 1
        if cnt:
            tot += float(cnt) * (T - Tp - (E - 1)) * (E + 2) * s_y
    return tot * N


def _algorithmic_bytes_per_pair(N, T, s_y):
    # rho write (4 B) + every target read once + every library read once
    # + optE, spread over the N^2 pairs.
    return 4.0 + (N * T * s_y + N * T * 4.0 + 4.0 * N) / float(N) / float(N)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def sample_rows_of(N, sample_rows, seed=7):
    """Seeded library rows (and series) the oracle samples, spread over all N
    (so they fall in different library blocks and E groups)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=min(N, sample_rows), replace=False)).astype(np.int64)


def cpu_baseline(Y, optE, sample_rows, N, E_max=20, keep=None):
    """The FP64 oracle, as it stands, on `sample_rows` seeded library rows x
    all targets (phase 2) plus phase 1 of the same series; scaled to
    pairs/s.  optE=None: the targets' E are the oracle's phase-1 values of
    the sampled series, repeated over all N targets.  keep (a dict): receives
    the sampled rows, the oracle's phase-1 optE of those series and its rho
    rows (library-major), for the parity record."""
    from oracle import oracle as orc

    cores = orc.default_threads()
    if sample_rows <= 0:
        sample_rows = 2 * cores
    rows = sample_rows_of(N, sample_rows)
    sample_rows = rows.size
    t0 = time.perf_counter()
    oE, _ = orc.optimal_E(Y[rows], E_max, nthreads=cores)
    t1 = time.perf_counter()
    if optE is None:
        optE = np.resize(oE, N).astype(np.int32)
    R = orc.ccm_rho_rows(Y, optE, rows=rows, nthreads=cores)
    t2 = time.perf_counter()
    if keep is not None:
        keep.update(rows=rows, optE=oE, rho=R)
    # whole-path time for N^2 pairs, extrapolated: phase 1 for N series and
    # phase 2 for N library rows.
    per_series_p1 = (t1 - t0) / sample_rows
    per_row_p2 = (t2 - t1) / sample_rows
    est = N * (per_series_p1 + per_row_p2)
    # the same on one thread (2 series + 2 library rows)
    one = min(2, sample_rows)
    t3 = time.perf_counter()
    orc.optimal_E(Y[rows[:one]], E_max, nthreads=1)
    t4 = time.perf_counter()
    orc.ccm_rho_rows(Y, optE, rows=rows[:one], nthreads=1)
    t5 = time.perf_counter()
    est1 = N * ((t4 - t3) + (t5 - t4)) / one
    return {"value": float(N) * N / est, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": float(N) * N / est1,
            "sample": f"phase 1 on {sample_rows} seeded series + phase 2 for the same {sample_rows} library rows x "
                      f"all {N} targets "
                      f"({t2 - t0:.1f} s of CPU wall time), extrapolated to N={N}; single thread: {one} series + "
                      f"{one} rows ({t5 - t3:.1f} s)"}


def parity_record(gpu_cols, gpu_optE_rows, keep, tol):
    """Element-by-element comparison of the GPU's rho on the sampled library
    rows (gpu_cols: [N targets][rows], target-major columns) and its phase-1
    optE of the sampled series with the oracle's (keep from cpu_baseline)."""
    R = keep["rho"]  # [rows][N] library-major
    G = np.asarray(gpu_cols, dtype=np.float64).T
    nan_o, nan_g = np.isnan(R), np.isnan(G)
    both = ~nan_o & ~nan_g
    err = np.abs(G[both] - R[both])
    return {"library_rows": int(R.shape[0]), "targets": int(R.shape[1]), "pairs": int(R.size),
            "max_abs_err": float(err.max()) if err.size else None,
            "mean_abs_err": float(err.mean()) if err.size else None,
            "p99_abs_err": float(np.percentile(err, 99)) if err.size else None,
            "nan_mismatches": int(np.sum(nan_o != nan_g)), "tol": tol,
            "within_tol": bool(err.size and err.max() < tol and not np.any(nan_o != nan_g)),
            "optE_series": int(keep["optE"].size),
            "optE_mismatches": int(np.sum(np.asarray(gpu_optE_rows) != keep["optE"])),
            "rows": "seeded sample of library rows and series (see cpu_baseline.sample), all targets"}


def run_reference(args):
    """The oracle as the reference arm (host cores; rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import edm_synth

    N, T, dens, bmax, E_max = WORKLOADS[args.workload]
    Y = edm_synth.coupled_logistic(N, T, dens, bmax, 0, 1)
    # phase 1 of all N series is hours of FP64 CPU work: each step times the
    # oracle on a bounded sample (see cpu_baseline) and scales to N^2 pairs.
    for _ in range(args.warmup + args.steps):
        cb = cpu_baseline(Y, None, args.cpu_rows, N, E_max)
    val = cb["value"]
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(N) * N / val * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "N": N, "T": T, "E_max": E_max},
            "cpu_baseline": cb, "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_batched(args, lib, edm, _abi, torch, edm_synth):
    """The batched form: every step runs both phases for 256 datasets of
    uneven (N, T) through one replay of the captured CUDA graph."""
    dev = torch.device("cuda", 0)
    specs = edm_synth.batched_specs()
    data = [edm_synth.batched_dataset(sp) for sp in specs]
    prec = edm.EDM_PRECISION_FP16_TARGETS if args.precision == "fp16" else edm.EDM_PRECISION_FP32
    Ys = [torch.from_numpy(Y).to(dev) for Y in data]
    batch = edm.CCMBatch(Ys, E_max=20, precision=prec)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):  # the first run tunes and captures
        batch.run()
    torch.cuda.synchronize()
    pairs = float(sum(Y.shape[0] ** 2 for Y in data))
    launches0 = [lib.edm_launch_count(k) for k in range(_abi.EDM_KERNEL_BATCH)]
    lib.edm_profile_enable(1)
    lib.edm_profile_read(_abi.EDM_KERNEL_BATCH, None, None, None)
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        batch.run()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    lib.edm_profile_enable(0)
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = sum(lib.edm_launch_count(k) - launches0[k] for k in range(_abi.EDM_KERNEL_BATCH))
    m, n, u = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    lib.edm_profile_read(_abi.EDM_KERNEL_BATCH, ctypes.byref(m), ctypes.byref(n), ctypes.byref(u))
    peak, peak_kind = _peaks()
    s_y = 2.0 if args.precision == "fp16" else 4.0
    alg = sum(Y.shape[0] ** 2 * 4.0 + Y.shape[0] * Y.shape[1] * (4.0 + s_y) + 4.0 * Y.shape[0] for Y in data)
    g_s = m.value / 1e3 / max(1, n.value)
    achieved = alg / g_s / 1e9 if g_s > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_kind": peak_kind, "kernel": "batched graph (all kernels of one replay)"}
    # end to end: series in from pinned host memory, both phases, every rho
    # map and optE back to pinned host memory, all inside the timed region
    e2e = None
    if not args.no_e2e:
        Yh = [torch.from_numpy(Y).pin_memory() for Y in data]
        Rh = [torch.empty((Y.shape[0], Y.shape[0]), dtype=torch.float32, pin_memory=True) for Y in data]
        Eh = [torch.empty(Y.shape[0], dtype=torch.int32, pin_memory=True) for Y in data]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for Yd, Yp in zip(Ys, Yh):
                Yd.copy_(Yp, non_blocking=True)
            optE, rho = batch.run()
            for a, b in zip(Rh, rho):
                a.copy_(b, non_blocking=True)
            for a, b in zip(Eh, optE):
                a.copy_(b, non_blocking=True)
            torch.cuda.synchronize()
        ems = (time.perf_counter() - t0) * 1e3 / args.steps
        e2e = {"value": pairs / (ems / 1e3), "unit": UNIT, "ms_per_step": ems,
               "h2d_bytes_per_step": int(sum(Y.nbytes for Y in data)),
               "d2h_bytes_per_step": int(sum(Y.shape[0] ** 2 * 4 + Y.shape[0] * 4 for Y in data)),
               "host_buffers": "pinned", "api": "CCMBatch.run (edm_ccm_rho_batched)"}
    # the adjoint of the global mean rho (indices and optE frozen) for every
    # dataset, timed the same way (per-dataset edm_ccm_rho_backward calls)
    backward = None
    if not args.no_backward:
        grads = batch.mean_rho_grad()  # warm-up (workspaces)
        torch.cuda.synchronize()
        bl0 = [lib.edm_launch_count(k) for k in range(_abi.EDM_KERNEL_BATCH)]
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.steps):
            grads = batch.mean_rho_grad()
        b1.record(stream)
        torch.cuda.synchronize()
        bms = b0.elapsed_time(b1) / args.steps
        backward = {"ms_per_step": bms, "what": "dL/dY of the global mean rho over all 256 datasets "
                    "(edm_ccm_rho_backward per dataset: kNN tables rebuilt, target and library passes)",
                    "gpu_launches": sum(lib.edm_launch_count(k) - bl0[k] for k in range(_abi.EDM_KERNEL_BATCH)),
                    "grad_values": int(sum(g.numel() for g in grads))}
    line = {"metric": "cross-map pairs/s, batched form (256 datasets, 1 GB300)", "value": pairs / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f16-targets/f32-accumulate", "data": "synthetic",
            "config": {"workload": BATCHED, "datasets": len(data), "pairs": pairs, "E_max": 20,
                       "precision": args.precision, "graph": "one cudaGraphLaunch per step",
                       "l2": "series 0.9 GB in total, rho 0.39 GB (rho alone exceeds L2)"},
            "roofline": roofline, "cpu_baseline": None, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
            "backward": backward}
    print(json.dumps(line), flush=True)
    return 0


# The paper's dataset-size study (Sec. IV, "Impact of Dataset Size"): runtime
# and its split between kNN and lookup while the number of series grows at
# 10,000 time steps, and while the number of time steps grows at 1,000
# series (up to 40,000).  Synthetic coupled maps stand in for its dummy
# datasets; the coupling density keeps about 10 inputs per map.
SWEEPS = {
    "series": [(n, 10000) for n in (500, 1000, 2000, 4000, 8000)],
    "steps": [(1000, t) for t in (1000, 2000, 5000, 10000, 20000, 40000)],
}


def bench_sweep(args, lib, edm, _abi, torch, edm_synth):
    """One JSON line per (N, T) of the sweep: step time (both phases, CUDA
    events), pairs/s and the per-kernel split from per-launch events."""
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    E_max = 20
    sizes = SWEEPS[args.sweep]
    if args.size:
        sizes = [tuple(int(v) for v in args.size.lower().split("x"))]
    for N, T in sizes:
        Y = edm_synth.coupled_logistic(N, T, min(0.05, 10.0 / N), 0.02, seed_data=0, seed_noise=1)
        Yd = torch.from_numpy(Y).to(dev)
        rho = torch.empty((N, N), dtype=torch.float32, device=dev)
        ws = torch.empty(edm.edm_ccm_workspace_bytes(N, T), dtype=torch.uint8, device=dev)

        def step():
            optE, _ = edm.edm_optimal_E(Yd, E_max=E_max, return_rho=False)
            edm.edm_ccm_rho(Yd, optE, out=rho, workspace=ws)
            return optE

        optE = step()  # warm-up
        torch.cuda.synchronize()
        lib.edm_profile_enable(1)
        for k in range(4):
            lib.edm_profile_read(k, None, None, None)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            optE = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        lib.edm_profile_enable(0)
        ms = ev0.elapsed_time(ev1) / args.steps
        split = {}
        for k in range(4):
            m, n, u = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
            lib.edm_profile_read(k, ctypes.byref(m), ctypes.byref(n), ctypes.byref(u))
            split[_abi.KERNEL_NAMES[k]] = round(m.value / args.steps, 3)
        hist = np.bincount(optE.cpu().numpy(), minlength=E_max + 1)[1:].tolist()
        value = float(N) * N / (ms / 1e3)
        line = {"sweep": args.sweep, "N": N, "T": T, "ms_per_step": ms, "pairs_per_s": value,
                "steps": args.steps, "warmup": 1, "kernels_ms": split,
                "lookup_tiles": "global/L2" if T > 3103 else "shared memory", "optE_histogram": hist,
                "data": "synthetic coupled logistic maps, density min(5%, 10/N), b_max 0.02"}
        # the paper's GPU-over-CPU comparison along T: the FP64 oracle on the
        # host cores (bounded sample, extrapolated), up to 10,000 steps (a
        # longer series takes minutes of CPU time per point)
        if args.sweep == "steps" and T <= 10000 and not args.no_cpu:
            cb = cpu_baseline(Y, optE.cpu().numpy(), args.cpu_rows, N, E_max)
            line["cpu_baseline"] = cb
            line["speedup_vs_cpu"] = value / cb["value"]
        print(json.dumps(line), flush=True)
        del Yd, rho, ws
        torch.cuda.empty_cache()
    return 0


def bench_self_scheduled(args, lib, edm, _abi, torch, edm_synth, dist, world, rank, local):
    """One problem over all ranks (strong scaling): the paper's self-scheduled
    decomposition (Sec. III-C) with the CUDA entry points -- every rank takes
    the next block of series (phase 1), then, after every block's optE is in
    the store (the paper's broadcast), the next block of library rows
    (phase 2), writing its own columns of a target-major rho; no data-path
    collective.  A step is one full run; `value` = N^2 / (max over ranks of
    the step time)."""
    from paper_2011_11082_gb300.sharding import run_self_scheduled

    dev = torch.device("cuda", local)
    N, T, dens, bmax, E_max = WORKLOADS[args.workload]
    Y = edm_synth.coupled_logistic(N, T, dens, bmax, seed_data=0, seed_noise=1)  # the same problem on every rank
    Yd = torch.from_numpy(Y).to(dev)
    rho = torch.empty((N, N), dtype=torch.float32, device=dev)
    ws = torch.empty(edm.edm_ccm_workspace_bytes(N, T), dtype=torch.uint8, device=dev)
    store = dist.distributed_c10d._get_default_store() if dist else None
    if store is None:
        import torch.distributed as tdist

        store = tdist.HashStore()  # one rank: a local store
    stream = torch.cuda.current_stream(dev)

    def opt(Yb):
        e, _ = edm.edm_optimal_E(Yb, E_max=E_max, return_rho=False)
        return e.cpu().numpy()

    def rows(Yf, optE, lo, hi):
        edm.edm_ccm_rho(Yd, optE.to(dev), lib_begin=lo, lib_count=hi - lo, out=rho[:, lo:hi], workspace=ws)
        return hi - lo

    def step(k):
        _, mine = run_self_scheduled(Yd, opt, rows, store, block=args.lib_block, phase1_block=args.series_block,
                                     tag=f"bench/{k}")
        return mine

    k = 0
    for _ in range(args.warmup):
        step(k)
        k += 1
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    blocks = 0
    for _ in range(args.steps):
        blocks += len(step(k))
        k += 1
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    if rank == 0:
        line = {"metric": METRIC, "value": float(N) * N / (ms / 1e3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "N": N, "T": T, "E_max": E_max, "tau": 1, "Tp": 1,
                           "partition": "self-scheduled blocks: phase 1 by series, optE through the store, "
                                        "phase 2 by library rows",
                           "series_block": args.series_block, "lib_block": args.lib_block,
                           "l2": "inputs larger than L2 (series 0.6 GB, rho 41 GB)"},
                "blocks_rank0": blocks, "e2e": None, "cpu_baseline": None, "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n101729_t1500", choices=sorted(WORKLOADS) + [BATCHED])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--lookup", default="chunked", choices=["chunked", "scalar"],
                    help="phase-2 gather kernels: 16-byte chunked (default) or scalar (comparison)")
    ap.add_argument("--knn", default="auto", choices=["auto", "warp"],
                    help="kNN tables: thread-per-query kernel where it applies (auto) or warp-per-query only")
    ap.add_argument("--cpu-rows", type=int, default=0, help="library rows the oracle times (0: 2 x cores)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp16", action="store_true", help="skip the FP16-target sub-record of an FP32 run")
    ap.add_argument("--no-backward", action="store_true", help="batched workload: skip timing the adjoint")
    ap.add_argument("--partition", default="replicas", choices=["replicas", "self"],
                    help="N > 1: independent problems per rank (replicas, weak scaling) or one problem "
                         "self-scheduled over the ranks in blocks (self, strong scaling)")
    ap.add_argument("--series-block", type=int, default=8192, help="--partition self: series per phase-1 block")
    ap.add_argument("--lib-block", type=int, default=4096, help="--partition self: library rows per phase-2 block")
    ap.add_argument("--sweep", default=None, choices=sorted(SWEEPS),
                    help="dataset-size sweep (one JSON line per size) instead of the benchmark line")
    ap.add_argument("--size", default=None, help="with --sweep: one size NxT instead of the sweep's list")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import edm_synth
    import paper_2011_11082_gb300 as edm
    from paper_2011_11082_gb300 import _abi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    lib = _abi.load()
    if args.workload == BATCHED:
        return bench_batched(args, lib, edm, _abi, torch, edm_synth)
    if args.partition == "self":
        return bench_self_scheduled(args, lib, edm, _abi, torch, edm_synth, dist, world, rank, local)
    if args.sweep:
        return bench_sweep(args, lib, edm, _abi, torch, edm_synth)

    N, T, dens, bmax, E_max = WORKLOADS[args.workload]
    # independent problems per rank (weak scaling): rank r uses data seed r
    Y = edm_synth.coupled_logistic(N, T, dens, bmax, seed_data=rank, seed_noise=1 + rank)
    Yd = torch.from_numpy(Y).to(dev)
    prec = edm.EDM_PRECISION_FP16_TARGETS if args.precision == "fp16" else edm.EDM_PRECISION_FP32
    flags = (edm.EDM_FLAG_LOOKUP_SCALAR if args.lookup == "scalar" else 0) | \
        (edm.EDM_FLAG_KNN_WARP if args.knn == "warp" else 0)
    rho = torch.empty((N, N), dtype=torch.float32, device=dev)
    ws = torch.empty(edm.edm_ccm_workspace_bytes(N, T, precision=prec), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(prec_k, ws_k, warmup, steps):
        """W warm-up steps, then K steps between events on the launching
        stream (barrier + synchronize on both sides), clocks sampled during
        the timed region; per-kernel times from per-launch events."""
        def step():
            optE, _ = edm.edm_optimal_E(Yd, E_max=E_max, return_rho=False)
            edm.edm_ccm_rho(Yd, optE, precision=prec_k, out=rho, workspace=ws_k, flags=flags)
            return optE

        for _ in range(warmup):
            optE = step()
        torch.cuda.synchronize()
        launches0 = [lib.edm_launch_count(k) for k in range(4)]
        lib.edm_profile_enable(1)
        for k in range(4):
            lib.edm_profile_read(k, None, None, None)
        clocks = ClockSampler(local)
        clocks.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            optE = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = clocks.stop()
        lib.edm_profile_enable(0)
        ms = ev0.elapsed_time(ev1) / steps
        launches = sum(lib.edm_launch_count(k) - launches0[k] for k in range(4))
        prof = {}
        for k in range(4):
            m, n, u = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
            lib.edm_profile_read(k, ctypes.byref(m), ctypes.byref(n), ctypes.byref(u))
            prof[_abi.KERNEL_NAMES[k]] = {"ms": m.value / steps, "launches": n.value / steps, "units": u.value / steps}
        if dist:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, prof, clk, launches, optE

    def smem_roofline(prof, optE, s_y, clk):
        """The bound that holds: the lookup reads every gathered value from
        shared memory (peak = 128 B/clk/SM x SMs x the SM clock seen)."""
        hist_now = np.bincount(optE.cpu().numpy(), minlength=E_max + 1)[1:]
        sm_bytes = _smem_gather_bytes(hist_now, T, 1, s_y, N)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        clk_hz = (clk.get("sm_mhz") or 2070.0) * 1e6
        sm_peak = SMEM_BYTES_PER_CLK * n_sm * clk_hz / 1e12
        lk_ms = prof["lookup_kernel"]["ms"]
        sm_ach = sm_bytes / (lk_ms / 1e3) / 1e12 if lk_ms > 0 else 0.0
        return {"bound": "smem", "achieved": sm_ach, "peak": sm_peak, "unit": "TB/s", "frac": sm_ach / sm_peak,
                "kernel": "lookup_kernel", "bytes_per_step": sm_bytes,
                "peak_from": f"{SMEM_BYTES_PER_CLK:.0f} B/clk/SM x {n_sm} SMs x {clk_hz / 1e6:.0f} MHz"}

    # parity sample: the library rows (and series) the oracle leg computes
    cpu_rows = args.cpu_rows if args.cpu_rows > 0 else 2 * (len(os.sched_getaffinity(0)) or 1)
    par_rows = torch.from_numpy(sample_rows_of(N, cpu_rows)).to(dev)

    ms, prof, clk, launches, optE = timed(prec, ws, args.warmup, args.steps)
    value = world * float(N) * N / (ms / 1e3)
    gpu_cols = rho.index_select(1, par_rows).cpu().numpy()
    gpu_optE_rows = optE.index_select(0, par_rows).cpu().numpy()

    # roofline of the dominant kernel (lookup): algorithmic bytes / time
    peak, peak_kind = _peaks()
    s_y = 2.0 if args.precision == "fp16" else 4.0
    bpp = _algorithmic_bytes_per_pair(N, T, s_y)
    lk = prof["lookup_kernel"]
    lk_launches = max(1, lk["launches"])
    per_launch_bytes = lk["units"] * bpp / lk_launches
    per_launch_s = lk["ms"] / 1e3 / lk_launches
    achieved = per_launch_bytes / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": _measured_traffic(args.workload, args.precision, lk["units"] / lk_launches),
                "peak_kind": peak_kind,
                "kernel": "lookup_kernel", "bytes_per_pair": bpp,
                "path_frac": (N * float(N) * bpp / (ms / 1e3) / 1e9) / peak}
    roofline_smem = smem_roofline(prof, optE, s_y, clk)

    # the FP16-target form on the same workload and steps (FP32 runs stay the
    # headline): its step time, kernel split and shared-memory roofline
    fp16 = None
    f16_cols = None
    if args.precision == "fp32" and not args.no_fp16:
        p16 = edm.EDM_PRECISION_FP16_TARGETS
        ws16 = ws if ws.numel() >= edm.edm_ccm_workspace_bytes(N, T, precision=p16) else \
            torch.empty(edm.edm_ccm_workspace_bytes(N, T, precision=p16), dtype=torch.uint8, device=dev)
        # at most 5 timed steps: a sub-record, and each step of the full-size
        # workload is about 13 s (the FP32 headline keeps every step asked for)
        steps16 = min(args.steps, 5)
        ms16, prof16, clk16, launches16, optE16 = timed(p16, ws16, min(args.warmup, 3), steps16)
        f16_cols = rho.index_select(1, par_rows).cpu().numpy()
        fp16 = {"ms_per_step": ms16, "value": world * float(N) * N / (ms16 / 1e3), "unit": UNIT,
                "steps": steps16, "warmup": min(args.warmup, 3), "speedup_vs_fp32": ms / ms16,
                "lookup_speedup_vs_fp32": prof["lookup_kernel"]["ms"] / max(1e-9, prof16["lookup_kernel"]["ms"]),
                "dtype": "f16-targets/f32-accumulate", "kernels": prof16,
                "roofline_smem": smem_roofline(prof16, optE16, 2.0, clk16), "clocks": clk16,
                "gpu_launches": launches16}
        del ws16

    # end to end through the public API with host buffers: edm_ccm_host
    # copies the series in, runs both phases and streams rho back to the host
    # (all inside the timed region)
    e2e = None
    if not args.no_e2e:
        try:
            del ws
            torch.cuda.empty_cache()
            Yh = torch.from_numpy(Y).pin_memory()
            try:
                rho_h = torch.empty((N, N), dtype=torch.float32, pin_memory=True)
                pinned = True
            except Exception:
                rho_h = torch.empty((N, N), dtype=torch.float32)
                pinned = False
            e_ws = None
            for _ in range(1):  # warm-up of the host path (allocates its workspace)
                p = edm.make_params(E_max=E_max, precision=prec, flags=flags)
                need = int(lib.edm_ccm_host_workspace_bytes(N, T, 0, ctypes.byref(p)))
                e_ws = torch.empty(need, dtype=torch.uint8, device=dev)
            e2e_steps = max(1, min(args.steps, 2))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                edm.edm_ccm_host(Yh, E_max=E_max, precision=prec, rho_out=rho_h, workspace=e_ws)
            torch.cuda.synchronize()
            ems = (time.perf_counter() - t0) * 1e3 / e2e_steps
            if dist:
                t = torch.tensor([ems], device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                ems = float(t.item())
            e2e = {"value": world * float(N) * N / (ems / 1e3), "unit": UNIT, "ms_per_step": ems,
                   "h2d_bytes_per_step": int(Y.nbytes), "d2h_bytes_per_step": int(N * N * 4 + N * 4),
                   "host_buffers": "pinned" if pinned else "pageable", "api": "edm_ccm_host"}
            del rho_h
        except Exception as ex:  # pragma: no cover
            e2e = {"value": None, "unit": UNIT, "error": repr(ex)[:200]}

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        keep = {}
        cpu = cpu_baseline(Y, optE.cpu().numpy(), cpu_rows, N, E_max, keep=keep)
        parity = parity_record(gpu_cols, gpu_optE_rows, keep, 1e-4)
        if fp16 is not None:
            fp16["parity"] = parity_record(f16_cols, gpu_optE_rows, keep, 1e-3)

    if rank == 0:
        hist = np.bincount(optE.cpu().numpy(), minlength=E_max + 1)[1:].tolist()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f16-targets/f32-accumulate",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "T": T, "E_max": E_max, "tau": 1, "Tp": 1,
                       "precision": args.precision, "lookup": args.lookup, "knn": args.knn, "l2": "inputs larger than L2 (series 0.6 GB, rho 41 GB)",
                       "optE_histogram": hist},
            "roofline": roofline, "roofline_smem": roofline_smem, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches, "kernels": prof, "parity": parity, "fp16": fp16,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
