"""Host-side accounting of bench.py (no GPU): the byte counts behind the
roofline figures, the DRAM-traffic record and its validity check, and the
sweep sizes."""

import json
import os

import numpy as np

import bench


def test_algorithmic_bytes_per_pair_bench_size():
    # 4 B of rho per pair + the series read once (targets and libraries,
    # FP32) + optE, spread over N^2 pairs: 42.6 GB at N = 101,729, T = 1,500
    N, T = 101729, 1500
    bpp = bench._algorithmic_bytes_per_pair(N, T, 4.0)
    total = bpp * N * N
    assert abs(total - (4.0 * N * N + 8.0 * N * T + 4.0 * N)) < 1.0
    assert 42.5e9 < total < 42.7e9
    # FP16 targets: 2 bytes per target value
    assert bench._algorithmic_bytes_per_pair(N, T, 2.0) < bpp


def test_smem_gather_bytes_counts_gathers_and_observation():
    # one target of E = 2 at T = 10, Tp = 1: rows t = 1..8 (8 rows), each
    # reads E + 1 = 3 gathered values and 1 observation; N libraries
    hist = np.zeros(20, dtype=np.int64)
    hist[1] = 1
    got = bench._smem_gather_bytes(hist, 10, 1, 4.0, 7)
    assert got == 8 * 4 * 4.0 * 7


def test_traffic_record_matches_sources_or_is_dropped(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "lookup_dram_traffic.json")))
    e = rec["n16384_t1500/fp32"]
    assert e["bytes_per_pair"] > 4.0  # at least the rho write
    assert abs(e["bytes_per_pair"] * e["pairs_per_captured_launch"] - e["bytes_per_captured_launch"]) < 1.0
    # a stale record (other sources) gives no traffic figure
    stale = dict(rec)
    stale["n16384_t1500/fp32"] = dict(e, sources="0" * 16)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "lookup_dram_traffic.json").write_text(json.dumps(stale))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_lookup_sources_hash", lambda: "1" * 16)
    assert bench._measured_traffic("n16384_t1500", "fp32", 1e6) is None
    # a current record scales with the pairs of the launch
    monkeypatch.setattr(bench, "_lookup_sources_hash", lambda: "0" * 16)
    assert bench._measured_traffic("n16384_t1500", "fp32", 2e6) == e["bytes_per_pair"] * 2e6
    assert bench._measured_traffic("n16384_t1500", "fp16", 2e6) is None
    # no record for the full-size workload (its traffic is not scaled from the small case)
    assert bench._measured_traffic("n101729_t1500", "fp32", 2e6) is None


def test_sweep_sizes():
    # the paper's study: series at 10,000 time steps; time steps at 1,000
    # series up to 40,000
    assert all(T == 10000 for _, T in bench.SWEEPS["series"])
    assert all(N == 1000 for N, _ in bench.SWEEPS["steps"])
    assert max(T for _, T in bench.SWEEPS["steps"]) == 40000
