"""The seeded generator: deterministic, z-normalised, inside (0,1) before noise."""

import numpy as np
import pytest

import edm_synth as synth


def test_deterministic_and_normalised():
    a = synth.workload("n64_t500")
    b = synth.workload("n64_t500")
    assert a.dtype == np.float32 and a.shape == (64, 500)
    assert np.array_equal(a, b)
    assert np.allclose(a.mean(axis=1), 0.0, atol=1e-5)
    assert np.allclose(a.std(axis=1), 1.0, atol=1e-4)


def test_coupling_density_and_diagonal():
    Y, meta = synth.coupled_logistic(400, 50, 0.05, 0.05, seed_data=3, seed_noise=4, return_meta=True)
    nnz = meta["rows"].size
    expect = 400 * 399 * 0.05
    assert abs(nnz - expect) < 5 * np.sqrt(expect)
    assert np.all(meta["rows"] != meta["cols"])
    assert np.all((meta["vals"] >= 0) & (meta["vals"] <= 0.05))
    flat = meta["rows"] * 400 + meta["cols"]
    assert np.unique(flat).size == flat.size


def test_guard_rejects_divergent_coupling():
    with pytest.raises(RuntimeError):
        synth.coupled_logistic(50, 50, 0.5, 2.0, seed_data=1, seed_noise=2)


def test_batched_specs_ranges():
    specs = synth.batched_specs()
    assert len(specs) == 256
    assert all(32 <= s.N <= 1024 and 200 <= s.T <= 3000 for s in specs)
    assert specs == synth.batched_specs()


def test_sine_integer_period_bit_identical():
    x = synth.sine_series(100, 10)
    assert np.array_equal(x[:10], x[10:20]) and np.array_equal(x[:10], x[90:100])
