"""Coupled logistic maps and a few textbook series, drawn from fixed seeds.

The paper's datasets (whole-brain zebrafish calcium recordings) are not
available, so the workloads use a standard stand-in for a large nonlinear
dynamical network: N logistic maps with sparse, weak, one-way couplings,

    x_i(t+1) = x_i(t) * (r_i - r_i * x_i(t) - sum_j b_ij * x_j(t)),

observed with additive Gaussian noise and z-normalised per series.

Draw order (numpy PCG64, ``default_rng(seed_data)``): growth rates r, then
the coupling pattern, then the coupling values, then the initial states; the
trajectory is deterministic; the observation noise comes from a second
generator ``default_rng(seed_noise)``.  The coupling pattern makes every
off-diagonal entry nonzero independently with probability ``density``; it is
drawn as geometric gaps between successes over the flattened off-diagonal
index space, which has exactly that distribution and costs O(nnz).
The simulation runs in float64; the returned series are float32.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

try:  # scipy is present on both machines; the dense fallback serves tiny N.
    import scipy.sparse as _sp
except Exception:  # pragma: no cover
    _sp = None


@dataclass(frozen=True)
class WorkloadSpec:
    name: str
    N: int
    T: int
    density: float
    b_max: float
    E_max: int
    tau: int = 1
    Tp: int = 1
    seed_data: int = 0
    seed_noise: int = 1
    notes: str = ""


# The five workloads.  Sizes, densities, coupling ranges and E_max follow the
# benchmark configurations; "batched" draws its 256 (N, T) pairs from seed 4.
WORKLOADS = {
    "n64_t500": WorkloadSpec("n64_t500", 64, 500, 0.05, 0.05, 10),
    "n2048_t1500": WorkloadSpec("n2048_t1500", 2048, 1500, 0.01, 0.02, 20),
    # 1% density at N=16,384 would give each map ~164 inputs and drive it out
    # of (0,1); 0.1% keeps ~16 inputs per map, as in the N=2,048 workload.
    "n16384_t1500": WorkloadSpec("n16384_t1500", 16384, 1500, 0.001, 0.02, 20),
    "n101729_t1500": WorkloadSpec("n101729_t1500", 101729, 1500, 0.0001, 0.02, 20),
}


def _coupling(rng: np.random.Generator, N: int, density: float, b_max: float):
    """Sparse coupling matrix: rows, cols, values (b_ii = 0)."""
    n_off = N * (N - 1)
    if density <= 0.0 or n_off == 0:
        return (np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0))
    # Geometric gaps between Bernoulli(density) successes over [0, n_off).
    expect = n_off * density
    chunk = int(expect + 10.0 * np.sqrt(expect) + 64)
    pos_parts = []
    last = -1
    while True:
        gaps = rng.geometric(density, size=chunk).astype(np.int64)
        cs = last + np.cumsum(gaps)
        keep = cs < n_off
        pos_parts.append(cs[keep])
        if not keep.all():
            break
        last = int(cs[-1])
    pos = np.concatenate(pos_parts)
    rows = pos // (N - 1)
    colp = pos % (N - 1)
    cols = colp + (colp >= rows)  # skip the diagonal
    vals = rng.uniform(0.0, b_max, size=pos.size)
    return rows, cols, vals


def coupled_logistic(
    N: int,
    T: int,
    density: float,
    b_max: float,
    seed_data: int = 0,
    seed_noise: int = 1,
    r_range=(3.6, 3.9),
    burn_in: int = 200,
    noise_sigma: float = 0.01,
    return_meta: bool = False,
):
    """Return Y float32 [N][T], each row z-normalised (population std)."""
    rng = np.random.default_rng(seed_data)
    r = rng.uniform(r_range[0], r_range[1], size=N)
    rows, cols, vals = _coupling(rng, N, density, b_max)
    x = rng.uniform(0.2, 0.8, size=N)
    if _sp is not None:
        B = _sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
        matvec = B.dot
    else:  # pragma: no cover
        Bd = np.zeros((N, N))
        Bd[rows, cols] = vals
        matvec = Bd.dot
    X = np.empty((T, N), dtype=np.float64)
    for step in range(burn_in + T):
        if step >= burn_in:
            X[step - burn_in] = x
        x = x * (r - r * x - matvec(x))
        if not (np.all(x > 0.0) and np.all(x < 1.0)):
            raise RuntimeError(
                f"coupled logistic map left (0,1) at step {step}; "
                "the coupling range is too strong for this seed"
            )
    rng_noise = np.random.default_rng(seed_noise)
    X += rng_noise.normal(0.0, noise_sigma, size=X.shape)
    Y = np.ascontiguousarray(X.T)  # [N][T]
    mu = Y.mean(axis=1, keepdims=True)
    sd = Y.std(axis=1, keepdims=True)
    sd[sd == 0.0] = 1.0
    Y = ((Y - mu) / sd).astype(np.float32)
    if return_meta:
        return Y, {"r": r, "rows": rows, "cols": cols, "vals": vals}
    return Y


def workload(name: str) -> np.ndarray:
    s = WORKLOADS[name]
    return coupled_logistic(s.N, s.T, s.density, s.b_max, s.seed_data, s.seed_noise)


@dataclass(frozen=True)
class BatchedSpec:
    index: int
    N: int
    T: int
    seed_data: int
    seed_noise: int


def batched_specs(count: int = 256, master_seed: int = 4, n_range=(32, 1024), t_range=(200, 3000)):
    """The (N, T, seeds) of the batched workload, drawn from ``master_seed``."""
    rng = np.random.default_rng(master_seed)
    Ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    Ts = rng.integers(t_range[0], t_range[1] + 1, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=(count, 2))
    return [BatchedSpec(i, int(Ns[i]), int(Ts[i]), int(seeds[i, 0]), int(seeds[i, 1])) for i in range(count)]


def batched_dataset(spec: BatchedSpec, density: float = 0.01, b_max: float = 0.02) -> np.ndarray:
    return coupled_logistic(spec.N, spec.T, density, b_max, spec.seed_data, spec.seed_noise)


def sample_pairs(N: int, count: int, seed: int = 3):
    """``count`` (library, target) index pairs drawn uniformly with replacement."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, N, size=count)
    j = rng.integers(0, N, size=count)
    return i.astype(np.int64), j.astype(np.int64)


def sine_series(T: int, period: float, phase: float = 0.0, integer_period: bool = True) -> np.ndarray:
    """sin(2*pi*t/period + phase); with an integer period the phase index is
    taken modulo the period first so equal phases give bit-identical values."""
    t = np.arange(T, dtype=np.float64)
    if integer_period:
        p = int(period)
        t = np.mod(t, p)
    return np.sin(2.0 * np.pi * t / period + phase).astype(np.float32)


def logistic_series(T: int, r: float = 3.8, x0: float = 0.4, burn_in: int = 100) -> np.ndarray:
    x = x0
    out = np.empty(T, dtype=np.float64)
    for step in range(burn_in + T):
        if step >= burn_in:
            out[step - burn_in] = x
        x = r * x * (1.0 - x)
    return out.astype(np.float32)


def white_noise(T: int, seed: int = 7) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(T).astype(np.float32)


def library_subsets(T: int, lo: int, hi: int, sizes, samples: int, seed: int = 8) -> np.ndarray:
    """Random library subsets for the convergence test: for each size L in
    `sizes` and each of `samples` draws, L distinct times from [lo, hi]
    without replacement, as bit masks uint32[len(sizes) * samples][ceil(T/32)]
    (bit s of word s // 32 = time s allowed), size-major."""
    rng = np.random.default_rng(seed)
    words = (T + 31) // 32
    out = np.zeros((len(sizes) * samples, words), np.uint32)
    pool = np.arange(lo, hi + 1)
    for a, L in enumerate(sizes):
        for b in range(samples):
            pick = rng.choice(pool, size=int(L), replace=False)
            row = out[a * samples + b]
            np.bitwise_or.at(row, pick // 32, (np.uint32(1) << (pick % 32).astype(np.uint32)))
    return out
