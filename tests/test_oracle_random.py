"""The oracle against the independent brute force on seeded random draws of
the method's parameters (series length, E per target, tau, Tp, exclusion
radius, lag ranges, candidate subsets), on continuous series and on
quantised series full of exact distance ties (the tie rule: ascending
(d^2, candidate time)).  Complements the fixed grids of the oracle pins."""

import numpy as np
import pytest

import brute_force as bf
from oracle import oracle as orc

CASES = 24


def _series(rng, N, T, quantised):
    Y = rng.standard_normal((N, T))
    if quantised:
        Y = np.round(Y * 2.0) / 2.0  # a few distinct values: many exact ties
    return Y


def _draw(rng):
    tau = int(rng.integers(1, 4))
    Tp = int(rng.integers(0, 4))
    excl = int(rng.choice([-1, 0, 1, 3]))
    T = int(rng.integers(24, 61))
    return tau, Tp, excl, T


def _max_E(T, tau, Tp, excl):
    # largest E whose table still has E + 1 candidates beyond the exclusion window
    E = 1
    while E < 5:
        n = T - Tp - E * tau - (2 * excl + 1 if excl >= 0 else 0)
        if n < E + 2:
            break
        E += 1
    return E


@pytest.mark.parametrize("quantised", [False, True])
def test_ccm_matrix_random_parameters(quantised):
    rng = np.random.default_rng(101 if quantised else 100)
    for case in range(CASES):
        tau, Tp, excl, T = _draw(rng)
        N = int(rng.integers(2, 4))
        Y = _series(rng, N, T, quantised)
        E_hi = _max_E(T, tau, Tp, excl)
        optE = rng.integers(1, E_hi + 1, size=N).astype(np.int32)
        R = orc.ccm_rho_rows(Y, optE, tau=tau, Tp=Tp, excl=excl, nthreads=1)
        B = bf.ccm_matrix(Y, optE, tau=tau, Tp=Tp, excl=excl)
        both_nan = np.isnan(R) & np.isnan(B)
        assert np.all(both_nan | (np.abs(R - B) < 1e-12)), (case, tau, Tp, excl, T, optE, R, B)
        # the tables themselves, indices exactly
        for i in range(N):
            E = int(optE[0])
            oi, ow = orc.ccm_table(Y[i], E, tau, Tp, excl)
            bi, bw, _ = bf.ccm_table(Y[i], E, tau, Tp, excl)
            assert np.array_equal(oi, bi), (case, i, E)
            assert np.allclose(ow, bw, rtol=0, atol=1e-14)


@pytest.mark.parametrize("quantised", [False, True])
def test_simplex_random_parameters(quantised):
    rng = np.random.default_rng(201 if quantised else 200)
    for case in range(CASES):
        tau = int(rng.integers(1, 3))
        Tp = int(rng.integers(0, 3))
        T = int(rng.integers(40, 81))
        x = _series(rng, 1, T, quantised)[0]
        for E in range(1, 4):
            if T // 2 - Tp - (E - 1) * tau < E + 1 or (T - T // 2) - Tp - (E - 1) * tau < 2:
                continue
            a = orc.simplex_rho(x, E, tau, Tp)
            b = bf.simplex_rho(x, E, tau, Tp)
            assert (np.isnan(a) and np.isnan(b)) or abs(a - b) < 1e-12, (case, E, tau, Tp, a, b)


def test_lags_random_parameters():
    rng = np.random.default_rng(300)
    for case in range(CASES):
        tau = int(rng.integers(1, 3))
        excl = int(rng.choice([-1, 0, 2]))
        T = int(rng.integers(36, 61))
        lag_min = int(rng.integers(-3, 2))
        lag_max = lag_min + int(rng.integers(0, 4))
        N = 2
        Y = _series(rng, N, T, quantised=bool(case % 2))
        optE = rng.integers(1, 4, size=N).astype(np.int32)
        R = orc.ccm_rho_lags(Y, optE, lag_min, lag_max, tau=tau, excl=excl, nthreads=1)
        for i in range(N):
            for j in range(N):
                b = bf.ccm_lags_pair(Y[i], Y[j], int(optE[j]), list(range(lag_min, lag_max + 1)), tau, excl)
                got = R[:, i, j]
                ok = (np.isnan(got) & np.isnan(b)) | (np.abs(got - b) < 1e-12)
                assert ok.all(), (case, i, j, got, b)


def test_subsets_random_masks():
    rng = np.random.default_rng(400)
    for case in range(CASES // 2):
        T = int(rng.integers(40, 61))
        excl = int(rng.choice([-1, 0, 1]))
        N = 2
        Y = _series(rng, N, T, quantised=bool(case % 2))
        optE = rng.integers(1, 4, size=N).astype(np.int32)
        words = (T + 31) // 32
        allowed = rng.random(T) < 0.6
        allowed[: T // 3 + 10] = True  # enough candidates for every query
        mask = np.zeros(words, np.uint32)
        for s in np.nonzero(allowed)[0]:
            mask[s // 32] |= np.uint32(1 << (s % 32))
        R = orc.ccm_rho_subsets(Y, optE, mask[None, :], excl=excl, nthreads=1)
        times = set(int(s) for s in np.nonzero(allowed)[0])
        for i in range(N):
            for j in range(N):
                b = bf.ccm_pair_subset(Y[i], Y[j], int(optE[j]), times, excl=excl)
                a = R[0, i, j]
                assert (np.isnan(a) and np.isnan(b)) or abs(a - b) < 1e-12, (case, i, j, a, b)
