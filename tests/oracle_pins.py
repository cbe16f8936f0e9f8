"""Pins that tie the FP64 oracle to facts fixed outside it.

Each pin takes an oracle library handle (``lib=None`` is the committed
oracle) so the same checks can be run against copies of the oracle with a
planted mistake.  A pin raises AssertionError when the oracle disagrees with:
  * a hand-worked example (tests/golden/knn_E1_hand.json),
  * an independent brute-force restatement on tiny inputs (brute_force.py),
  * closed forms (integer-period sine, self-inclusion, two-neighbour weights),
  * invariances (affine maps, permutations of the series),
  * textbook facts (np.corrcoef, irrational-frequency sine needs E >= 2).
"""

from __future__ import annotations

import json
import math
import os

import numpy as np

import brute_force as bf
import edm_synth as synth
from oracle import oracle as orc

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _tiny_series(seed, N=3, T=40):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, T)).astype(np.float32)


# --------------------------------------------------------------------------
def pin_hand_example(lib=None):
    g = json.load(open(os.path.join(GOLDEN, "knn_E1_hand.json")))
    x = np.array(g["series"])
    idx, w = orc.ccm_table(x, g["E"], g["tau"], g["Tp"], g["excl"], lib=lib)
    assert idx.tolist() == g["idx"], (idx.tolist(), g["idx"])
    for r, (d1, d2) in enumerate(g["dist"]):
        ratio = d2 / d1
        w1 = 1.0 / (1.0 + math.exp(1.0 - ratio))
        assert abs(w[r, 0] - w1) < 1e-15 and abs(w[r, 1] - (1.0 - w1)) < 1e-15, (r, w[r])
    pred = [w[r, 0] * g["future_of_neighbours"][r][0] + w[r, 1] * g["future_of_neighbours"][r][1] for r in range(5)]
    rho_expected = float(np.corrcoef(g["observed"], pred)[0, 1])
    rho = orc.lookup_rho(x, g["E"], idx, w, g["tau"], g["Tp"], lib=lib)
    assert abs(rho - rho_expected) < 1e-14, (rho, rho_expected)


def pin_knn_brute(lib=None):
    Y = _tiny_series(11, N=3, T=37)
    for x in Y:
        for E in (1, 2, 3, 4):
            for tau in (1, 2):
                for Tp in (0, 1, 2):
                    for excl in (0, 2) if Tp == 0 else (-1, 0, 2):
                        idx, w = orc.ccm_table(x, E, tau, Tp, excl, lib=lib)
                        bidx, bw, _ = bf.ccm_table(x, E, tau, Tp, excl)
                        assert np.array_equal(idx, bidx), (E, tau, Tp, excl)
                        assert np.allclose(w, bw, rtol=0, atol=1e-14), (E, tau, Tp, excl)


def pin_generic_knn_brute(lib=None):
    """Cross-series kNN (phase-1 shape: queries from one series, candidates from another)."""
    Y = _tiny_series(12, N=2, T=30)
    for E in (1, 2, 3):
        L = E - 1
        idx, d2 = orc.knn(Y[0], L, 28, Y[1], L, 25, E, tau=1, same=False, excl=-1, lib=lib)
        Vq = bf.embed(Y[0], E, 1)[: 29 - L]
        Vc = bf.embed(Y[1], E, 1)[: 26 - L]
        bidx, bd2 = bf.neighbours(bf.distance_matrix(Vq, Vc), np.arange(L, 26), E + 1)
        assert np.array_equal(idx, bidx)
        assert np.array_equal(d2, bd2)


def pin_simplex_brute(lib=None):
    # an even and an odd length: the split point is floor(T/2)
    Y = list(_tiny_series(13, N=2, T=48)) + list(_tiny_series(15, N=2, T=47))
    for x in Y:
        for E in (1, 2, 3, 4):
            for Tp in (1, 2):
                a = orc.simplex_rho(x, E, 1, Tp, lib=lib)
                b = bf.simplex_rho(x, E, 1, Tp)
                assert abs(a - b) < 1e-12, (E, Tp, a, b)
    x = synth.logistic_series(60)
    optE, rho = orc.optimal_E(x[None, :], 6, lib=lib)
    bE, brho = bf.optimal_E(x, 6)
    assert optE[0] == bE and np.allclose(rho[0], brho, atol=1e-12)


def pin_ccm_matrix_brute(lib=None):
    Y = _tiny_series(14, N=4, T=36)
    optE = np.array([1, 3, 2, 3], np.int32)
    for Tp, excl in ((1, 0), (1, 3), (2, -1)):
        R = orc.ccm_rho_rows(Y, optE, Tp=Tp, excl=excl, nthreads=2, lib=lib)
        B = bf.ccm_matrix(Y, optE, Tp=Tp, excl=excl)
        assert np.allclose(R, B, rtol=0, atol=1e-12), (Tp, excl, np.abs(R - B).max())
    li = np.array([0, 3, 2, 1, 0])
    lj = np.array([1, 0, 2, 3, 0])
    P = orc.ccm_rho_pairs(Y, optE, li, lj, lib=lib)
    assert np.allclose(P, bf.ccm_matrix(Y, optE)[li, lj], rtol=0, atol=1e-12)


def pin_pearson_textbook(lib=None):
    rng = np.random.default_rng(3)
    a = rng.standard_normal(101)
    b = 0.3 * a + rng.standard_normal(101)
    assert abs(orc.pearson(a, b, lib=lib) - np.corrcoef(a, b)[0, 1]) < 1e-14
    assert math.isnan(orc.pearson(np.ones(10), b[:10], lib=lib))


def pin_weights_closed_form(lib=None):
    for d1, d2 in ((1.0, 1.0), (0.5, 2.0), (2.0, 3.0)):
        w = orc.weights(np.array([d1 * d1, d2 * d2]), lib=lib)
        w1 = 1.0 / (1.0 + math.exp(1.0 - d2 / d1))
        assert abs(w[0] - w1) < 1e-15 and abs(w[1] - (1 - w1)) < 1e-15
    # d_1 = 0: only exact duplicates keep weight, shared equally.
    w = orc.weights(np.array([0.0, 0.0, 0.25, 1.0]), lib=lib)
    assert np.array_equal(w, [0.5, 0.5, 0.0, 0.0])
    w = orc.weights(np.array([1.0, 4.0, 9.0]), lib=lib)
    assert abs(w.sum() - 1.0) < 1e-15 and w[0] > w[1] > w[2]


def pin_integer_period_sine(lib=None):
    """A series of integer period P: every embedded point has exact duplicates
    one or more periods away, so d_1 = 0 and the forecast is exact: rho = 1."""
    P = 12
    for E in (2, 3, 5):
        T = (E + 4) * P + E + 1
        x = synth.sine_series(T, P)
        c = np.cos(2 * np.pi * np.mod(np.arange(T), P) / P).astype(np.float32)
        idx, w = orc.ccm_table(x, E, lib=lib)
        for y in (x, c):
            rho = orc.lookup_rho(y, E, idx, w, lib=lib)
            assert abs(rho - 1.0) < 1e-12, (E, rho)


def pin_self_inclusion_exact(lib=None):
    """Tp = 0 and no exclusion: each query is its own nearest neighbour at
    distance 0, takes all the weight, and the prediction is the observation."""
    x = synth.logistic_series(400)
    for E in (1, 2, 4):
        idx, w = orc.ccm_table(x, E, Tp=0, excl=-1, lib=lib)
        rho = orc.lookup_rho(x, E, idx, w, Tp=0, lib=lib)
        assert rho == 1.0, (E, rho)


def pin_affine_invariance(lib=None):
    Y = synth.coupled_logistic(3, 150, 0.3, 0.05, seed_data=5, seed_noise=6).astype(np.float64)
    optE = np.array([2, 3, 2], np.int32)
    R = orc.ccm_rho_rows(Y, optE, nthreads=1, lib=lib)
    Z = Y.copy()
    Z[0] = 2.5 * Y[0] + 7.0  # library-and-target 0 scaled and shifted
    Z[1] = -0.5 * Y[1] - 1.0  # a negative scale too
    R2 = orc.ccm_rho_rows(Z, optE, nthreads=1, lib=lib)
    # A library map a*x+b scales every distance by |a| (same neighbours, same
    # ratios d_n/d_1, same weights); a target map c*y+d maps the prediction
    # and the observation alike (the weights sum to one), so rho is unchanged
    # for any a, c != 0.
    assert np.allclose(R2, R, rtol=0, atol=1e-10), np.abs(R2 - R).max()


def pin_permutation_equivariance(lib=None):
    Y = synth.coupled_logistic(6, 120, 0.2, 0.05, seed_data=8, seed_noise=9)
    optE = np.array([1, 2, 3, 2, 1, 4], np.int32)
    R = orc.ccm_rho_rows(Y, optE, nthreads=1, lib=lib)
    perm = np.array([3, 0, 5, 1, 4, 2])
    Rp = orc.ccm_rho_rows(Y[perm], optE[perm], nthreads=1, lib=lib)
    assert np.array_equal(Rp, R[np.ix_(perm, perm)])


def pin_logistic_self_crossmap(lib=None):
    """Noise-free logistic map, library = target, leave-one-out, Tp = 1."""
    x = synth.logistic_series(1500)
    idx, w = orc.ccm_table(x, 1, lib=lib)
    rho = orc.lookup_rho(x, 1, idx, w, lib=lib)
    assert rho > 0.99998, rho


def pin_white_noise(lib=None):
    T = 800
    a = synth.white_noise(T, seed=21)
    b = synth.white_noise(T, seed=22)
    idx, w = orc.ccm_table(a, 2, lib=lib)
    rho = orc.lookup_rho(b, 2, idx, w, lib=lib)
    assert abs(rho) < 4.0 / math.sqrt(T), rho
    assert abs(orc.simplex_rho(a, 2, lib=lib)) < 6.0 / math.sqrt(T / 2)


def pin_optE_sine(lib=None):
    """E = 1 cannot tell the rising branch of a sine from the falling one."""
    x = synth.sine_series(600, 2 * math.pi * 3.1, integer_period=False)
    optE, rho = orc.optimal_E(x[None, :], 5, lib=lib)
    assert optE[0] >= 2 and rho[0, 1] > rho[0, 0], (optE, rho)
    # integer period: every E >= 2 forecasts exactly; ties go to the smaller E
    x = synth.sine_series(400, 16)
    optE, rho = orc.optimal_E(x[None, :], 6, lib=lib)
    assert optE[0] == 2, (optE, rho)


def pin_optE_logistic(lib=None):
    x = synth.logistic_series(1000)
    optE, rho = orc.optimal_E(x[None, :], 6, lib=lib)
    assert optE[0] in (1, 2), (optE, rho)


def pin_direction(lib=None):
    """x drives y one way: y's manifold predicts x better than the reverse,
    i.e. rho(library y -> target x) > rho(library x -> target y)."""
    T = 1000
    x = np.empty(T + 100)
    y = np.empty(T + 100)
    x[0], y[0] = 0.4, 0.2
    for t in range(T + 99):
        x[t + 1] = x[t] * (3.8 - 3.8 * x[t])
        y[t + 1] = y[t] * (3.5 - 3.5 * y[t] - 0.1 * x[t])
    Y = np.stack([x[100:], y[100:]])
    optE = np.array([2, 2], np.int32)
    R = orc.ccm_rho_rows(Y, optE, nthreads=1, lib=lib)
    assert R[1, 0] > R[0, 1] + 0.05, R


def pin_lags_brute(lib=None):
    """Time-delay cross mapping against the per-pair brute force, negative,
    zero and positive lags, with and without exclusion."""
    Y = _tiny_series(15, N=3, T=44)
    optE = np.array([2, 1, 3], np.int32)
    for lag_min, lag_max, excl in ((-3, 2, 0), (0, 4, 1), (-2, -1, -1)):
        R = orc.ccm_rho_lags(Y, optE, lag_min, lag_max, excl=excl, nthreads=2, lib=lib)
        lags = list(range(lag_min, lag_max + 1))
        for i in range(3):
            for j in range(3):
                b = bf.ccm_lags_pair(Y[i], Y[j], int(optE[j]), lags, excl=excl)
                assert np.allclose(R[:, i, j], b, rtol=0, atol=1e-12, equal_nan=True), (lag_min, i, j)


def pin_lags_reduce_to_ccm(lib=None):
    """A single lag l = Tp >= 0 is the plain cross map with that horizon."""
    Y = _tiny_series(16, N=4, T=60)
    optE = np.array([2, 3, 1, 2], np.int32)
    for Tp in (0, 1, 2):
        R = orc.ccm_rho_lags(Y, optE, Tp, Tp, excl=0 if Tp else -1, nthreads=2, lib=lib)
        P = orc.ccm_rho_rows(Y, optE, Tp=Tp, excl=0 if Tp else -1, nthreads=2, lib=lib)
        assert np.array_equal(R[0], P), Tp


def pin_lags_integer_period_sine(lib=None):
    """Integer period: exact duplicates predict every lag exactly (rho = 1)."""
    P = 10
    x = synth.sine_series(8 * P + 6, P)
    Y = np.stack([x, x])
    R = orc.ccm_rho_lags(Y, np.array([3, 3], np.int32), -4, 4, nthreads=1, lib=lib)
    assert np.all(np.abs(R - 1.0) < 1e-12), R


def _mask_times(mask_row, T):
    return {s for s in range(T) if (int(mask_row[s // 32]) >> (s % 32)) & 1}


def pin_subsets_brute(lib=None):
    """Convergence cross map (library subsets) against the per-pair brute
    force, with and without exclusion."""
    Y = _tiny_series(17, N=3, T=48)
    optE = np.array([2, 1, 3], np.int32)
    masks = synth.library_subsets(48, 2, 46, sizes=(14, 30), samples=2, seed=5)
    for excl in (0, 2):
        R = orc.ccm_rho_subsets(Y, optE, masks, excl=excl, nthreads=2, lib=lib)
        for u in range(masks.shape[0]):
            allowed = _mask_times(masks[u], 48)
            for i in range(3):
                for j in range(3):
                    b = bf.ccm_pair_subset(Y[i], Y[j], int(optE[j]), allowed, excl=excl)
                    assert abs(R[u, i, j] - b) < 1e-12, (excl, u, i, j)


def pin_subsets_full_library_is_ccm(lib=None):
    """Every candidate allowed: exactly the plain cross map."""
    Y = _tiny_series(18, N=4, T=70)
    optE = np.array([2, 3, 1, 2], np.int32)
    full = np.full((1, 3), 0xFFFFFFFF, np.uint32)
    R = orc.ccm_rho_subsets(Y, optE, full, nthreads=2, lib=lib)
    assert np.array_equal(R[0], orc.ccm_rho_rows(Y, optE, nthreads=2, lib=lib))


ALL_PINS = [
    pin_hand_example,
    pin_knn_brute,
    pin_generic_knn_brute,
    pin_simplex_brute,
    pin_ccm_matrix_brute,
    pin_pearson_textbook,
    pin_weights_closed_form,
    pin_integer_period_sine,
    pin_self_inclusion_exact,
    pin_affine_invariance,
    pin_permutation_equivariance,
    pin_logistic_self_crossmap,
    pin_white_noise,
    pin_optE_sine,
    pin_optE_logistic,
    pin_direction,
    pin_lags_brute,
    pin_lags_reduce_to_ccm,
    pin_lags_integer_period_sine,
    pin_subsets_brute,
    pin_subsets_full_library_is_ccm,
]
