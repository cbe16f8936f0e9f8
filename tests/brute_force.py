"""Independent brute-force restatement of the method for tiny inputs.

Written separately from the C oracle and structured differently: embeddings
are materialised as matrices, the full query x candidate distance matrix is
formed, neighbours are ordered with a stable lexicographic sort, every pair
of the CCM matrix rebuilds its own table (the per-pair form of Algorithm 1,
not the per-library reuse of Algorithm 2), and correlations come from
numpy.corrcoef.  Used only as a pin for the oracle.
"""

from __future__ import annotations

import numpy as np


def embed(x: np.ndarray, E: int, tau: int) -> np.ndarray:
    """Row r <-> time t = (E-1)*tau + r; column m = x(t - m*tau)."""
    x = np.asarray(x, dtype=np.float64)
    L = (E - 1) * tau
    T = x.size
    cols = [x[L - m * tau: T - m * tau] for m in range(E)]
    return np.stack(cols, axis=1)


def distance_matrix(Vq: np.ndarray, Vc: np.ndarray) -> np.ndarray:
    D = np.zeros((Vq.shape[0], Vc.shape[0]))
    for m in range(Vq.shape[1]):
        diff = Vq[:, m][:, None] - Vc[:, m][None, :]
        D = D + diff * diff
    return D


def neighbours(D: np.ndarray, cand_times: np.ndarray, k: int, mask=None):
    """Per row: the k smallest (distance, candidate time), ascending."""
    idx = np.zeros((D.shape[0], k), np.int64)
    d2 = np.zeros((D.shape[0], k))
    for q in range(D.shape[0]):
        row = D[q].copy()
        times = cand_times.copy()
        if mask is not None:
            keep = mask[q]
            row, times = row[keep], times[keep]
        order = np.lexsort((times, row))[:k]
        idx[q] = times[order]
        d2[q] = row[order]
    return idx, d2


def exp_weights(d2_row: np.ndarray) -> np.ndarray:
    d = np.sqrt(d2_row)
    if d[0] > 0:
        u = np.exp(-d / d[0])
    else:
        u = (d == 0).astype(np.float64)
    return u / u.sum()


def corr(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size < 2 or np.all(a == a[0]) or np.all(b == b[0]):
        return float("nan")
    return float(np.corrcoef(a, b)[0, 1])


def ccm_table(x, E, tau=1, Tp=1, excl=0):
    x = np.asarray(x, np.float64)
    L = (E - 1) * tau
    T = x.size
    V = embed(x, E, tau)[: T - Tp - L]  # times L .. T-1-Tp
    times = np.arange(L, T - Tp)
    D = distance_matrix(V, V)
    mask = None
    if excl >= 0:
        mask = np.abs(times[:, None] - times[None, :]) > excl
    idx, d2 = neighbours(D, times, E + 1, mask)
    w = np.stack([exp_weights(r) for r in d2])
    return idx, w, d2


def ccm_pair(x_lib, y_tgt, E, tau=1, Tp=1, excl=0) -> float:
    idx, w, _ = ccm_table(x_lib, E, tau, Tp, excl)
    y = np.asarray(y_tgt, np.float64)
    L = (E - 1) * tau
    pred = (w * y[idx + Tp]).sum(axis=1)
    obs = y[np.arange(L, y.size - Tp) + Tp]
    return corr(obs, pred)


def ccm_matrix(Y, optE, tau=1, Tp=1, excl=0) -> np.ndarray:
    Y = np.asarray(Y, np.float64)
    N = Y.shape[0]
    R = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            R[i, j] = ccm_pair(Y[i], Y[j], int(optE[j]), tau, Tp, excl)
    return R


def simplex_rho(x, E, tau=1, Tp=1) -> float:
    x = np.asarray(x, np.float64)
    h = x.size // 2
    lib, tgt = x[:h], x[h:]
    L = (E - 1) * tau
    Vl = embed(lib, E, tau)[: lib.size - Tp - L]
    Vt = embed(tgt, E, tau)[: tgt.size - Tp - L]
    lib_times = np.arange(L, lib.size - Tp)
    if Vt.shape[0] < 1 or Vl.shape[0] < E + 1:
        return float("nan")
    D = distance_matrix(Vt, Vl)
    idx, d2 = neighbours(D, lib_times, E + 1)
    pred = np.array([np.dot(exp_weights(d2[q]), lib[idx[q] + Tp]) for q in range(idx.shape[0])])
    obs = tgt[np.arange(L, tgt.size - Tp) + Tp]
    return corr(obs, pred)


def optimal_E(x, E_max, tau=1, Tp=1):
    rhos = np.array([simplex_rho(x, E, tau, Tp) for E in range(1, E_max + 1)])
    vals = np.where(np.isnan(rhos), -np.inf, rhos)
    return int(np.argmax(vals)) + 1, rhos


def ccm_lags_pair(x_lib, y_tgt, E, lags, tau=1, excl=0) -> np.ndarray:
    """Time-delay cross mapping, per pair: one table over the embedded
    points whose every lag stays inside the series (queries = candidates =
    t in [max(L, -min(lags)), T-1-max(max(lags), 0)]), then for each lag l
    corr(y(t+l), sum_n w y(s_n+l))."""
    x = np.asarray(x_lib, np.float64)
    y = np.asarray(y_tgt, np.float64)
    T = x.size
    L = (E - 1) * tau
    A = max(L, -min(lags))
    B = T - 1 - max(max(lags), 0)
    times = np.arange(A, B + 1)
    V = embed(x, E, tau)[A - L: B - L + 1]
    D = distance_matrix(V, V)
    mask = np.abs(times[:, None] - times[None, :]) > excl if excl >= 0 else None
    idx, d2 = neighbours(D, times, E + 1, mask)
    w = np.stack([exp_weights(r) for r in d2])
    out = []
    for lag in lags:
        pred = (w * y[idx + lag]).sum(axis=1)
        out.append(corr(y[times + lag], pred))
    return np.array(out)


def ccm_pair_subset(x_lib, y_tgt, E, allowed, tau=1, Tp=1, excl=0) -> float:
    """Plain cross map with the candidate points restricted to the set
    `allowed` of times (queries: every embedded point)."""
    x = np.asarray(x_lib, np.float64)
    y = np.asarray(y_tgt, np.float64)
    T = x.size
    L = (E - 1) * tau
    times = np.arange(L, T - Tp)
    V = embed(x, E, tau)[: T - Tp - L]
    keep = np.array([t in allowed for t in times])
    D = distance_matrix(V, V[keep])
    ct = times[keep]
    mask = np.abs(times[:, None] - ct[None, :]) > excl if excl >= 0 else None
    idx, d2 = neighbours(D, ct, E + 1, mask)
    w = np.stack([exp_weights(r) for r in d2])
    pred = (w * y[idx + Tp]).sum(axis=1)
    return corr(y[times + Tp], pred)
