"""The FP64 adjoint reference (torch autograd, frozen indices) against central
finite differences of the C oracle's frozen-table rho (CPU only)."""

import numpy as np
import torch

import edm_synth as synth
from oracle import adjoint
from oracle import oracle as orc


def test_adjoint_reference_matches_fd_of_oracle():
    Y = synth.coupled_logistic(3, 90, 0.3, 0.05, seed_data=31, seed_noise=32).astype(np.float64)
    optE = np.array([2, 3, 1], np.int32)
    tables = {}
    for i in range(3):
        for E in set(optE.tolist()):
            tables[(i, E)] = orc.ccm_table(Y[i], E)[0]

    def loss(Yv):
        tot = 0.0
        for i in range(3):
            for j in range(3):
                E = int(optE[j])
                tot += orc.rho_frozen(Yv[i], Yv[j], E, tables[(i, E)])
        return tot / 9.0

    L, G = adjoint.mean_rho_and_grad(Y, optE, tables)
    assert abs(L - loss(Y)) < 1e-13
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(25):
        a, t = int(rng.integers(0, 3)), int(rng.integers(0, 90))
        Yp, Ym = Y.copy(), Y.copy()
        Yp[a, t] += h
        Ym[a, t] -= h
        fd = (loss(Yp) - loss(Ym)) / (2 * h)
        assert abs(fd - G[a, t]) < 1e-7 + 1e-5 * abs(fd), (a, t, fd, G[a, t])


def test_adjoint_reference_pair_closed_form_target_gradient():
    """For a fixed table, rho is a function of the target y through p and o.
    With library = target-independent weights, d rho / d y matches the
    textbook Pearson derivative chained through p = W y (checked via autograd
    of an explicit dense W)."""
    x = synth.logistic_series(60).astype(np.float64)
    y = synth.white_noise(60, seed=3).astype(np.float64)
    E = 2
    idx, w = orc.ccm_table(x, E)
    nq = idx.shape[0]
    W = np.zeros((nq, 60))
    for r in range(nq):
        for n in range(E + 1):
            W[r, idx[r, n] + 1] += w[r, n]
    S = np.zeros((nq, 60))
    S[np.arange(nq), np.arange(E - 1, E - 1 + nq) + 1] = 1.0
    yt = torch.tensor(y, requires_grad=True)
    p = torch.tensor(W) @ yt
    o = torch.tensor(S) @ yt
    pc, oc = p - p.mean(), o - o.mean()
    r_dense = (pc * oc).sum() / torch.sqrt((pc * pc).sum() * (oc * oc).sum())
    r_dense.backward()
    g_dense = yt.grad.numpy().copy()
    yt2 = torch.tensor(y, requires_grad=True)
    r = adjoint.rho_frozen(torch.tensor(x), yt2, E, torch.as_tensor(idx))
    r.backward()
    assert abs(float(r.detach()) - float(r_dense.detach())) < 1e-13
    assert np.allclose(yt2.grad.numpy(), g_dense, atol=1e-13)
