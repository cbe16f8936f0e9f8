"""Hand-written adjoint (through the C ABI) against the FP64 reference
gradient (PyTorch CPU float64 autograd, frozen tables from the C oracle) and
against central finite differences of the oracle's frozen-index rho."""

import numpy as np
import pytest
import torch

import edm_synth as synth
from oracle import adjoint
from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def edm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2011_11082_gb300 as m

    return m


def _tables(Y, optE):
    return {(i, E): orc.ccm_table(Y[i], E)[0] for i in range(Y.shape[0]) for E in set(optE.tolist())}


def test_backward_matches_fp64_reference_gradient(edm):
    Y = synth.coupled_logistic(7, 160, 0.2, 0.05, seed_data=51, seed_noise=52)
    optE = np.array([1, 2, 3, 2, 4, 2, 3], np.int32)
    L_ref, G_ref = adjoint.mean_rho_and_grad(Y.astype(np.float64), optE, _tables(Y, optE))
    Yd = torch.from_numpy(Y).cuda().requires_grad_(True)
    rho = edm.ccm_rho_autograd(Yd, torch.from_numpy(optE).cuda())
    L = rho.mean()
    L.backward()
    assert abs(L.item() - L_ref) < 1e-5
    G = Yd.grad.cpu().numpy()
    scale = np.abs(G_ref).max()
    assert np.abs(G - G_ref).max() < 1e-4 * scale + 1e-7, (np.abs(G - G_ref).max(), scale)


def test_backward_general_upstream_gradient(edm):
    """L = sum_ij C_ij rho_ij with random C: the adjoint applies C exactly."""
    Y = synth.coupled_logistic(5, 140, 0.2, 0.05, seed_data=53, seed_noise=54)
    optE = np.array([2, 1, 3, 2, 2], np.int32)
    C = np.random.default_rng(7).standard_normal((5, 5))
    Yt = torch.tensor(Y.astype(np.float64), requires_grad=True)
    tot = 0
    tabs = _tables(Y, optE)
    for i in range(5):
        for j in range(5):
            E = int(optE[j])
            tot = tot + C[i, j] * adjoint.rho_frozen(Yt[i], Yt[j], E, torch.as_tensor(tabs[(i, E)]))
    tot.backward()
    G_ref = Yt.grad.numpy()
    g_t = torch.from_numpy(C.T.astype(np.float32)).contiguous().cuda()  # target-major
    G = edm.edm_ccm_rho_backward(torch.from_numpy(Y).cuda(), torch.from_numpy(optE).cuda(), g_t).cpu().numpy()
    assert np.abs(G - G_ref).max() < 1e-4 * np.abs(G_ref).max() + 1e-7, (np.abs(G - G_ref).max(), np.abs(G_ref).max())


def test_backward_finite_differences_batched_style(edm):
    """A batched-workload-sized dataset: dL/dY of the mean rho against
    central differences (h = 1e-3) of the oracle's frozen-index rho on 50
    sampled entries."""
    spec = synth.batched_specs()[0]
    N, T = min(spec.N, 96), min(spec.T, 700)
    Y = synth.coupled_logistic(N, T, 0.01, 0.02, seed_data=spec.seed_data, seed_noise=spec.seed_noise)
    Yd = torch.from_numpy(Y).cuda()
    optE, _ = edm.edm_optimal_E(Yd, E_max=8, return_rho=False)
    oE = optE.cpu().numpy()
    Yg = Yd.clone().requires_grad_(True)
    rho = edm.ccm_rho_autograd(Yg, optE)
    rho.mean().backward()
    G = Yg.grad.cpu().numpy()
    tabs = {}
    Y64 = Y.astype(np.float64)

    def tab(i, E):
        if (i, E) not in tabs:
            tabs[(i, E)] = orc.ccm_table(Y64[i], E)[0]
        return tabs[(i, E)]

    rng = np.random.default_rng(5)
    h = 1e-3
    worst = 0.0
    for _ in range(50):
        a, t = int(rng.integers(0, N)), int(rng.integers(0, T))

        def L_of(Yv):
            s = 0.0
            for j in range(N):  # series a as library
                E = int(oE[j])
                s += orc.rho_frozen(Yv[a], Yv[j], E, tab(a, E))
            Ea = int(oE[a])
            for i in range(N):  # series a as target (i == a counted above)
                if i != a:
                    s += orc.rho_frozen(Yv[i], Yv[a], Ea, tab(i, Ea))
            return s / (N * N)

        Yp, Ym = Y64.copy(), Y64.copy()
        Yp[a, t] += h
        Ym[a, t] -= h
        fd = (L_of(Yp) - L_of(Ym)) / (2 * h)
        err = abs(fd - G[a, t])
        worst = max(worst, err / (abs(fd) + 1e-4))
        assert err < 1e-4 + 2e-2 * abs(fd), (a, t, fd, G[a, t])


def test_backward_degenerate_series(edm):
    """A constant series (row 3) and a two-level step (row 5).  As a target,
    the constant series has zero observation variance: rho is NaN for every
    library, and those pairs add nothing to the gradient.  As a library, its
    distances are all 0 (neighbours by the tie rule, duplicate-only weights):
    predictions equal but for the rows next to the exclusion window (on the
    step target they are all equal: NaN again), and no gradient flows through
    its distances.  Against the FP64 reference of L = sum over the finite
    pairs of C_ij rho_ij; the adjoint gets C everywhere and must add nothing
    for the NaN pairs."""
    T = 300
    Y = synth.coupled_logistic(10, T, 0.05, 0.05, seed_data=81, seed_noise=82)
    Y[3, :] = 0.7
    Y[5, : T // 2] = -0.4
    Y[5, T // 2:] = 1.3
    optE = np.random.default_rng(83).integers(1, 6, size=10).astype(np.int32)
    C = np.random.default_rng(84).standard_normal((10, 10))
    tabs = _tables(Y, optE)
    Yt = torch.tensor(Y.astype(np.float64), requires_grad=True)
    tot = 0
    for i in range(10):
        for j in range(10):
            r = adjoint.rho_frozen(Yt[i], Yt[j], int(optE[j]), torch.as_tensor(tabs[(i, int(optE[j]))]))
            if torch.isfinite(r):  # NaN: a side of zero variance
                tot = tot + C[i, j] * r
    tot.backward()
    G_ref = Yt.grad.numpy()
    g_t = torch.from_numpy(C.T.astype(np.float32)).contiguous().cuda()  # target-major, C everywhere
    G = edm.edm_ccm_rho_backward(torch.from_numpy(Y).cuda(), torch.from_numpy(optE).cuda(), g_t).cpu().numpy()
    assert np.isfinite(G).all()
    assert np.abs(G - G_ref).max() < 1e-4 * np.abs(G_ref).max() + 1e-7, (np.abs(G - G_ref).max(), np.abs(G_ref).max())
