"""Long series (the paper's time-step sweep reaches T = 40,000) through the C
ABI against the FP64 oracle.

Beyond about 3,100 steps a target tile no longer fits shared memory and the
lookup reads it from global memory / L2; beyond about 30,000 the kNN
kernels stage the series with fewer register slots per lane (shorter
candidate chunks).  Bars as in the other parity tests: neighbour indices
bit-exact, optimal E identical, rho within 1e-4 absolute.
"""

import numpy as np
import pytest
import torch

import edm_synth as synth
from oracle import oracle as orc

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-4
W_TOL = 1e-6


@pytest.fixture(scope="module")
def edm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2011_11082_gb300 as m

    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_ccm_global_memory_tiles(edm):
    """T = 3,200: tiles read from L2; E = 1..12 covers both register classes
    of the lookup (K <= 9 and K > 9); 40 targets = tiles with ragged tails."""
    N, T = 40, 3200
    Y = synth.coupled_logistic(N, T, 0.05, 0.05, seed_data=31, seed_noise=32)
    oE = np.random.default_rng(33).integers(1, 13, size=N).astype(np.int32)
    Yd, Ed = _dev(Y), torch.from_numpy(oE).cuda()
    rho_t = edm.edm_ccm_rho(Yd, Ed)
    rows = np.random.default_rng(34).choice(N, 5, replace=False)
    R = orc.ccm_rho_rows(Y, oE, rows=rows)
    got = rho_t.cpu().numpy()[:, rows].T
    assert np.abs(got - R).max() < RHO_TOL
    # long series keep FP32 tiles: the FP16 request gives the same bits
    rho_h = edm.edm_ccm_rho(Yd, Ed, precision=edm.EDM_PRECISION_FP16_TARGETS)
    assert torch.equal(rho_h, rho_t)
    # a library sub-range lands in its own columns
    part = edm.edm_ccm_rho(Yd, Ed, lib_begin=7, lib_count=9)
    assert torch.equal(part, rho_t[:, 7:16])


def test_ccm_global_memory_tiles_end_to_end(edm):
    """Both phases at T = 3,600 (E chosen on the GPU, identical to the oracle's)."""
    N, T = 36, 3600
    Y = synth.coupled_logistic(N, T, 0.05, 0.05, seed_data=35, seed_noise=36)
    Yd = _dev(Y)
    optE, rhoE = edm.edm_optimal_E(Yd, E_max=8)
    oE, orhoE = orc.optimal_E(Y, 8)
    assert np.array_equal(optE.cpu().numpy(), oE)
    assert np.nanmax(np.abs(rhoE.cpu().numpy() - orhoE)) < 2e-5
    rho_t = edm.edm_ccm_rho(Yd, optE)
    rows = np.array([0, 17, 35])
    R = orc.ccm_rho_rows(Y, oE, rows=rows)
    assert np.abs(rho_t.cpu().numpy()[:, rows].T - R).max() < RHO_TOL


def test_lags_global_memory_tiles(edm):
    N, T = 24, 3300
    Y = synth.coupled_logistic(N, T, 0.05, 0.05, seed_data=37, seed_noise=38)
    oE = np.random.default_rng(39).integers(1, 7, size=N).astype(np.int32)
    rho = edm.edm_ccm_rho_lags(_dev(Y), torch.from_numpy(oE).cuda(), -2, 1)
    rows = np.array([3, 20])
    R = orc.ccm_rho_lags(Y, oE, -2, 1, rows=rows)
    got = rho.cpu().numpy()[:, :, rows].transpose(0, 2, 1)
    assert np.abs(got - R).max() < RHO_TOL


@pytest.mark.parametrize("E,flags", [(2, 0), (3, 4), (7, 0)])
def test_knn_table_t40000_sampled_rows(edm, E, flags):
    """T = 40,000 (the sweep's longest series): thread kernel (E = 2), warp
    kernel with shortened candidate chunks (E = 3 forced, E = 7); 48 sampled
    query rows against the oracle's kNN of those rows."""
    T = 40000
    x = synth.coupled_logistic(1, T, 0.0, 0.0, seed_data=41, seed_noise=42)
    idx, w = edm.edm_knn_table(_dev(x), E, flags=flags)
    idx, w = idx.cpu().numpy()[0], w.cpu().numpy()[0]
    L = E - 1
    rows = np.sort(np.random.default_rng(43).choice(T - 1 - L, 48, replace=False))
    rows[0], rows[-1] = 0, T - 1 - L - 1  # first and last query
    for r in rows:
        t = L + int(r)
        oi, od2 = orc.knn(x[0], t, t, x[0], L, T - 2, E, same=True, excl=0)
        assert np.array_equal(idx[r], oi[0]), (E, t, idx[r], oi[0])
        assert np.abs(w[r] - orc.weights(od2[0])).max() < W_TOL


def test_optimal_E_t36000(edm):
    """Phase 1 on 18,000-point halves (the simplex kernel's shortened chunks)."""
    T = 36000
    Y = synth.coupled_logistic(2, T, 0.05, 0.02, seed_data=44, seed_noise=45)
    optE, rhoE = edm.edm_optimal_E(_dev(Y), E_max=3)
    oE, orhoE = orc.optimal_E(Y, 3)
    assert np.array_equal(optE.cpu().numpy(), oE)
    assert np.nanmax(np.abs(rhoE.cpu().numpy() - orhoE)) < 2e-5


def test_too_long_series_rejected(edm):
    x = torch.zeros((1, 60000), dtype=torch.float32, device="cuda")
    with pytest.raises(edm.EdmError) as ei:
        edm.edm_knn_table(x, 2)
    assert ei.value.status == 5  # EDM_ERR_UNSUPPORTED
