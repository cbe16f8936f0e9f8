"""Time-delay cross mapping (edm_ccm_rho_lags) through the C ABI against the
FP64 oracle: several lags from one table per (library, E), negative, zero
and positive lags, both kNN kernels (tau = 1 and tau = 2), FP16 targets, and
the reduction of a single lag to the plain cross map."""

import numpy as np
import pytest
import torch

import edm_synth as synth
from oracle import oracle as orc

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-4


@pytest.fixture(scope="module")
def edm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2011_11082_gb300 as m

    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case(seed, N=24, T=300):
    Y = synth.coupled_logistic(N, T, 0.08, 0.05, seed_data=seed, seed_noise=seed + 1)
    oE, _ = orc.optimal_E(Y, 6)
    return Y, oE


@pytest.mark.parametrize("lag_min,lag_max,excl,tau", [(-3, 3, 0, 1), (0, 5, 2, 1), (-6, -1, -1, 1), (-2, 2, 0, 2)])
def test_lags_match_oracle(edm, lag_min, lag_max, excl, tau):
    Y, oE = _case(71)
    R = orc.ccm_rho_lags(Y, oE, lag_min, lag_max, tau=tau, excl=excl)  # [lag][lib][tgt]
    G = edm.edm_ccm_rho_lags(_dev(Y), torch.from_numpy(oE).cuda(), lag_min, lag_max, tau=tau,
                             exclusion_radius=excl).cpu().numpy()  # [lag][tgt][lib]
    G = np.transpose(G, (0, 2, 1))
    assert np.abs(G - R).max() < RHO_TOL, np.abs(G - R).max()


def test_single_lag_is_the_plain_cross_map(edm):
    Y, oE = _case(73, N=37, T=420)
    Yd, Ed = _dev(Y), torch.from_numpy(oE).cuda()
    for Tp in (1, 2):
        a = edm.edm_ccm_rho_lags(Yd, Ed, Tp, Tp)[0]
        b = edm.edm_ccm_rho(Yd, Ed, Tp=Tp)
        assert torch.equal(a, b), Tp


def test_lags_fp16_targets(edm):
    Y, oE = _case(75, N=70, T=500)
    R = orc.ccm_rho_lags(Y, oE, -4, 4)
    G = edm.edm_ccm_rho_lags(_dev(Y), torch.from_numpy(oE).cuda(), -4, 4,
                             precision=edm.EDM_PRECISION_FP16_TARGETS).cpu().numpy()
    assert np.abs(np.transpose(G, (0, 2, 1)) - R).max() < 1e-3


def test_lags_window_too_short_is_rejected(edm):
    Y, oE = _case(77, N=4, T=40)
    with pytest.raises(edm.EdmError) as ei:
        edm.edm_ccm_rho_lags(_dev(Y), torch.from_numpy(np.full(4, 6, np.int32)).cuda(), -18, 18)
    assert ei.value.status == 1
