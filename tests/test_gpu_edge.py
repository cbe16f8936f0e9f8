"""Edge cases and seeded random parameter draws through the C ABI against
the FP64 oracle: a constant target (zero variance: rho = NaN), a constant
series in phase 1 (every rho_E NaN: optE = 1), an empty library range, and
random (tau, Tp, exclusion radius, E per target, N, T) draws in both target
precisions."""

import numpy as np
import pytest
import torch

import edm_synth as synth
from oracle import oracle as orc

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-4
FP16_TOL = 1e-3


@pytest.fixture(scope="module")
def edm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2011_11082_gb300 as m

    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_constant_target_gives_nan(edm):
    Y = synth.coupled_logistic(10, 300, 0.05, 0.05, seed_data=81, seed_noise=82)
    Y[3, :] = 0.7
    oE = np.random.default_rng(83).integers(1, 6, size=10).astype(np.int32)
    got = edm.edm_ccm_rho(_dev(Y), torch.from_numpy(oE).cuda()).cpu().numpy().T  # [library][target]
    R = orc.ccm_rho_rows(Y, oE)
    assert np.isnan(R[:, 3]).all() and np.isnan(got[:, 3]).all()
    # every other target, from every non-constant library, as the oracle
    keep_i = [i for i in range(10) if i != 3]
    keep_j = [j for j in range(10) if j != 3]
    assert np.abs(got[np.ix_(keep_i, keep_j)] - R[np.ix_(keep_i, keep_j)]).max() < RHO_TOL
    # phase 1 on the constant series: every rho_E is NaN and optE = 1
    optE, rhoE = edm.edm_optimal_E(_dev(Y), E_max=5)
    oE1, orhoE = orc.optimal_E(Y, 5)
    assert np.isnan(orhoE[3]).all() and np.isnan(rhoE.cpu().numpy()[3]).all()
    assert oE1[3] == 1 and int(optE[3]) == 1
    assert np.array_equal(optE.cpu().numpy(), oE1)


def test_empty_library_range(edm):
    Y = synth.coupled_logistic(6, 200, 0.05, 0.05, seed_data=84, seed_noise=85)
    Ed = torch.full((6,), 2, dtype=torch.int32, device="cuda")
    out = edm.edm_ccm_rho(_dev(Y), Ed, lib_begin=4, lib_count=0)
    assert tuple(out.shape) == (6, 0)


def test_random_parameters_against_oracle(edm):
    rng = np.random.default_rng(86)
    for case in range(8):
        tau = int(rng.integers(1, 4))
        Tp = int(rng.integers(0, 3))
        excl = int(rng.choice([-1, 0, 3]))
        N = int(rng.integers(5, 41))
        T = int(rng.integers(120, 401))
        Y = synth.coupled_logistic(N, T, 0.05, 0.05, seed_data=1000 + case, seed_noise=2000 + case)
        Yd = _dev(Y)
        # phase 1 (the oracle's optE must match exactly)
        E_max = 4
        optE, _ = edm.edm_optimal_E(Yd, E_max=E_max, tau=tau, Tp=Tp)
        oE, _ = orc.optimal_E(Y, E_max, tau=tau, Tp=Tp)
        assert np.array_equal(optE.cpu().numpy(), oE), (case, tau, Tp)
        # phase 2 with random E per target (up to 8), both precisions
        E = rng.integers(1, 9, size=N).astype(np.int32)
        Ed = torch.from_numpy(E).cuda()
        rows = np.sort(rng.choice(N, min(N, 4), replace=False))
        R = orc.ccm_rho_rows(Y, E, rows=rows, tau=tau, Tp=Tp, excl=excl)
        for prec, tol in ((edm.EDM_PRECISION_FP32, RHO_TOL), (edm.EDM_PRECISION_FP16_TARGETS, FP16_TOL)):
            got = edm.edm_ccm_rho(Yd, Ed, tau=tau, Tp=Tp, exclusion_radius=excl, precision=prec)
            got = got.cpu().numpy()[:, rows].T
            assert np.abs(got - R).max() < tol, (case, prec, tau, Tp, excl, N, T)
