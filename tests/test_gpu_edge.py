"""Edge cases and seeded random parameter draws through the C ABI against
the FP64 oracle: a constant target (zero variance: rho = NaN), a constant
library and a near-constant one (a constant plus one step) whose
predictions are almost equal, a constant series in phase 1 (every rho_E
NaN: optE = 1), an empty library range, and random (tau, Tp, exclusion
radius, E per target, N, T) draws in both target precisions."""

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


def _degenerate_series(T=1500):
    Y = synth.coupled_logistic(10, T, 0.05, 0.05, seed_data=81, seed_noise=82)
    Y[3, :] = 0.7  # constant
    Y[5, : T // 2] = -0.4  # constant, then one step
    Y[5, T // 2:] = 1.3
    return Y


def _same_nan_and_close(got, R, tol):
    """NaN exactly where the oracle has NaN (a side of zero variance), the
    rest within tol; returns the largest error."""
    nan_o, nan_g = np.isnan(R), np.isnan(got)
    assert np.array_equal(nan_o, nan_g), np.argwhere(nan_o != nan_g)[:5]
    err = np.abs(got[~nan_o] - R[~nan_o])
    assert err.max() < tol, err.max()
    return float(err.max())


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_constant_series_against_oracle(edm, prec):
    """Row 3 (a constant library: every distance 0, neighbours by the tie
    rule, predictions equal but for a few rows) and row 5 (two constant
    levels) must match the oracle like every other library; column 3 (a
    constant target) is NaN on both sides."""
    Y = _degenerate_series()
    oE = np.random.default_rng(83).integers(1, 6, size=10).astype(np.int32)
    p, tol = (edm.EDM_PRECISION_FP32, RHO_TOL) if prec == "fp32" else (edm.EDM_PRECISION_FP16_TARGETS, FP16_TOL)
    got = edm.edm_ccm_rho(_dev(Y), torch.from_numpy(oE).cuda(), precision=p).cpu().numpy().T  # [library][target]
    R = orc.ccm_rho_rows(Y, oE)
    assert np.isnan(R[:, 3]).all()
    _same_nan_and_close(got, R, tol)
    # the constant library's skill is small but defined for most targets;
    # it is not rounding noise
    assert np.sum(np.isfinite(R[3])) >= 7 and np.nanmax(np.abs(R[3])) > 1e-3


def test_constant_library_scalar_and_warp_paths(edm):
    """The same degenerate libraries through the scalar-gather lookup and the
    warp kNN kernel (every lookup kernel family sums shifted moments)."""
    Y = _degenerate_series()
    oE = np.random.default_rng(87).integers(1, 6, size=10).astype(np.int32)
    R = orc.ccm_rho_rows(Y, oE)
    for flags in (edm.EDM_FLAG_LOOKUP_SCALAR, edm.EDM_FLAG_KNN_WARP):
        got = edm.edm_ccm_rho(_dev(Y), torch.from_numpy(oE).cuda(), flags=flags).cpu().numpy().T
        _same_nan_and_close(got, R, RHO_TOL)


def test_constant_target_gives_nan(edm):
    Y = _degenerate_series()
    oE = np.random.default_rng(83).integers(1, 6, size=10).astype(np.int32)
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


def test_unusable_optE_gives_nan_rows_or_invalid(edm):
    """optE values outside 1..EDM_MAX_E: the device-planned call (no host
    synchronisation) writes NaN for those targets and the oracle's values
    for every other; with EDM_FLAG_VALIDATE optE is checked on the host and
    the call returns EDM_ERR_INVALID."""
    Y = synth.coupled_logistic(20, 300, 0.05, 0.05, seed_data=94, seed_noise=95)
    E = np.random.default_rng(96).integers(1, 6, size=20).astype(np.int32)
    R = orc.ccm_rho_rows(Y, E)
    Eb = E.copy()
    Eb[4], Eb[11] = 0, edm.EDM_MAX_E + 1
    got = edm.edm_ccm_rho(_dev(Y), torch.from_numpy(Eb).cuda()).cpu().numpy()  # [target][library]
    assert np.isnan(got[[4, 11]]).all()
    keep = [j for j in range(20) if j not in (4, 11)]
    assert np.abs(got[keep].T - R[:, keep]).max() < RHO_TOL
    with pytest.raises(edm.EdmError) as ei:
        edm.edm_ccm_rho(_dev(Y), torch.from_numpy(Eb).cuda(), flags=edm.EDM_FLAG_VALIDATE)
    assert ei.value.status == 1


def test_cross_map_needs_no_host_synchronisation(edm):
    """The cross map plans its E grouping on the device, so a whole call can
    be recorded into a CUDA graph (a synchronisation or a device-to-host read
    would end the capture with an error) and replayed: the replay on new data
    equals a direct call."""
    Y1 = synth.coupled_logistic(300, 500, 0.05, 0.05, seed_data=97, seed_noise=98)
    Y2 = synth.coupled_logistic(300, 500, 0.05, 0.05, seed_data=99, seed_noise=100)
    Yd = _dev(Y1)
    E = torch.from_numpy(np.random.default_rng(101).integers(1, 9, size=300).astype(np.int32)).cuda()
    out = torch.empty((300, 300), dtype=torch.float32, device="cuda")
    ws = torch.empty(edm.edm_ccm_workspace_bytes(300, 500), dtype=torch.uint8, device="cuda")
    edm.edm_ccm_rho(Yd, E, out=out, workspace=ws)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            edm.edm_ccm_rho(Yd, E, out=out, workspace=ws)
    Yd.copy_(_dev(Y2))
    g.replay()
    torch.cuda.synchronize()
    ref = edm.edm_ccm_rho(_dev(Y2), E)
    assert torch.equal(out, ref)
