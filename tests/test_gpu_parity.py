"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars: neighbour indices bit-exact; optimal E identical; rho within 1e-4
absolute (weights within 1e-6).  Sizes span several tiles and ragged tails.
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


def _tie_series(T):
    """Series with exact distance ties (integer-period sine, a step pattern)."""
    s = synth.sine_series(T, 16)
    step = (np.arange(T) % 7).astype(np.float32) - 3.0
    return np.stack([s, step])


@pytest.mark.parametrize("E", [1, 2, 3, 5, 8, 13, 20])
def test_knn_tables_bit_exact(edm, E):
    Y = np.concatenate([synth.coupled_logistic(6, 500, 0.05, 0.05, seed_data=3, seed_noise=4), _tie_series(500)])
    Yd = _dev(Y)
    for tau, Tp, excl in ((1, 1, 0), (2, 1, 3), (1, 0, 0), (1, 2, -1)):
        idx, w = edm.edm_knn_table(Yd, E, tau=tau, Tp=Tp, exclusion_radius=excl)
        idx, w = idx.cpu().numpy(), w.cpu().numpy()
        for i in range(Y.shape[0]):
            oi, ow = orc.ccm_table(Y[i], E, tau, Tp, excl)
            assert np.array_equal(idx[i], oi), (E, tau, Tp, excl, i, np.argwhere(idx[i] != oi)[:5])
            assert np.abs(w[i] - ow).max() < W_TOL, (E, tau, Tp, excl, i)


def test_knn_tables_long_series_chunked(edm):
    """T = 3000 exceeds one candidate chunk per lane (chunked path)."""
    Y = synth.coupled_logistic(3, 3000, 0.1, 0.05, seed_data=5, seed_noise=6)
    Yd = _dev(Y)
    for E in (2, 7):
        idx, w = edm.edm_knn_table(Yd, E)
        idx, w = idx.cpu().numpy(), w.cpu().numpy()
        for i in range(3):
            oi, ow = orc.ccm_table(Y[i], E)
            assert np.array_equal(idx[i], oi)
            assert np.abs(w[i] - ow).max() < W_TOL


def test_optimal_E_small_workload(edm):
    Y = synth.workload("n64_t500")
    optE, rho = edm.edm_optimal_E(_dev(Y), E_max=10)
    oE, orho = orc.optimal_E(Y, 10)
    assert np.array_equal(optE.cpu().numpy(), oE)
    assert np.nanmax(np.abs(rho.cpu().numpy() - orho)) < 2e-5


def test_optimal_E_n2048_sample(edm):
    Y = synth.workload("n2048_t1500")
    optE, rho = edm.edm_optimal_E(_dev(Y), E_max=20)
    sel = np.random.default_rng(0).choice(Y.shape[0], 192, replace=False)
    oE, orho = orc.optimal_E(Y[sel], 20)
    got = optE.cpu().numpy()[sel]
    bad = np.nonzero(got != oE)[0]
    assert bad.size == 0, [(int(sel[b]), int(got[b]), int(oE[b]), orho[b]) for b in bad[:3]]
    assert np.nanmax(np.abs(rho.cpu().numpy()[sel] - orho)) < 2e-5


def test_optimal_E_odd_T_tau2(edm):
    Y = synth.coupled_logistic(40, 401, 0.05, 0.05, seed_data=9, seed_noise=10)
    optE, rho = edm.edm_optimal_E(_dev(Y), E_max=8, tau=2, Tp=2)
    oE, orho = orc.optimal_E(Y, 8, tau=2, Tp=2)
    assert np.array_equal(optE.cpu().numpy(), oE)
    assert np.nanmax(np.abs(rho.cpu().numpy() - orho)) < 2e-5


def test_ccm_full_small_workload(edm):
    Y = synth.workload("n64_t500")
    oE, _ = orc.optimal_E(Y, 10)
    rho_t = edm.edm_ccm_rho(_dev(Y), torch.from_numpy(oE).cuda())
    R = orc.ccm_rho_rows(Y, oE)
    got = rho_t.t().cpu().numpy()
    assert np.abs(got - R).max() < RHO_TOL


def test_ccm_n2048_sampled_rows(edm):
    Y = synth.workload("n2048_t1500")
    Yd = _dev(Y)
    optE, _ = edm.edm_optimal_E(Yd, E_max=20)
    rho_t = edm.edm_ccm_rho(Yd, optE)
    oE = optE.cpu().numpy()
    rows = np.random.default_rng(1).choice(Y.shape[0], 12, replace=False)
    R = orc.ccm_rho_rows(Y, oE, rows=rows)
    got = rho_t.cpu().numpy()[:, rows].T
    assert np.abs(got - R).max() < RHO_TOL


def test_ccm_ragged_and_subranges(edm):
    Y = synth.coupled_logistic(37, 260, 0.05, 0.05, seed_data=11, seed_noise=12)
    rng = np.random.default_rng(2)
    oE = rng.integers(1, 7, size=37).astype(np.int32)
    R = orc.ccm_rho_rows(Y, oE)
    Yd, Ed = _dev(Y), torch.from_numpy(oE).cuda()
    full = edm.edm_ccm_rho(Yd, Ed).cpu().numpy().T
    assert np.abs(full - R).max() < RHO_TOL
    # a library sub-range written into a wider buffer
    out = torch.full((37, 20), float("nan"), device="cuda")
    edm.edm_ccm_rho(Yd, Ed, lib_begin=9, lib_count=13, out=out)
    blk = out.cpu().numpy()
    assert np.abs(blk[:, :13].T - R[9:22]).max() < RHO_TOL
    assert np.isnan(blk[:, 13:]).all()


def test_ccm_single_series_and_uniform_E(edm):
    Y = synth.coupled_logistic(1, 120, 0.0, 0.0, seed_data=13, seed_noise=14)
    for E in (1, 4):
        oE = np.array([E], np.int32)
        got = edm.edm_ccm_rho(_dev(Y), torch.from_numpy(oE).cuda()).cpu().numpy()
        assert abs(got[0, 0] - orc.ccm_rho_rows(Y, oE)[0, 0]) < RHO_TOL


def test_ccm_tau_Tp_exclusion_variants(edm):
    Y = synth.coupled_logistic(20, 300, 0.05, 0.05, seed_data=15, seed_noise=16)
    oE = np.random.default_rng(3).integers(1, 6, size=20).astype(np.int32)
    for tau, Tp, excl in ((2, 1, 0), (1, 2, 5), (1, 0, -1)):
        R = orc.ccm_rho_rows(Y, oE, tau=tau, Tp=Tp, excl=excl)
        got = edm.edm_ccm_rho(_dev(Y), torch.from_numpy(oE).cuda(), tau=tau, Tp=Tp,
                              exclusion_radius=excl).cpu().numpy().T
        assert np.abs(got - R).max() < RHO_TOL, (tau, Tp, excl)


def test_ccm_closed_forms(edm):
    """Integer-period sine predicts itself exactly; self-inclusion gives 1."""
    T = 400
    x = synth.sine_series(T, 16)
    c = np.cos(2 * np.pi * np.mod(np.arange(T), 16) / 16).astype(np.float32)
    Y = np.stack([x, c])
    got = edm.edm_ccm_rho(_dev(Y), torch.tensor([3, 3], dtype=torch.int32, device="cuda")).cpu().numpy()
    assert np.abs(got - 1.0).max() < 1e-5
    L = synth.logistic_series(300)[None, :]
    got = edm.edm_ccm_rho(_dev(L), torch.tensor([2], dtype=torch.int32, device="cuda"), Tp=0,
                          exclusion_radius=-1).cpu().numpy()
    assert abs(got[0, 0] - 1.0) < 1e-6


def test_ccm_deterministic(edm):
    Y = synth.coupled_logistic(70, 350, 0.05, 0.05, seed_data=17, seed_noise=18)
    Yd = _dev(Y)
    optE, _ = edm.edm_optimal_E(Yd, E_max=8)
    a = edm.edm_ccm_rho(Yd, optE).cpu().numpy()
    b = edm.edm_ccm_rho(Yd, optE).cpu().numpy()
    assert np.array_equal(a, b, equal_nan=True)


# ---------------------------------------------------------------------------
# FP16-target form: rho error against the FP64 oracle within 1e-3; and the
# scalar-gather kernels (comparison path) at the FP32 bar.
FP16_TOL = 1e-3


def test_ccm_fp16_targets_small_workload(edm):
    Y = synth.workload("n64_t500")
    oE, _ = orc.optimal_E(Y, 10)
    rho_t = edm.edm_ccm_rho(_dev(Y), torch.from_numpy(oE).cuda(), precision=edm.EDM_PRECISION_FP16_TARGETS)
    R = orc.ccm_rho_rows(Y, oE)
    assert np.abs(rho_t.t().cpu().numpy() - R).max() < FP16_TOL


def test_ccm_fp16_targets_n2048_rows_and_large_E(edm):
    Y = synth.workload("n2048_t1500")
    Yd = _dev(Y)
    optE, _ = edm.edm_optimal_E(Yd, E_max=20)
    oE = optE.cpu().numpy()
    assert oE.max() >= 12  # exercises the FP32 fallback tiles of large E too
    rho_t = edm.edm_ccm_rho(Yd, optE, precision=edm.EDM_PRECISION_FP16_TARGETS)
    rows = np.random.default_rng(4).choice(Y.shape[0], 8, replace=False)
    R = orc.ccm_rho_rows(Y, oE, rows=rows)
    err = np.abs(rho_t.cpu().numpy()[:, rows].T - R)
    assert err.max() < FP16_TOL, err.max()


def test_ccm_scalar_lookup_matches(edm):
    Y = synth.coupled_logistic(90, 400, 0.05, 0.05, seed_data=19, seed_noise=20)
    oE = np.random.default_rng(6).integers(1, 16, size=90).astype(np.int32)
    R = orc.ccm_rho_rows(Y, oE)
    Yd, Ed = _dev(Y), torch.from_numpy(oE).cuda()
    got = edm.edm_ccm_rho(Yd, Ed, flags=edm.EDM_FLAG_LOOKUP_SCALAR).t().cpu().numpy()
    assert np.abs(got - R).max() < RHO_TOL
    got2 = edm.edm_ccm_rho(Yd, Ed).t().cpu().numpy()
    assert np.abs(got2 - R).max() < RHO_TOL


def test_ccm_host_buffers_end_to_end(edm):
    """edm_ccm_host: host series in, host optE and target-major rho out, in
    several library blocks (copy-back overlapped with compute)."""
    Y = synth.workload("n64_t500")
    Yh = torch.from_numpy(Y).pin_memory()
    optE, rho_t = edm.edm_ccm_host(Yh, E_max=10, block=24)
    oE, _ = orc.optimal_E(Y, 10)
    assert np.array_equal(optE.numpy(), oE)
    R = orc.ccm_rho_rows(Y, oE)
    assert np.abs(rho_t.numpy().T - R).max() < RHO_TOL


def test_ccm_long_series_narrow_tiles(edm):
    """T = 2,200 does not fit 128-byte tile rows: the 64-byte-row kernels
    (16 FP32 / 32 FP16 targets per row) take over."""
    Y = synth.coupled_logistic(45, 2200, 0.05, 0.05, seed_data=61, seed_noise=62)
    oE = np.random.default_rng(8).integers(1, 14, size=45).astype(np.int32)
    R = orc.ccm_rho_rows(Y, oE)
    Yd, Ed = _dev(Y), torch.from_numpy(oE).cuda()
    got = edm.edm_ccm_rho(Yd, Ed).t().cpu().numpy()
    assert np.abs(got - R).max() < RHO_TOL
    got16 = edm.edm_ccm_rho(Yd, Ed, precision=edm.EDM_PRECISION_FP16_TARGETS).t().cpu().numpy()
    assert np.abs(got16 - R).max() < FP16_TOL


def test_validation_flag_names_first_bad_series(edm):
    """EDM_FLAG_VALIDATE: a non-finite value is reported (first bad series)
    before any compute kernel runs; clean data gives the unvalidated results."""
    from paper_2011_11082_gb300 import _abi

    lib = _abi.load()
    Y = synth.coupled_logistic(12, 300, 0.05, 0.05, seed_data=61, seed_noise=62)
    clean = _dev(Y)
    bad = Y.copy()
    bad[9, 3] = np.inf
    bad[7, 120] = np.nan
    Yb = _dev(bad)
    with pytest.raises(edm.EdmError) as ei:
        edm.edm_optimal_E(Yb, E_max=6, flags=edm.EDM_FLAG_VALIDATE)
    assert ei.value.status == 1 and "series 7" in str(ei.value)
    assert lib.edm_last_bad_series() == 7
    optE = torch.full((12,), 2, dtype=torch.int32, device="cuda")
    with pytest.raises(edm.EdmError):
        edm.edm_ccm_rho(Yb, optE, flags=edm.EDM_FLAG_VALIDATE)
    assert lib.edm_last_bad_series() == 7
    a, _ = edm.edm_optimal_E(clean, E_max=6, flags=edm.EDM_FLAG_VALIDATE)
    assert lib.edm_last_bad_series() == -1
    b, _ = edm.edm_optimal_E(clean, E_max=6)
    assert torch.equal(a, b)
    r1 = edm.edm_ccm_rho(clean, a, flags=edm.EDM_FLAG_VALIDATE)
    r2 = edm.edm_ccm_rho(clean, a)
    assert torch.equal(r1, r2)


def test_knn_fp64_fallback_counts(edm):
    """The certified FP32 ranking falls back to FP64 only near ties: on the
    coupled maps the re-rank share is reported and small; exact duplicates
    (an integer-period sine) always take the FP64 path."""
    Y = synth.workload("n64_t500")
    Yd = _dev(Y)
    edm.edm_knn_counters(reset=True)
    oE, _ = edm.edm_optimal_E(Yd, E_max=10, return_rho=False)
    edm.edm_ccm_rho(Yd, oE)
    torch.cuda.synchronize()
    rr, ex = edm.edm_knn_counters(reset=True)
    n_E = len(set(oE.cpu().numpy().tolist()))
    queries = 64 * 250 * 10 + 64 * 500 * n_E  # phase 1 (all E) + phase 2 tables (upper bound)
    print(f"n64_t500: FP64 re-ranks {rr}, exhaustive {ex}, of about {queries} (query, E) selections")
    assert rr + ex <= 0.01 * queries
    sine = np.stack([synth.sine_series(240, 12.0), synth.sine_series(240, 12.0, phase=0.3)])
    edm.edm_knn_table(_dev(sine), 3)
    torch.cuda.synchronize()
    rr2, ex2 = edm.edm_knn_counters(reset=True)
    assert rr2 + ex2 > 0


def test_bulk_copies_complete_and_unaligned_rows(edm):
    """Series rows and target tiles reach shared memory by bulk copies on an
    mbarrier (16-byte aligned rows) or plain loads (other rows): both give
    the oracle's results, and no bounded wait gives up."""
    edm.edm_wait_timeouts(reset=True)
    # T = 301 with a row pitch of 301 floats: most rows start off a 16-byte
    # boundary (plain staging); a padded pitch of 304 aligns every row
    Y = synth.coupled_logistic(40, 301, 0.05, 0.05, seed_data=91, seed_noise=92)
    E = np.random.default_rng(93).integers(1, 7, size=40).astype(np.int32)
    R = orc.ccm_rho_rows(Y, E, rows=np.arange(6))
    for pitch in (301, 304):
        buf = torch.zeros((40, pitch), dtype=torch.float32, device="cuda")
        buf[:, :301] = _dev(Y)
        got = edm.edm_ccm_rho(buf[:, :301], torch.from_numpy(E).cuda()).cpu().numpy()[:, :6].T
        assert np.abs(got - R).max() < RHO_TOL, pitch
    assert edm.edm_wait_timeouts(reset=True) == 0
