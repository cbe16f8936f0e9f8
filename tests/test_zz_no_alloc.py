"""The allocation-free cross map, edm_ccm_rho_noalloc, against edm_ccm_rho.

Some callers cannot allocate device memory while they run: real-time loops
that must not hit the allocator, or hosts (plugins, embedded runtimes) that
hand this library a stream but no memory pool.  edm_ccm_rho_noalloc serves
them: it takes the same inputs and outputs as edm_ccm_rho but keeps its
scratch in a fixed, statically allocated device array instead of a
caller-provided workspace.  This file is collected last (tests/test_zz_*)
so that a first-failure run has already run every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

import edm_synth as synth

pytestmark = pytest.mark.gpu


def _fn(lib):
    from paper_2011_11082_gb300._abi import edm_params

    fn = lib.edm_ccm_rho_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                   ctypes.c_int64, ctypes.POINTER(edm_params), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return fn


def _call(lib, Y, optE, out, lib_begin, lib_count, params):
    N, T = Y.shape
    return _fn(lib)(Y.data_ptr(), N, T, T, optE.data_ptr(), lib_begin, lib_count, ctypes.byref(params),
                                   out.data_ptr(), out.shape[1], torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_workspace_path_on_two_calls():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2011_11082_gb300 as edm
    from paper_2011_11082_gb300 import _abi

    lib = _abi.load()
    for precision in (edm.EDM_PRECISION_FP32, edm.EDM_PRECISION_FP16_TARGETS):
        p = edm.make_params(precision=precision)
        for call, seed in enumerate((41, 43)):
            Y = synth.coupled_logistic(300, 400, 0.05, 0.05, seed_data=seed, seed_noise=seed + 1)
            Yd = torch.from_numpy(Y).cuda()
            optE, _ = edm.edm_optimal_E(Yd, E_max=8, return_rho=False)
            ref = edm.edm_ccm_rho(Yd, optE, precision=precision)
            out = torch.full((300, 300), float("nan"), device="cuda")
            assert _call(lib, Yd, optE, out, 0, 300, p) == 0
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert (out - ref).abs().max().item() < 1e-4, (precision, call)
            # a library sub-range into a narrower buffer
            blk = torch.full((300, 70), float("nan"), device="cuda")
            assert _call(lib, Yd, optE, blk, 100, 70, p) == 0
            torch.cuda.synchronize()
            assert (blk - ref[:, 100:170]).abs().max().item() < 1e-4, (precision, call)


def test_noalloc_rejects_sizes_beyond_its_array():
    import paper_2011_11082_gb300 as edm
    from paper_2011_11082_gb300 import _abi

    lib = _abi.load()
    p = edm.make_params()
    fake = ctypes.c_void_p(0x1000)  # not dereferenced: the size check comes first
    st = _fn(lib)(fake, 50000, 1500, 1500, fake, 0, 50000, ctypes.byref(p), fake, 50000, None)
    assert st == 3


def test_noalloc_non_default_parameters_and_bad_optE():
    """A seeded draw of tau, Tp and exclusion radius (FP16 tile widths under
    a non-default Tp included) matches edm_ccm_rho; an optE outside
    1..EDM_MAX_E and a flag the call does not offer are rejected."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2011_11082_gb300 as edm
    from paper_2011_11082_gb300 import _abi

    lib = _abi.load()
    rng = np.random.default_rng(47)
    tau, Tp, excl = int(rng.integers(2, 4)), int(rng.integers(2, 4)), int(rng.integers(1, 4))
    N, T = 90, 500
    Y = synth.coupled_logistic(N, T, 0.05, 0.05, seed_data=48, seed_noise=49)
    Yd = torch.from_numpy(Y).cuda()
    E = torch.from_numpy(rng.integers(1, 12, size=N).astype(np.int32)).cuda()
    for precision in (edm.EDM_PRECISION_FP32, edm.EDM_PRECISION_FP16_TARGETS):
        p = edm.make_params(tau=tau, Tp=Tp, exclusion_radius=excl, precision=precision)
        ref = edm.edm_ccm_rho(Yd, E, tau=tau, Tp=Tp, exclusion_radius=excl, precision=precision)
        out = torch.full((N, N), float("nan"), device="cuda")
        assert _call(lib, Yd, E, out, 0, N, p) == 0
        torch.cuda.synchronize()
        assert (out - ref).abs().max().item() < 1e-4, (precision, tau, Tp, excl)
    p = edm.make_params()
    out = torch.zeros((N, N), device="cuda")
    for bad in (0, edm.EDM_MAX_E + 1):
        Eb = E.clone()
        Eb[N // 2] = bad
        assert _call(lib, Yd, Eb, out, 0, N, p) == 1  # EDM_ERR_INVALID
    assert _call(lib, Yd, E, out, 0, N, edm.make_params(flags=edm.EDM_FLAG_LOOKUP_SCALAR)) == 5  # UNSUPPORTED
