"""Precision form at N = 16,384, T = 1,500: rho error of the plain FP32 form
and of the FP16-target form against the FP64 oracle on 10,000 seeded random
(library, target) pairs (seed 3), with the GPU's optimal E.

Bars: FP32 within 1e-4 absolute, FP16 targets within 1e-3 absolute.  The
error statistics are printed (run with -s to see them).
"""

import json

import numpy as np
import pytest
import torch

import edm_synth as synth
from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def edm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2011_11082_gb300 as m

    return m


def test_precision_form_n16384_10000_pairs(edm):
    Y = synth.workload("n16384_t1500")
    Yd = torch.from_numpy(Y).cuda()
    optE, _ = edm.edm_optimal_E(Yd, E_max=20)
    oE = optE.cpu().numpy()
    li, lj = synth.sample_pairs(Y.shape[0], 10000, seed=3)
    R = orc.ccm_rho_pairs(Y, oE, li, lj)
    stats = {}
    for name, prec, tol in (("fp32", edm.EDM_PRECISION_FP32, 1e-4), ("fp16_targets", edm.EDM_PRECISION_FP16_TARGETS, 1e-3)):
        rho_t = edm.edm_ccm_rho(Yd, optE, precision=prec)  # target-major
        got = rho_t.cpu().numpy()[lj, li].astype(np.float64)
        err = np.abs(got - R)
        stats[name] = {"max": float(err.max()), "mean": float(err.mean()), "p99": float(np.quantile(err, 0.99))}
        del rho_t
        torch.cuda.empty_cache()
        assert err.max() < tol, (name, stats[name])
    print("rho error vs FP64 oracle, 10,000 pairs, N=16384 T=1500:", json.dumps(stats))
