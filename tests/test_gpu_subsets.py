"""CCM convergence (edm_ccm_rho_subsets) through the C ABI against the FP64
oracle: library subsets of several sizes, the full library reducing to the
plain cross map, convergence of rho with library size on a deterministic
series, and the rejection of subsets too small for the largest E."""

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


def _masks_dev(m):
    return torch.from_numpy(m.view(np.int32)).cuda()


@pytest.mark.parametrize("excl", [0, 3])
def test_subsets_match_oracle(edm, excl):
    Y = synth.coupled_logistic(20, 300, 0.08, 0.05, seed_data=81, seed_noise=82)
    oE, _ = orc.optimal_E(Y, 6)
    masks = synth.library_subsets(300, 5, 298, sizes=(40, 120, 250), samples=2, seed=9)
    R = orc.ccm_rho_subsets(Y, oE, masks, excl=excl)  # [u][lib][tgt]
    G = edm.edm_ccm_rho_subsets(_dev(Y), torch.from_numpy(oE).cuda(), _masks_dev(masks),
                                exclusion_radius=excl).cpu().numpy()  # [u][tgt][lib]
    assert np.abs(np.transpose(G, (0, 2, 1)) - R).max() < RHO_TOL


def test_full_library_is_the_plain_cross_map(edm):
    Y = synth.coupled_logistic(33, 400, 0.08, 0.05, seed_data=83, seed_noise=84)
    oE, _ = orc.optimal_E(Y, 6)
    Yd, Ed = _dev(Y), torch.from_numpy(oE).cuda()
    full = np.full((1, (400 + 31) // 32), 0xFFFFFFFF, np.uint32)
    a = edm.edm_ccm_rho_subsets(Yd, Ed, _masks_dev(full))[0]
    b = edm.edm_ccm_rho(Yd, Ed, flags=edm.EDM_FLAG_KNN_WARP)
    assert torch.equal(a, b)


def test_skill_converges_with_library_size(edm):
    """Logistic map cross-mapping itself (leave-one-out): the mean skill over
    random libraries grows with the library size."""
    x = synth.logistic_series(600)
    Y = np.stack([x, synth.logistic_series(600, x0=0.31)])
    oE = np.array([2, 2], np.int32)
    sizes = (20, 60, 200, 560)
    masks = synth.library_subsets(600, 1, 598, sizes=sizes, samples=4, seed=10)
    G = edm.edm_ccm_rho_subsets(_dev(Y), torch.from_numpy(oE).cuda(), _masks_dev(masks)).cpu().numpy()
    curve = G[:, 0, 0].reshape(len(sizes), 4).mean(axis=1)
    assert np.all(np.diff(curve) > 0), curve
    R = orc.ccm_rho_subsets(Y, oE, masks)
    assert np.abs(np.transpose(G, (0, 2, 1)) - R).max() < RHO_TOL


def test_subset_too_small_is_rejected(edm):
    """A subset that leaves fewer than E+1 candidates: EDM_ERR_INVALID with
    EDM_FLAG_VALIDATE (checked on the host), else a NaN plane (checked on the
    device, no host synchronisation)."""
    Y = synth.coupled_logistic(4, 200, 0.08, 0.05, seed_data=85, seed_noise=86)
    masks = synth.library_subsets(200, 5, 198, sizes=(5,), samples=1, seed=11)
    full = np.full((1, (200 + 31) // 32), 0xFFFFFFFF, np.uint32)
    E = torch.full((4,), 6, dtype=torch.int32, device="cuda")
    with pytest.raises(edm.EdmError) as ei:
        edm.edm_ccm_rho_subsets(_dev(Y), E, _masks_dev(masks), flags=edm.EDM_FLAG_VALIDATE)
    assert ei.value.status == 1
    G = edm.edm_ccm_rho_subsets(_dev(Y), E, _masks_dev(np.concatenate([masks, full]))).cpu().numpy()
    assert np.isnan(G[0]).all() and np.isfinite(G[1]).all()
