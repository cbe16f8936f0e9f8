"""Adjoint on the batched workload itself: 256 datasets (N ~ U[32, 1024],
T ~ U[200, 3000], master seed 4), L = (sum over datasets and pairs of rho) /
sum_d N_d^2 with indices and optE frozen.  The gradient from the batched
adjoint against central differences (h = 1e-3) of the oracle's
frozen-index rho on 50 entries drawn (seed 5) uniformly over every series
value of the workload.

A central difference only measures the derivative where the frozen-index
rho is smooth on the scale of h: an entry that enters a table row whose
nearest distance d_1 is within 3h (its weights exp(-d/d_1) change within
the step) is skipped, as in the small batched test; at least 20 of the 50
must be checked."""

import numpy as np
import pytest
import torch

import edm_synth as synth
from oracle import oracle as orc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def edm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2011_11082_gb300 as m

    return m


def _min_d1_touching(x, t, Es, table):
    """Smallest d_1 over library x's table rows (tau = 1) whose query vector or
    a neighbour vector contains x(t)."""
    m = np.inf
    for E in Es:
        idx = table(E)
        d1 = np.sqrt(orc.ccm_table_d2(x, E, idx)[:, 0])
        q = np.arange(idx.shape[0]) + (E - 1)
        rows = ((q >= t) & (q <= t + E - 1)) | ((idx >= t) & (idx <= t + E - 1)).any(axis=1)
        if rows.any():
            m = min(m, float(d1[rows].min()))
    return m


def test_config4_gradient_against_central_differences(edm):
    specs = synth.batched_specs()
    data = [synth.batched_dataset(sp) for sp in specs]
    Ys = [torch.from_numpy(Y).cuda() for Y in data]
    b = edm.CCMBatch(Ys, E_max=20)
    optE, _ = b.run()
    grads = b.mean_rho_grad()
    torch.cuda.synchronize()
    total = float(sum(Y.shape[0] ** 2 for Y in data))
    sizes = np.array([Y.size for Y in data], dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(5)
    picks = rng.integers(0, int(starts[-1]), size=50)
    h = 1e-3
    cache = {}
    checked = 0
    for p in picks:
        d = int(np.searchsorted(starts, p, side="right") - 1)
        N, T = data[d].shape
        a, t = divmod(int(p - starts[d]), T)
        Y64 = data[d].astype(np.float64)
        oE = optE[d].cpu().numpy()
        Ea = int(oE[a])

        def tab_lib(E):  # library a's table at E
            key = ("lib", d, a, E)
            if key not in cache:
                cache[key] = orc.ccm_table(Y64[a], E)[0]
            return cache[key]

        key = ("all", d, Ea)  # every library's table at the target's E
        if key not in cache:
            cache[key] = orc.ccm_tables(Y64, Ea)
        tabs_Ea = cache[key]
        if _min_d1_touching(Y64[a], t, sorted(set(oE.tolist())), tab_lib) < 3 * h:
            continue

        def L_of(Yv):  # every rho that involves series a (others are constant)
            s = 0.0
            for j in range(N):
                s += orc.rho_frozen(Yv[a], Yv[j], int(oE[j]), tab_lib(int(oE[j])))
            for i in range(N):
                if i != a:
                    s += orc.rho_frozen(Yv[i], Yv[a], Ea, tabs_Ea[i])
            return s

        def fd_at(hh):
            Yp, Ym = Y64.copy(), Y64.copy()
            Yp[a, t] += hh
            Ym[a, t] -= hh
            return (L_of(Yp) - L_of(Ym)) / (2 * hh)

        fd, fd2 = fd_at(h), fd_at(h / 2)
        trunc = abs(fd - fd2) * 4.0 / 3.0
        g = float(grads[d][a, t]) * total  # d(sum of rho)/dY[a, t]
        checked += 1
        assert abs(fd - g) < 1e-6 + 1e-2 * abs(fd) + 1.5 * trunc, (d, a, t, N, T, fd, g, trunc)
    assert checked >= 20, checked
