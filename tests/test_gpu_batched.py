"""Batched form (edm_ccm_rho_batched) through the C ABI: equal to the
per-dataset entry points, replays its captured graph on new data, agrees
with the FP64 oracle at the batched workload's full sizes, and its adjoint
matches finite differences of the oracle."""

import numpy as np
import pytest
import torch

import edm_synth as synth
from oracle import adjoint
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


def _small_batch(seed, count=7, n_range=(9, 140), t_range=(120, 1700)):
    specs = synth.batched_specs(count, master_seed=seed, n_range=n_range, t_range=t_range)
    return [synth.batched_dataset(s, density=0.05, b_max=0.05) for s in specs]


def _per_dataset(edm, Ys, E_max, precision):
    # The batched form builds every table with the warp-per-query kernel
    # (its E set is planned on the device); the per-dataset call is asked
    # for the same kernel, so a dataset's results are the same bits.  (By
    # default a single-E table set with E <= 6 uses the thread-per-query
    # kernel: same neighbours, weights equal up to summation order.)
    out = []
    for Y in Ys:
        optE, _ = edm.edm_optimal_E(Y, E_max=E_max, return_rho=False)
        out.append((optE, edm.edm_ccm_rho(Y, optE, precision=precision, flags=edm.EDM_FLAG_KNN_WARP)))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_per_dataset_calls(edm, precision):
    Ys = [_dev(Y) for Y in _small_batch(21)]
    b = edm.CCMBatch(Ys, E_max=8, precision=precision)
    optE, rho = b.run()
    torch.cuda.synchronize()
    ref = _per_dataset(edm, Ys, 8, precision)
    for d, (oE, r) in enumerate(ref):
        assert torch.equal(optE[d], oE), d
        # same kernels and tile shapes within a dataset: identical bits
        diff = (rho[d] - r).abs().max().item()
        assert diff == 0.0 or diff < 1e-6, (d, diff)


def test_batched_graph_replays_on_new_data(edm):
    from paper_2011_11082_gb300 import _abi

    lib = _abi.load()
    first = _small_batch(22)
    # new data of the same shapes (the graph holds the buffers, not values)
    second = [synth.coupled_logistic(Y.shape[0], Y.shape[1], 0.05, 0.05, seed_data=100 + d, seed_noise=200 + d)
              for d, Y in enumerate(first)]
    Ys = [_dev(Y) for Y in first]
    b = edm.CCMBatch(Ys, E_max=8)
    b.run()
    torch.cuda.synchronize()
    n0 = lib.edm_launch_count(_abi.EDM_KERNEL_LOOKUP)
    for Yd, Y2 in zip(Ys, second):
        Yd.copy_(_dev(Y2))
    optE, rho = b.run()
    torch.cuda.synchronize()
    assert lib.edm_launch_count(_abi.EDM_KERNEL_LOOKUP) - n0 == len(Ys)  # one lookup per dataset per replay
    for d, (oE, r) in enumerate(_per_dataset(edm, Ys, 8, 0)):
        assert torch.equal(optE[d], oE), d
        assert (rho[d] - r).abs().max().item() < 1e-6, d
    # and against the oracle on one dataset of the new data
    d = int(np.argmax([Y.shape[0] for Y in second]))
    oE, _ = orc.optimal_E(second[d], 8)
    assert np.array_equal(optE[d].cpu().numpy(), oE)
    R = orc.ccm_rho_rows(second[d], oE)
    assert np.abs(rho[d].t().cpu().numpy() - R).max() < RHO_TOL


def test_batched_small_datasets_against_oracle(edm):
    """Every optE and every rho of small uneven datasets against the FP64
    oracle (the batched path has its own device-side planning)."""
    data = _small_batch(24, count=3, n_range=(10, 40), t_range=(150, 400)) + _small_batch(25, count=3)
    b = edm.CCMBatch([_dev(Y) for Y in data], E_max=6)
    optE, rho = b.run()
    torch.cuda.synchronize()
    for d, Y in enumerate(data):
        oE, orho = orc.optimal_E(Y, 6)
        got = optE[d].cpu().numpy()
        bad = np.nonzero(got != oE)[0]
        assert bad.size == 0, (d, Y.shape, [(int(k), int(got[k]), int(oE[k]), orho[k].tolist()) for k in bad[:3]])
        R = orc.ccm_rho_rows(Y, oE)
        assert np.abs(rho[d].t().cpu().numpy() - R).max() < RHO_TOL, d


@pytest.mark.slow
def test_batched_workload_full_size_samples(edm):
    """The 256-dataset batched workload (N ~ U[32, 1024], T ~ U[200, 3000],
    E_max = 20): optE of sampled series and rho of sampled pairs against the
    oracle, in the graph-replayed launch configuration."""
    specs = synth.batched_specs()
    data = [synth.batched_dataset(s) for s in specs]
    Ys = [_dev(Y) for Y in data]
    b = edm.CCMBatch(Ys, E_max=20)
    b.run()
    optE, rho = b.run()  # replay
    torch.cuda.synchronize()
    rng = np.random.default_rng(6)
    for d in rng.choice(len(specs), 6, replace=False):
        Y = data[d]
        N = Y.shape[0]
        got_E = optE[d].cpu().numpy()
        rows = rng.choice(N, min(N, 12), replace=False)
        oE, orho = orc.optimal_E(Y[rows], 20)
        bad = np.nonzero(got_E[rows] != oE)[0]
        assert bad.size == 0, (int(d), [(int(rows[k]), int(got_E[rows[k]]), int(oE[k])) for k in bad[:3]])
        li, lj = synth.sample_pairs(N, 24, seed=int(d))
        R = orc.ccm_rho_pairs(Y, got_E, li, lj)
        G = rho[d].cpu().numpy()[lj, li]
        assert np.abs(G - R).max() < RHO_TOL, int(d)


def test_batched_mean_rho_gradient(edm):
    """L = (sum over datasets and pairs of rho) / sum_d N_d^2 (indices and
    optE frozen).  The batched adjoint against (1) the FP64 reference
    gradient -- PyTorch float64 autograd through the oracle's frozen tables
    -- on every entry of every dataset, and (2) central differences
    (h = 1e-3) of the oracle's frozen-index rho on 50 sampled entries
    (seed 5).  A central difference only measures the derivative where the
    frozen-index rho is smooth on the scale of h: where a table row that
    Y[a, t] enters (a query vector or a neighbour vector containing x_a(t))
    has its nearest distance d_1 within a few h, the weights exp(-d/d_1)
    change within the step.  Samples with such a row (d_1 < 3h) are covered
    by check (1) only."""
    data = _small_batch(24, count=3, n_range=(10, 40), t_range=(150, 400))
    Ys = [_dev(Y) for Y in data]
    b = edm.CCMBatch(Ys, E_max=6)
    optE, _ = b.run()
    grads = [g.cpu().numpy() for g in b.mean_rho_grad()]
    total = float(sum(Y.shape[0] ** 2 for Y in data))
    tabs = {}

    def tab(d, i, E):
        if (d, i, E) not in tabs:
            tabs[(d, i, E)] = orc.ccm_table(data[d][i].astype(np.float64), E)[0]
        return tabs[(d, i, E)]

    # (1) FP64 reference gradient, every entry
    for d, Y in enumerate(data):
        N = Y.shape[0]
        oE = optE[d].cpu().numpy()
        Yt = torch.tensor(Y.astype(np.float64), requires_grad=True)
        s = 0
        for i in range(N):
            for j in range(N):
                E = int(oE[j])
                s = s + adjoint.rho_frozen(Yt[i], Yt[j], E, torch.as_tensor(tab(d, i, E)))
        (s / total).backward()
        G = Yt.grad.numpy()
        assert np.abs(grads[d] - G).max() < 1e-4 * np.abs(G).max() + 1e-7, d

    # (2) central differences on 50 sampled entries
    rng = np.random.default_rng(5)
    h = 1e-3
    checked = 0
    for _ in range(50):
        d = int(rng.integers(0, len(data)))
        Y64 = data[d].astype(np.float64)
        N, T = Y64.shape
        oE = optE[d].cpu().numpy()
        a, t = int(rng.integers(0, N)), int(rng.integers(0, T))

        def L_of(Yv):
            s = 0.0
            for j in range(N):
                s += orc.rho_frozen(Yv[a], Yv[j], int(oE[j]), tab(d, a, int(oE[j])))
            for i in range(N):
                if i != a:
                    s += orc.rho_frozen(Yv[i], Yv[a], int(oE[a]), tab(d, i, int(oE[a])))
            return s / total

        def fd_at(hh):
            Yp, Ym = Y64.copy(), Y64.copy()
            Yp[a, t] += hh
            Ym[a, t] -= hh
            return (L_of(Yp) - L_of(Ym)) / (2 * hh)

        if _min_d1_touching(data[d][a].astype(np.float64), t, sorted(set(oE.tolist())),
                            lambda E: tab(d, a, E)) < 3 * h:
            continue  # not smooth on the scale of h (near-duplicate point)
        fd, fd2 = fd_at(h), fd_at(h / 2)
        checked += 1
        trunc = abs(fd - fd2) * 4.0 / 3.0  # O(h^2) truncation estimate
        g = grads[d][a, t]
        assert abs(fd - g) < 1e-6 + 1e-2 * abs(fd) + 1.5 * trunc, (d, a, t, fd, g, trunc)
    assert checked >= 20, checked


def _min_d1_touching(x, t, Es, table):
    """Smallest nearest-neighbour distance d_1 over the rows of library x's
    tables (tau = 1) whose query vector or a neighbour vector contains x(t)."""
    m = np.inf
    for E in Es:
        idx = table(E)
        d1 = np.sqrt(orc.ccm_table_d2(x, E, idx)[:, 0])
        q = np.arange(idx.shape[0]) + (E - 1)
        rows = ((q >= t) & (q <= t + E - 1)) | ((idx >= t) & (idx <= t + E - 1)).any(axis=1)
        if rows.any():
            m = min(m, float(d1[rows].min()))
    return m
