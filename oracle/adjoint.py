"""FP64 reference gradient of the cross-map rho with the neighbour indices frozen.

TEST INFRASTRUCTURE (same rules as ``oracle.py``).  The paper has no
gradients; this is the derivative of its rho (Sec. II-B simplex weights,
Algorithm 5 lookup, Pearson corrcoef) with respect to the series values,
holding every kNN index (and every optimal E) fixed at the values found on
the unperturbed data.  Written with plain PyTorch CPU float64 ops so autograd
does the calculus; it shares no code with the C oracle or the CUDA adjoint.

Reading at d = 0: the distance is sqrt(d^2) with gradient 0 where d^2 = 0,
and when the nearest distance is 0 the duplicate-only weights are constant.
"""

from __future__ import annotations

import torch


def _safe_sqrt(d2: torch.Tensor) -> torch.Tensor:
    pos = d2 > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, d2, torch.ones_like(d2))), torch.zeros_like(d2))


def rho_frozen(x: torch.Tensor, y: torch.Tensor, E: int, idx: torch.Tensor, tau: int = 1, Tp: int = 1) -> torch.Tensor:
    """rho(library x -> target y) for a frozen table ``idx`` [nq][E+1] of
    unshifted candidate times; rows are queries t = (E-1)tau + r."""
    L = (E - 1) * tau
    nq = idx.shape[0]
    t = torch.arange(L, L + nq)
    lags = torch.arange(E) * tau
    Vq = x[t[:, None] - lags[None, :]]  # [nq][E]
    Vc = x[idx[:, :, None] - lags[None, None, :]]  # [nq][k][E]
    diff = Vq[:, None, :] - Vc
    d = _safe_sqrt((diff * diff).sum(-1))  # [nq][k]
    d1 = d[:, :1]
    has = d1 > 0
    ratio = d / torch.where(has, d1, torch.ones_like(d1))
    u = torch.where(has, torch.exp(-ratio), (d == 0).to(d.dtype))
    w = u / u.sum(1, keepdim=True)
    p = (w * y[idx + Tp]).sum(1)
    o = y[t + Tp]
    pc = p - p.mean()
    oc = o - o.mean()
    return (pc * oc).sum() / torch.sqrt((pc * pc).sum() * (oc * oc).sum())


def mean_rho_and_grad(Y, optE, tables, tau: int = 1, Tp: int = 1):
    """L = mean over all (library i, target j) of rho_ij with frozen tables.

    ``tables[(i, E)]`` holds the int64 index table of library i at dimension
    E.  Returns (L, dL/dY) as float64 numpy arrays (Y is [N][T])."""
    import numpy as np

    Yt = torch.tensor(np.asarray(Y, dtype=np.float64), requires_grad=True)
    N = Yt.shape[0]
    total = torch.zeros((), dtype=torch.float64)
    for i in range(N):
        for j in range(N):
            E = int(optE[j])
            idx = torch.as_tensor(np.asarray(tables[(i, E)], dtype=np.int64))
            total = total + rho_frozen(Yt[i], Yt[j], E, idx, tau, Tp)
    Lval = total / (N * N)
    Lval.backward()
    return float(Lval.detach()), Yt.grad.detach().numpy().copy()
