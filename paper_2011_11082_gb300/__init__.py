"""GB300-native all-pairs Convergent Cross Mapping (the mpEDM hot path).

Thin Python binding over the C ABI of ``include/edm.h`` (libedm.so, built
in-tree for sm_103a).  Functions carry the C names; they only marshal torch
CUDA tensors into pointers, sizes and the current stream.  Every step of the
computation runs in the CUDA kernels; there is no CPU fallback, and the
first call fails loudly if the library or a GPU is missing.
"""

from __future__ import annotations

import ctypes

import torch

from . import _abi
from ._abi import (
    EDM_MAX_E,
    EDM_PRECISION_FP16_TARGETS,
    EDM_PRECISION_FP32,
    EDM_FLAG_LOOKUP_SCALAR,
    EDM_FLAG_VALIDATE,
    EDM_FLAG_KNN_WARP,
    EdmError,
    edm_params,
)

__all__ = [
    "edm_optimal_E",
    "edm_knn_table",
    "edm_ccm_rho",
    "edm_ccm_workspace_bytes",
    "edm_ccm_host",
    "edm_ccm_rho_lags",
    "edm_ccm_rho_subsets",
    "edm_ccm_rho_backward",
    "edm_ccm_backward_workspace_bytes",
    "edm_ccm_rho_batched",
    "edm_knn_counters",
    "edm_wait_timeouts",
    "CCMBatch",
    "ccm",
    "ccm_rho_autograd",
    "CCMRhoFunction",
    "make_params",
    "EdmError",
    "EDM_MAX_E",
]


def make_params(E_max=20, tau=1, Tp=1, exclusion_radius=0, precision=EDM_PRECISION_FP32, flags=0) -> edm_params:
    return edm_params(int(E_max), int(tau), int(Tp), int(exclusion_radius), int(precision), int(flags))


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ld(t: torch.Tensor) -> int:
    """Row pitch in elements (a single row's stride is meaningless)."""
    return int(t.stride(0)) if t.shape[0] > 1 else int(t.shape[1])


def _dev_f32(Y: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(Y, torch.Tensor) and Y.is_cuda and Y.dtype == torch.float32):
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if Y.dim() != 2 or Y.stride(1) != 1:
        raise TypeError(f"{name} must be 2-D [N][T] with unit stride along T")
    return Y


def edm_optimal_E(Y: torch.Tensor, E_max: int = 20, tau: int = 1, Tp: int = 1, return_rho: bool = True,
                  stream=None, flags: int = 0):
    """Phase 1 (simplex projection): optE int32[N] and rho_by_E float32[N][E_max].
    ``flags=EDM_FLAG_VALIDATE`` first checks Y for non-finite values (the
    error names the first bad series)."""
    lib = _abi.load()
    Y = _dev_f32(Y, "Y")
    N, T = Y.shape
    optE = torch.empty(N, dtype=torch.int32, device=Y.device)
    rho = torch.empty((N, E_max), dtype=torch.float32, device=Y.device) if return_rho else None
    p = make_params(E_max=E_max, tau=tau, Tp=Tp, flags=flags)
    st = lib.edm_optimal_E(Y.data_ptr(), N, T, _ld(Y), ctypes.byref(p), optE.data_ptr(),
                           rho.data_ptr() if rho is not None else None, _stream(stream))
    _abi.check(st, "edm_optimal_E")
    return optE, rho


def edm_knn_table(Y: torch.Tensor, E: int, tau: int = 1, Tp: int = 1, exclusion_radius: int = 0, stream=None,
                  flags: int = 0):
    """Phase-2 kNN tables of every row of Y at dimension E:
    idx int32[n][Tq][E+1] (neighbour times, unshifted) and w float32[n][Tq][E+1]."""
    lib = _abi.load()
    Y = _dev_f32(Y, "Y")
    n, T = Y.shape
    Tq = T - Tp - (E - 1) * tau
    if Tq < 1:
        raise ValueError("series too short for this E")
    idx = torch.empty((n, Tq, E + 1), dtype=torch.int32, device=Y.device)
    w = torch.empty((n, Tq, E + 1), dtype=torch.float32, device=Y.device)
    p = make_params(E_max=E, tau=tau, Tp=Tp, exclusion_radius=exclusion_radius, flags=flags)
    st = lib.edm_knn_table(Y.data_ptr(), n, T, _ld(Y), E, ctypes.byref(p), idx.data_ptr(), w.data_ptr(), Tq,
                           _stream(stream))
    _abi.check(st, "edm_knn_table")
    return idx, w


def edm_knn_counters(reset: bool = True) -> tuple[int, int]:
    """(queries re-ranked in FP64, queries re-solved by an exhaustive FP64
    scan) by the kNN kernels since the last reset (synchronises)."""
    lib = _abi.load()
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _abi.check(lib.edm_knn_counters(ctypes.byref(a), ctypes.byref(b), 1 if reset else 0), "edm_knn_counters")
    return int(a.value), int(b.value)


def edm_wait_timeouts(reset: bool = True) -> int:
    """Bounded bulk-copy waits of the kNN, lookup and adjoint kernels that
    gave up since the last reset (0 in a healthy run; synchronises)."""
    lib = _abi.load()
    a = ctypes.c_int64()
    _abi.check(lib.edm_wait_timeouts(ctypes.byref(a), 1 if reset else 0), "edm_wait_timeouts")
    return int(a.value)


def edm_ccm_workspace_bytes(N: int, T: int, tau: int = 1, Tp: int = 1, exclusion_radius: int = 0,
                            precision: int = EDM_PRECISION_FP32) -> int:
    lib = _abi.load()
    p = make_params(tau=tau, Tp=Tp, exclusion_radius=exclusion_radius, precision=precision)
    return int(lib.edm_ccm_workspace_bytes(N, T, ctypes.byref(p)))


def edm_ccm_rho(Y: torch.Tensor, optE: torch.Tensor, lib_begin: int = 0, lib_count: int | None = None,
                tau: int = 1, Tp: int = 1, exclusion_radius: int = 0, precision: int = EDM_PRECISION_FP32,
                out: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None,
                flags: int = 0) -> torch.Tensor:
    """Phase 2 cross map for libraries [lib_begin, lib_begin+lib_count).

    Returns the TARGET-MAJOR block ``out[j][i - lib_begin] = rho(library i ->
    target j)`` of shape [N][lib_count]; ``out.t()`` is the library-major map."""
    lib = _abi.load()
    Y = _dev_f32(Y, "Y")
    N, T = Y.shape
    if lib_count is None:
        lib_count = N - lib_begin
    if not (optE.is_cuda and optE.dtype == torch.int32 and optE.numel() == N and optE.is_contiguous()):
        raise TypeError("optE must be a contiguous int32 CUDA tensor of N entries")
    if out is None:
        out = torch.empty((N, lib_count), dtype=torch.float32, device=Y.device)
    if not (out.is_cuda and out.dtype == torch.float32 and out.dim() == 2 and out.stride(1) == 1
            and out.shape[0] == N and out.shape[1] >= lib_count):
        raise TypeError("out must be a float32 CUDA tensor [N][>=lib_count] with unit inner stride")
    if lib_count == 0 and 0 <= lib_begin <= N:
        return out  # an empty library range: nothing to compute (an empty tensor has no data pointer)
    p = make_params(tau=tau, Tp=Tp, exclusion_radius=exclusion_radius, precision=precision, flags=flags)
    need = int(lib.edm_ccm_workspace_bytes(N, T, ctypes.byref(p)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=Y.device)
    st = lib.edm_ccm_rho(Y.data_ptr(), N, T, _ld(Y), optE.data_ptr(), lib_begin, lib_count, ctypes.byref(p),
                         out.data_ptr(), _ld(out), workspace.data_ptr(), workspace.numel(), _stream(stream))
    _abi.check(st, "edm_ccm_rho")
    return out


def edm_ccm_rho_lags(Y: torch.Tensor, optE: torch.Tensor, lag_min: int, lag_max: int, tau: int = 1,
                     exclusion_radius: int = 0, precision: int = EDM_PRECISION_FP32, out: torch.Tensor | None = None,
                     workspace: torch.Tensor | None = None, stream=None, flags: int = 0) -> torch.Tensor:
    """Time-delay cross mapping: out[l - lag_min][j][i] = rho_l(library i ->
    target j) for every lag in lag_min..lag_max, one table per (library, E)."""
    lib = _abi.load()
    Y = _dev_f32(Y, "Y")
    N, T = Y.shape
    if not (optE.is_cuda and optE.dtype == torch.int32 and optE.numel() == N and optE.is_contiguous()):
        raise TypeError("optE must be a contiguous int32 CUDA tensor of N entries")
    n_lags = lag_max - lag_min + 1
    if out is None:
        out = torch.empty((n_lags, N, N), dtype=torch.float32, device=Y.device)
    if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and tuple(out.shape[:2]) == (n_lags, N)):
        raise TypeError("out must be a contiguous float32 CUDA tensor [n_lags][N][>=N]")
    p = make_params(tau=tau, Tp=max(lag_max, 0), exclusion_radius=exclusion_radius, precision=precision, flags=flags)
    need = int(lib.edm_ccm_rho_lags_workspace_bytes(N, T, lag_min, lag_max, ctypes.byref(p)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=Y.device)
    st = lib.edm_ccm_rho_lags(Y.data_ptr(), N, T, _ld(Y), optE.data_ptr(), lag_min, lag_max, ctypes.byref(p),
                              out.data_ptr(), out.shape[2], workspace.data_ptr(), workspace.numel(), _stream(stream))
    _abi.check(st, "edm_ccm_rho_lags")
    return out


def edm_ccm_rho_subsets(Y: torch.Tensor, optE: torch.Tensor, masks: torch.Tensor, tau: int = 1, Tp: int = 1,
                        exclusion_radius: int = 0, precision: int = EDM_PRECISION_FP32,
                        out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                        stream=None, flags: int = 0) -> torch.Tensor:
    """CCM convergence: out[u][j][i] = rho(library i -> target j) with each
    library's candidates restricted to subset u (masks: int32/uint32 CUDA
    tensor [n_sub][words], bit s = candidate time s allowed)."""
    lib = _abi.load()
    Y = _dev_f32(Y, "Y")
    N, T = Y.shape
    if not (optE.is_cuda and optE.dtype == torch.int32 and optE.numel() == N and optE.is_contiguous()):
        raise TypeError("optE must be a contiguous int32 CUDA tensor of N entries")
    if not (masks.is_cuda and masks.dtype in (torch.int32, torch.uint32) and masks.dim() == 2 and masks.is_contiguous()):
        raise TypeError("masks must be a contiguous 32-bit CUDA tensor [n_sub][words]")
    n_sub, words = masks.shape
    if out is None:
        out = torch.empty((n_sub, N, N), dtype=torch.float32, device=Y.device)
    p = make_params(tau=tau, Tp=Tp, exclusion_radius=exclusion_radius, precision=precision, flags=flags)
    need = int(lib.edm_ccm_workspace_bytes(N, T, ctypes.byref(p)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=Y.device)
    st = lib.edm_ccm_rho_subsets(Y.data_ptr(), N, T, _ld(Y), optE.data_ptr(), masks.data_ptr(), n_sub, words,
                                 ctypes.byref(p), out.data_ptr(), out.shape[2], workspace.data_ptr(),
                                 workspace.numel(), _stream(stream))
    _abi.check(st, "edm_ccm_rho_subsets")
    return out


def edm_ccm_host(Y_host: torch.Tensor, E_max: int = 20, tau: int = 1, Tp: int = 1, exclusion_radius: int = 0,
                 precision: int = EDM_PRECISION_FP32, rho_out: torch.Tensor | None = None, block: int = 0,
                 workspace: torch.Tensor | None = None, device=None, stream=None):
    """Both phases with host buffers: (optE int32[N], rho target-major
    float32[N][N]) in host memory.  Pass pinned tensors for full bandwidth."""
    lib = _abi.load()
    if Y_host.is_cuda or Y_host.dtype != torch.float32 or Y_host.dim() != 2 or not Y_host.is_contiguous():
        raise TypeError("Y_host must be a contiguous float32 CPU tensor [N][T]")
    N, T = Y_host.shape
    dev = torch.device("cuda") if device is None else torch.device(device)
    optE = torch.empty(N, dtype=torch.int32, pin_memory=Y_host.is_pinned())
    if rho_out is None:
        rho_out = torch.empty((N, N), dtype=torch.float32, pin_memory=Y_host.is_pinned())
    p = make_params(E_max=E_max, tau=tau, Tp=Tp, exclusion_radius=exclusion_radius, precision=precision)
    need = int(lib.edm_ccm_host_workspace_bytes(N, T, block, ctypes.byref(p)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    st = lib.edm_ccm_host(Y_host.data_ptr(), N, T, ctypes.byref(p), optE.data_ptr(), rho_out.data_ptr(),
                          rho_out.stride(0), block, workspace.data_ptr(), workspace.numel(),
                          _stream(stream if stream is not None else torch.cuda.current_stream(dev)))
    _abi.check(st, "edm_ccm_host")
    return optE, rho_out


class CCMBatch:
    """Many datasets (uneven N, T) through both phases in one graph launch.

    Holds the descriptors, the per-dataset outputs and the workspace, so that
    every ``run()`` passes identical arguments to ``edm_ccm_rho_batched`` and
    replays the CUDA graph captured on the first run.  ``optE[d]`` is int32
    [N_d]; ``rho[d]`` is TARGET-MAJOR float32 [N_d][N_d] (``rho[d].t()`` is
    the library-major map)."""

    def __init__(self, Ys, E_max: int = 20, tau: int = 1, Tp: int = 1, exclusion_radius: int = 0,
                 precision: int = EDM_PRECISION_FP32):
        self.lib = _abi.load()
        self.Ys = [_dev_f32(Y, f"Ys[{d}]") for d, Y in enumerate(Ys)]
        if not self.Ys:
            raise ValueError("empty batch")
        dev = self.Ys[0].device
        self.params = make_params(E_max=E_max, tau=tau, Tp=Tp, exclusion_radius=exclusion_radius,
                                  precision=precision)
        self.optE = [torch.empty(Y.shape[0], dtype=torch.int32, device=dev) for Y in self.Ys]
        self.rho = [torch.empty((Y.shape[0], Y.shape[0]), dtype=torch.float32, device=dev) for Y in self.Ys]
        n = len(self.Ys)
        self.sets = (_abi.edm_dataset * n)()
        for d, Y in enumerate(self.Ys):
            N, T = Y.shape
            self.sets[d] = _abi.edm_dataset(Y.data_ptr(), N, T, _ld(Y), self.optE[d].data_ptr(),
                                            self.rho[d].data_ptr(), N)
        need = int(self.lib.edm_ccm_rho_batched_workspace_bytes(self.sets, n, ctypes.byref(self.params)))
        if need == 0:
            _abi.check(_abi.EDM_ERR_INVALID, "edm_ccm_rho_batched_workspace_bytes")
        self.workspace = torch.empty(need, dtype=torch.uint8, device=dev)

    def run(self, stream=None):
        st = self.lib.edm_ccm_rho_batched(self.sets, len(self.Ys), ctypes.byref(self.params),
                                          self.workspace.data_ptr(), self.workspace.numel(), _stream(stream))
        _abi.check(st, "edm_ccm_rho_batched")
        return self.optE, self.rho

    def mean_rho_grad(self):
        """dL/dY_d for L = (sum over datasets and all pairs of rho) / sum_d N_d^2,
        indices and optE frozen at the last run's values."""
        total = float(sum(Y.shape[0] ** 2 for Y in self.Ys))
        p = self.params
        grads = []
        for Y, E in zip(self.Ys, self.optE):
            g = torch.full((Y.shape[0], Y.shape[0]), 1.0 / total, dtype=torch.float32, device=Y.device)
            grads.append(edm_ccm_rho_backward(Y, E, g, tau=p.tau, Tp=p.Tp, exclusion_radius=p.exclusion_radius))
        return grads


def edm_ccm_rho_batched(Ys, E_max: int = 20, tau: int = 1, Tp: int = 1, exclusion_radius: int = 0,
                        precision: int = EDM_PRECISION_FP32, stream=None):
    """One-shot batched form: (list of optE, list of target-major rho).  Use
    ``CCMBatch`` to replay the captured graph on repeated calls."""
    return CCMBatch(Ys, E_max=E_max, tau=tau, Tp=Tp, exclusion_radius=exclusion_radius,
                    precision=precision).run(stream)


def edm_ccm_backward_workspace_bytes(N: int, T: int, tau: int = 1, Tp: int = 1, exclusion_radius: int = 0) -> int:
    lib = _abi.load()
    p = make_params(tau=tau, Tp=Tp, exclusion_radius=exclusion_radius)
    return int(lib.edm_ccm_backward_workspace_bytes(N, T, ctypes.byref(p)))


def edm_ccm_rho_backward(Y: torch.Tensor, optE: torch.Tensor, grad_rho_t: torch.Tensor, tau: int = 1, Tp: int = 1,
                         exclusion_radius: int = 0, workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dL/dY for L = sum_ij G(i,j) rho(i,j), indices and optE frozen.

    ``grad_rho_t`` is TARGET-MAJOR like the forward output:
    grad_rho_t[j][i] = dL/d rho(library i -> target j)."""
    lib = _abi.load()
    Y = _dev_f32(Y, "Y")
    N, T = Y.shape
    if not (optE.is_cuda and optE.dtype == torch.int32 and optE.numel() == N and optE.is_contiguous()):
        raise TypeError("optE must be a contiguous int32 CUDA tensor of N entries")
    g = _dev_f32(grad_rho_t, "grad_rho_t")
    if g.shape[0] != N or g.shape[1] < N:
        raise TypeError("grad_rho_t must be [N][>=N]")
    grad = torch.empty_like(Y)
    p = make_params(tau=tau, Tp=Tp, exclusion_radius=exclusion_radius)
    need = int(lib.edm_ccm_backward_workspace_bytes(N, T, ctypes.byref(p)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=Y.device)
    st = lib.edm_ccm_rho_backward(Y.data_ptr(), N, T, _ld(Y), optE.data_ptr(), g.data_ptr(), _ld(g), ctypes.byref(p),
                                  grad.data_ptr(), workspace.data_ptr(), workspace.numel(), _stream(stream))
    _abi.check(st, "edm_ccm_rho_backward")
    return grad


class CCMRhoFunction(torch.autograd.Function):
    """rho(library i -> target j) as a differentiable function of the series
    (library-major N x N output); optE and the neighbour indices are held
    fixed, as in the adjoint entry point."""

    @staticmethod
    def forward(ctx, Y, optE, tau=1, Tp=1, exclusion_radius=0, precision=EDM_PRECISION_FP32):
        Yc = Y.contiguous()
        rho_t = edm_ccm_rho(Yc, optE, tau=tau, Tp=Tp, exclusion_radius=exclusion_radius, precision=precision)
        ctx.save_for_backward(Yc, optE)
        ctx.cfg = (tau, Tp, exclusion_radius)
        return rho_t.t()

    @staticmethod
    def backward(ctx, g):
        Y, optE = ctx.saved_tensors
        tau, Tp, excl = ctx.cfg
        grad = edm_ccm_rho_backward(Y, optE, g.t().contiguous(), tau=tau, Tp=Tp, exclusion_radius=excl)
        return grad, None, None, None, None, None


def ccm_rho_autograd(Y: torch.Tensor, optE: torch.Tensor, tau: int = 1, Tp: int = 1, exclusion_radius: int = 0,
                     precision: int = EDM_PRECISION_FP32) -> torch.Tensor:
    """Library-major rho [N][N] with autograd support (backward through the
    hand-written adjoint kernels)."""
    return CCMRhoFunction.apply(Y, optE, tau, Tp, exclusion_radius, precision)


def ccm(Y: torch.Tensor, E_max: int = 20, tau: int = 1, Tp: int = 1, exclusion_radius: int = 0,
        precision: int = EDM_PRECISION_FP32):
    """Both phases: (optE, rho) with rho the library-major N x N view."""
    optE, _ = edm_optimal_E(Y, E_max=E_max, tau=tau, Tp=Tp, return_rho=False)
    rho_t = edm_ccm_rho(Y, optE, tau=tau, Tp=Tp, exclusion_radius=exclusion_radius, precision=precision)
    return optE, rho_t.t()
