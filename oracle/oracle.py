"""Python face of the FP64 CPU oracle (``edm_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It loads its own
shared library, built from ``edm_oracle.c`` with gcc; it never touches the
CUDA library and the CUDA path never touches it.

All routines take float32 or float64 arrays, promote them to float64 (exact)
and return float64 results.  Parameters follow the paper's notation:
E (embedding dimension), tau (lag), Tp (prediction horizon, 1 = one step
ahead), excl (exclusion radius around a query: -1 none, 0 itself only).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "edm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libedm_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP across library rows / series)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _declare(lib):
    """Attach the C signatures to a loaded oracle library."""
    lib.orc_ccm_rows.restype = _i64
    lib.orc_ccm_rows.argtypes = [_i64, _int, _int, _int]
    lib.orc_knn.restype = _int
    lib.orc_knn.argtypes = [_dp, _i64, _i64, _dp, _i64, _i64, _int, _int, _int, _int, _int, _i64p, _dp]
    lib.orc_weights.restype = None
    lib.orc_weights.argtypes = [_dp, _int, _dp]
    lib.orc_pearson.restype = ctypes.c_double
    lib.orc_pearson.argtypes = [_dp, _dp, _i64]
    lib.orc_simplex_rho.restype = ctypes.c_double
    lib.orc_simplex_rho.argtypes = [_dp, _i64, _int, _int, _int]
    lib.orc_optimal_E.restype = _int
    lib.orc_optimal_E.argtypes = [_dp, _i64, _i64, _i64, _int, _int, _int, _i32p, _dp, _int]
    lib.orc_ccm_table.restype = _int
    lib.orc_ccm_table.argtypes = [_dp, _i64, _int, _int, _int, _int, _i64p, _dp]
    lib.orc_ccm_table_d2.restype = _int
    lib.orc_ccm_table_d2.argtypes = [_dp, _i64, _int, _int, _int, _i64p, _dp]
    lib.orc_lookup_rho.restype = ctypes.c_double
    lib.orc_lookup_rho.argtypes = [_dp, _i64, _int, _int, _int, _i64p, _dp]
    lib.orc_rho_frozen.restype = ctypes.c_double
    lib.orc_rho_frozen.argtypes = [_dp, _dp, _i64, _int, _int, _int, _i64p]
    lib.orc_ccm_rho_rows.restype = _int
    lib.orc_ccm_rho_rows.argtypes = [_dp, _i64, _i64, _i64, _i32p, _i64p, _i64, _i64p, _i64, _int, _int,
                                     _int, _dp, _int]
    lib.orc_ccm_rho_pairs.restype = _int
    lib.orc_ccm_rho_pairs.argtypes = [_dp, _i64, _i64, _i64, _i32p, _i64p, _i64p, _i64, _int, _int, _int,
                                      _dp, _int]
    lib.orc_ccm_rho_lags.restype = _int
    lib.orc_ccm_rho_lags.argtypes = [_dp, _i64, _i64, _i64, _i32p, _i64p, _i64, _int, _int, _int, _int, _dp,
                                     _int]
    lib.orc_ccm_rho_subsets.restype = _int
    lib.orc_ccm_rho_subsets.argtypes = [_dp, _i64, _i64, _i64, _i32p, _i64p, _i64, ctypes.POINTER(ctypes.c_uint32), _i64,
                                        _i64, _int, _int, _int, _dp, _int]
    lib.orc_ccm_tables.restype = _int
    lib.orc_ccm_tables.argtypes = [_dp, _i64, _i64, _i64p, _i64, _int, _int, _int, _int, _i64p, _dp, _int]
    lib.orc_max_threads.restype = _int
    lib.orc_max_threads.argtypes = []
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
        return _lib


def load_library(path: str):
    """Load another build of ``edm_oracle.c`` (e.g. a copy with a planted
    mistake, compiled by a test) and return a handle usable as ``lib=``."""
    return _declare(ctypes.CDLL(path))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a, t):
    return a.ctypes.data_as(t)


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def ccm_rows(T: int, E: int, tau: int = 1, Tp: int = 1, lib=None) -> int:
    return int((lib or _load()).orc_ccm_rows(T, E, tau, Tp))


def knn(xq, t_lo, t_hi, xc, s_lo, s_hi, E, tau=1, same=False, excl=0, k=None, lib=None):
    """k nearest candidates (ascending (d2, s)) for queries t_lo..t_hi."""
    lib = lib or _load()
    k = E + 1 if k is None else k
    xq = _f64(xq)
    xc = xq if same else _f64(xc)
    nq = t_hi - t_lo + 1
    idx = np.zeros((nq, k), np.int64)
    d2 = np.zeros((nq, k), np.float64)
    rc = lib.orc_knn(_ptr(xq, _dp), t_lo, t_hi, _ptr(xc, _dp), s_lo, s_hi, E, tau, int(same), excl, k,
                     _ptr(idx, _i64p), _ptr(d2, _dp))
    if rc:
        raise ValueError(f"orc_knn failed ({rc})")
    return idx, d2


def weights(d2, lib=None) -> np.ndarray:
    d2 = _f64(d2)
    w = np.zeros_like(d2)
    (lib or _load()).orc_weights(_ptr(d2, _dp), d2.size, _ptr(w, _dp))
    return w


def pearson(a, b, lib=None) -> float:
    a, b = _f64(a), _f64(b)
    return float((lib or _load()).orc_pearson(_ptr(a, _dp), _ptr(b, _dp), a.size))


def simplex_rho(x, E, tau=1, Tp=1, lib=None) -> float:
    x = _f64(x)
    return float((lib or _load()).orc_simplex_rho(_ptr(x, _dp), x.size, E, tau, Tp))


def optimal_E(Y, E_max, tau=1, Tp=1, nthreads=None, lib=None):
    """Phase 1 for every row of Y: (optE int32[N], rho_by_E float64[N][E_max])."""
    Y = _f64(np.atleast_2d(Y))
    N, T = Y.shape
    optE = np.zeros(N, np.int32)
    rho = np.zeros((N, E_max), np.float64)
    rc = (lib or _load()).orc_optimal_E(_ptr(Y, _dp), N, T, T, E_max, tau, Tp, _ptr(optE, _i32p), _ptr(rho, _dp),
                               nthreads or default_threads())
    if rc:
        raise ValueError(f"orc_optimal_E failed ({rc})")
    return optE, rho


def ccm_table(x, E, tau=1, Tp=1, excl=0, lib=None):
    """Phase-2 table of one library: (idx int64[nq][E+1] (unshifted s), w float64[nq][E+1])."""
    x = _f64(x)
    nq = ccm_rows(x.size, E, tau, Tp, lib=lib)
    idx = np.zeros((nq, E + 1), np.int64)
    w = np.zeros((nq, E + 1), np.float64)
    rc = (lib or _load()).orc_ccm_table(_ptr(x, _dp), x.size, E, tau, Tp, excl, _ptr(idx, _i64p), _ptr(w, _dp))
    if rc:
        raise ValueError(f"orc_ccm_table failed ({rc})")
    return idx, w


def ccm_tables(Y, E, rows=None, tau=1, Tp=1, excl=0, nthreads=None, lib=None):
    """Neighbour indices of the phase-2 tables of library rows `rows` of Y at
    one E (as ccm_table, libraries spread over threads): int64
    [len(rows)][nq][E+1]."""
    Y = _f64(np.atleast_2d(Y))
    N, T = Y.shape
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nq = ccm_rows(T, E, tau, Tp, lib=lib)
    idx = np.zeros((rows.size, nq, E + 1), np.int64)
    rc = (lib or _load()).orc_ccm_tables(_ptr(Y, _dp), T, T, _ptr(rows, _i64p), rows.size, E, tau, Tp, excl,
                                         _ptr(idx, _i64p), None, nthreads or default_threads())
    if rc:
        raise ValueError(f"orc_ccm_tables failed ({rc})")
    return idx


def ccm_table_d2(x, E, idx, tau=1, Tp=1, lib=None):
    x = _f64(x)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    d2 = np.zeros(idx.shape, np.float64)
    (lib or _load()).orc_ccm_table_d2(_ptr(x, _dp), x.size, E, tau, Tp, _ptr(idx, _i64p), _ptr(d2, _dp))
    return d2


def lookup_rho(y, E, idx, w, tau=1, Tp=1, lib=None) -> float:
    y = _f64(y)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    w = _f64(w)
    return float((lib or _load()).orc_lookup_rho(_ptr(y, _dp), y.size, E, tau, Tp, _ptr(idx, _i64p), _ptr(w, _dp)))


def rho_frozen(x, y, E, idx, tau=1, Tp=1, lib=None) -> float:
    x, y = _f64(x), _f64(y)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    return float((lib or _load()).orc_rho_frozen(_ptr(x, _dp), _ptr(y, _dp), x.size, E, tau, Tp, _ptr(idx, _i64p)))


def ccm_rho_rows(Y, optE, rows=None, cols=None, tau=1, Tp=1, excl=0, nthreads=None, lib=None):
    """rho[r][c] = rho(library rows[r] -> target cols[c]) (library-major)."""
    Y = _f64(np.atleast_2d(Y))
    N, T = Y.shape
    optE = np.ascontiguousarray(optE, dtype=np.int32)
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    if cols is None:
        colp, ncol = None, N
    else:
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        colp, ncol = _ptr(cols, _i64p), cols.size
    rho = np.full((rows.size, ncol), np.nan, np.float64)
    rc = (lib or _load()).orc_ccm_rho_rows(_ptr(Y, _dp), N, T, T, _ptr(optE, _i32p), _ptr(rows, _i64p), rows.size, colp,
                                  ncol, tau, Tp, excl, _ptr(rho, _dp), nthreads or default_threads())
    if rc:
        raise ValueError(f"orc_ccm_rho_rows failed ({rc})")
    return rho


def ccm_rho_pairs(Y, optE, li, lj, tau=1, Tp=1, excl=0, nthreads=None, lib=None):
    Y = _f64(np.atleast_2d(Y))
    N, T = Y.shape
    optE = np.ascontiguousarray(optE, dtype=np.int32)
    li = np.ascontiguousarray(li, dtype=np.int64)
    lj = np.ascontiguousarray(lj, dtype=np.int64)
    rho = np.zeros(li.size, np.float64)
    rc = (lib or _load()).orc_ccm_rho_pairs(_ptr(Y, _dp), N, T, T, _ptr(optE, _i32p), _ptr(li, _i64p), _ptr(lj, _i64p),
                                   li.size, tau, Tp, excl, _ptr(rho, _dp), nthreads or default_threads())
    if rc:
        raise ValueError(f"orc_ccm_rho_pairs failed ({rc})")
    return rho


def ccm_rho_lags(Y, optE, lag_min, lag_max, rows=None, tau=1, excl=0, nthreads=None, lib=None):
    """Time-delay cross mapping: rho[l - lag_min][r][j] = rho_l(library
    rows[r] -> target j), one table per (library, E) over the points every
    lag keeps inside the series."""
    Y = _f64(np.atleast_2d(Y))
    N, T = Y.shape
    optE = np.ascontiguousarray(optE, dtype=np.int32)
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    rho = np.full((lag_max - lag_min + 1, rows.size, N), np.nan, np.float64)
    rc = (lib or _load()).orc_ccm_rho_lags(_ptr(Y, _dp), N, T, T, _ptr(optE, _i32p), _ptr(rows, _i64p), rows.size,
                                           tau, lag_min, lag_max, excl, _ptr(rho, _dp), nthreads or default_threads())
    if rc:
        raise ValueError(f"orc_ccm_rho_lags failed ({rc})")
    return rho


def ccm_rho_subsets(Y, optE, masks, rows=None, tau=1, Tp=1, excl=0, nthreads=None, lib=None):
    """CCM convergence: rho[u][r][j] = rho(library rows[r] -> target j) with
    the library's candidate points restricted to subset u (masks: uint32
    [n_sub][words], bit s = candidate time s allowed)."""
    Y = _f64(np.atleast_2d(Y))
    N, T = Y.shape
    optE = np.ascontiguousarray(optE, dtype=np.int32)
    masks = np.ascontiguousarray(np.atleast_2d(masks), dtype=np.uint32)
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    rho = np.full((masks.shape[0], rows.size, N), np.nan, np.float64)
    rc = (lib or _load()).orc_ccm_rho_subsets(_ptr(Y, _dp), N, T, T, _ptr(optE, _i32p), _ptr(rows, _i64p), rows.size,
                                              _ptr(masks, ctypes.POINTER(ctypes.c_uint32)), masks.shape[0],
                                              masks.shape[1], tau, Tp, excl, _ptr(rho, _dp),
                                              nthreads or default_threads())
    if rc:
        raise ValueError(f"orc_ccm_rho_subsets failed ({rc})")
    return rho


def max_threads(lib=None) -> int:
    return int((lib or _load()).orc_max_threads())
