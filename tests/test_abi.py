"""The C-ABI library builds, loads and exports every symbol of include/edm.h;
argument checks and size queries work without a GPU (no compute calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "edm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(edm_[a-zA-Z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_11082_gb300 import _abi

    return _abi.load()


def test_header_declares_the_path():
    names = declared_functions()
    for required in ("edm_optimal_E", "edm_knn_table", "edm_ccm_rho", "edm_ccm_workspace_bytes",
                     "edm_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2011_11082_gb300 import _abi

    raw = ctypes.CDLL(_abi.lib_path())
    for name in declared_functions():
        assert hasattr(raw, name), name
        assert name in _abi.SIGNATURES, f"binding lacks {name}"


def test_status_strings_and_version(lib):
    assert lib.edm_status_string(0) == b"EDM_OK"
    assert b"INVALID" in lib.edm_status_string(1)
    assert lib.edm_version() >= 0x000100


def test_argument_checks_need_no_gpu(lib):
    from paper_2011_11082_gb300 import make_params

    p = make_params(E_max=10)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: checks fail first
    # null pointers
    assert lib.edm_optimal_E(None, 4, 100, 100, ctypes.byref(p), None, None, None) == 1
    # T too short for E_max
    assert lib.edm_optimal_E(fake, 4, 30, 30, ctypes.byref(p), fake, None, None) == 1
    # E_max beyond the build limit
    p2 = make_params(E_max=21)
    assert lib.edm_optimal_E(fake, 4, 1000, 1000, ctypes.byref(p2), fake, None, None) == 5
    # bad tau / Tp / exclusion radius
    for bad in (make_params(tau=0), make_params(Tp=-1), make_params(exclusion_radius=-2)):
        assert lib.edm_optimal_E(fake, 4, 1000, 1000, ctypes.byref(bad), fake, None, None) == 1
    # knn: Tq inconsistent with T, E
    assert lib.edm_knn_table(fake, 2, 100, 100, 3, ctypes.byref(p), fake, fake, 50, None) == 1
    # ccm: library range outside [0, N), ld_rho too small, workspace too small
    ws_need = lib.edm_ccm_workspace_bytes(64, 500, ctypes.byref(p))
    assert ws_need > 0
    assert lib.edm_ccm_rho(fake, 64, 500, 500, fake, 60, 10, ctypes.byref(p), fake, 64, fake, ws_need, None) == 1
    assert lib.edm_ccm_rho(fake, 64, 500, 500, fake, 0, 64, ctypes.byref(p), fake, 32, fake, ws_need, None) == 1
    assert lib.edm_ccm_rho(fake, 64, 500, 500, fake, 0, 64, ctypes.byref(p), fake, 64, fake, ws_need - 1, None) == 3


def test_workspace_grows_with_problem(lib):
    from paper_2011_11082_gb300 import make_params

    p = make_params()
    a = lib.edm_ccm_workspace_bytes(1000, 1500, ctypes.byref(p))
    b = lib.edm_ccm_workspace_bytes(100000, 1500, ctypes.byref(p))
    assert b > a > 1000 * 1500 * 4


def test_batched_argument_checks_need_no_gpu(lib):
    from paper_2011_11082_gb300 import make_params
    from paper_2011_11082_gb300._abi import edm_dataset

    p = make_params(E_max=10)
    fake = 0x1000  # never dereferenced: checks fail first
    sets = (edm_dataset * 2)(edm_dataset(fake, 64, 500, 500, fake, fake, 64),
                             edm_dataset(fake, 300, 1200, 1216, fake, fake, 300))
    need = lib.edm_ccm_rho_batched_workspace_bytes(sets, 2, ctypes.byref(p))
    assert need > 0
    # the batch needs at least the larger dataset's own tile and table space
    assert need > lib.edm_ccm_rho_batched_workspace_bytes(sets, 1, ctypes.byref(p))
    assert lib.edm_ccm_rho_batched(sets, 2, ctypes.byref(p), fake, need - 1, None) == 3
    assert lib.edm_ccm_rho_batched(sets, 0, ctypes.byref(p), fake, need, None) == 1
    assert lib.edm_ccm_rho_batched(sets, 2, ctypes.byref(p), None, need, None) == 1
    bad = (edm_dataset * 1)(edm_dataset(fake, 64, 30, 30, fake, fake, 64))  # T too short for E_max
    assert lib.edm_ccm_rho_batched_workspace_bytes(bad, 1, ctypes.byref(p)) == 0
    assert lib.edm_ccm_rho_batched(bad, 1, ctypes.byref(p), fake, 1 << 30, None) == 1
    narrow = (edm_dataset * 1)(edm_dataset(fake, 64, 500, 500, fake, fake, 63))  # ld_rho < N
    assert lib.edm_ccm_rho_batched(narrow, 1, ctypes.byref(p), fake, 1 << 30, None) == 1
    big = (edm_dataset * 1)(edm_dataset(fake, 70000, 500, 500, fake, fake, 70000))  # N beyond 16-bit grid
    assert lib.edm_ccm_rho_batched(big, 1, ctypes.byref(p), fake, 1 << 40, None) == 5


def test_long_series_limits_and_workspace_need_no_gpu(lib):
    """Series beyond the shared-memory tile (about 3,100 steps) are accepted
    by the cross map (tiles read from L2) up to the kNN staging limit (about
    46,000 steps); the table area of the workspace shrinks with T."""
    from paper_2011_11082_gb300 import make_params
    from paper_2011_11082_gb300._abi import edm_dataset

    p = make_params()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: checks fail first
    # N = 1,000, T = 40,000: tiles (52 x 40,000 x 128 B) + tables of at
    # least 16 libraries (all E) -- well under the 14 GB a fixed 256-library
    # floor would take
    ws = lib.edm_ccm_workspace_bytes(1000, 40000, ctypes.byref(p))
    assert 52 * 40000 * 128 < ws < 2 * 1024**3
    assert lib.edm_ccm_rho(fake, 1000, 40000, 40000, fake, 0, 1000, ctypes.byref(p), fake, 1000, fake, ws - 1,
                           None) == 3
    # beyond the kNN staging limit: unsupported, for every entry point
    for T in (50000, 60000):
        assert lib.edm_knn_table(fake, 1, T, T, 2, ctypes.byref(p), fake, fake, T - 2, None) == 5
        assert lib.edm_optimal_E(fake, 1, T, T, ctypes.byref(p), fake, None, None) == 5
        big = lib.edm_ccm_workspace_bytes(8, T, ctypes.byref(p))
        assert lib.edm_ccm_rho(fake, 8, T, T, fake, 0, 8, ctypes.byref(p), fake, 8, fake, big, None) == 5
    # the batched form keeps its tiles in shared memory: about 3,100 steps at most
    long_set = (edm_dataset * 1)(edm_dataset(0x1000, 64, 5000, 5000, 0x1000, 0x1000, 64))
    assert lib.edm_ccm_rho_batched(long_set, 1, ctypes.byref(p), fake, 1 << 40, None) == 5


def test_backward_workspace_holds_every_library_up_to_1gb(lib):
    """The adjoint's table budget: the tables of all N libraries while they fit
    in 1 GB (one block: the library pass then runs one CTA per library over
    all of them), else 1 GB of tables; the rest (N^2 pair statistics, plans)
    grows with N^2 and N."""
    from paper_2011_11082_gb300 import edm_ccm_backward_workspace_bytes as ws

    for T in (1500, 3000):
        per_lib = ws(2, T) - ws(1, T)  # one library's tables (plus a few aligned bytes)
        assert per_lib > 200 * T  # every E's table: sum_E (E+1) rows of (4 + 2) bytes, ~1.4 KB per step
        # below the cap the tables grow by one library's bytes per library
        n_fit = (1 << 30) // per_lib
        assert abs((ws(n_fit, T) - ws(n_fit // 2, T)) - (n_fit - n_fit // 2) * per_lib) < 0.02 * ws(n_fit, T)
        # above it the tables stay at 1 GB: only the N^2 statistics grow
        big = 4 * n_fit
        extra = ws(2 * big, T) - ws(big, T)
        assert extra < 16 * ((2 * big) ** 2 - big ** 2) + 64 * big + (1 << 20)
        assert ws(big, T) >= (1 << 30) + 16 * big * big
