"""The FP64 oracle against its pins (CPU only)."""

import pytest

import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin()


def test_ccm_tables_equals_per_library_tables():
    """The multi-library table helper returns each library's own table (the
    same routine, one library per thread)."""
    import numpy as np

    import edm_synth as synth
    from oracle import oracle as orc

    Y = synth.coupled_logistic(9, 140, 0.1, 0.05, seed_data=31, seed_noise=32)
    rows = np.array([0, 3, 8, 5])
    for E, tau, Tp, excl in ((1, 1, 1, 0), (3, 2, 0, 2), (4, 1, 2, -1)):
        got = orc.ccm_tables(Y, E, rows=rows, tau=tau, Tp=Tp, excl=excl, nthreads=3)
        for r, i in enumerate(rows):
            idx, _ = orc.ccm_table(Y[i], E, tau=tau, Tp=Tp, excl=excl)
            assert np.array_equal(got[r], idx), (E, i)
