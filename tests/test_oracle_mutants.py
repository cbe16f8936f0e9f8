"""Plant plausible mistakes in copies of the oracle and check the pins catch each.

Each mutant is the committed ``oracle/edm_oracle.c`` with one textual change
(a dropped term, a wrong sign or index, a swapped operand), compiled with gcc
into a temporary directory.  Every mutant must fail at least one pin; a
mutant that passes all pins would mean the pins leave that part of the
oracle unchecked.  Nothing here touches a GPU.
"""

import os
import subprocess

import pytest

import oracle_pins
from oracle import oracle as orc

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "edm_oracle.c")

MUTANTS = {
    "lookup_drops_Tp_shift": ("p = p + w[r * k + n] * y[idx[r * k + n] + Tp];", "p = p + w[r * k + n] * y[idx[r * k + n]];"),
    "observation_drops_Tp": ("obs[r] = y[L + r + Tp];", "obs[r] = y[L + r];"),
    "weight_sign_flipped": ("u = exp(-dn / d1);", "u = exp(dn / d1);"),
    "weights_not_normalised": ("w[n] = w[n] / sum;", "w[n] = w[n] / (sum + 1.0);"),
    "distance_not_squared": ("double sq = diff * diff;", "double sq = fabs(diff);"),
    "tie_break_reversed": ("(da == db && ia < ib)", "(da == db && ia > ib)"),
    "exclusion_off_by_one": ("same && excl >= 0 && llabs(s - t) <= excl", "same && excl >= 0 && llabs(s - t) < excl"),
    "subset_exclusion_off_by_one": ("        if (excl >= 0 && llabs(s - t) <= excl)\n            continue;\n        double d = embed_dist2(x, t, x, s",
                                    "        if (excl >= 0 && llabs(s - t) < excl)\n            continue;\n        double d = embed_dist2(x, t, x, s"),
    "phase1_split_rounded_up": ("int64_t h = T / 2;", "int64_t h = (T + 1) / 2;"),
    "phase1_future_from_target": ("p = p + w[n] * lib[idx[n] + Tp];", "p = p + w[n] * tgt[idx[n] + Tp];"),
    "pearson_uncentred_b": ("double da = a[i] - ma, db = b[i] - mb;", "double da = a[i] - ma, db = b[i];"),
    "argmax_ties_to_larger_E": ("if (!any || v > bv) {", "if (!any || v >= bv) {"),
    "weights_use_squared_distance": ("double dn = sqrt(d2[n]);", "double dn = d2[n];"),
    "nearest_distance_wrong_row": ("double d1 = sqrt(d2[0]);", "double d1 = sqrt(d2[k - 1]);"),
    "lag_step_ignores_tau": ("xa[ta - (int64_t)m * tau] - xb[tb - (int64_t)m * tau]", "xa[ta - (int64_t)m] - xb[tb - (int64_t)m]"),
    "lags_gather_without_lag": ("p = p + w[q * k + n] * y[idx[q * k + n] + l];", "p = p + w[q * k + n] * y[idx[q * k + n]];"),
    "lags_observation_unshifted": ("obs[q] = y[A + q + l];", "obs[q] = y[A + q];"),
    "lags_window_start_shifted": ("int64_t A = L > -(int64_t)lag_min ? L : -(int64_t)lag_min;",
                                  "int64_t A = 1 + (L > -(int64_t)lag_min ? L : -(int64_t)lag_min);"),
    "subset_mask_inverted": ("if (!((mask[s / 32] >> (s % 32)) & 1u))", "if (((mask[s / 32] >> (s % 32)) & 1u))"),
    "table_query_window_shifted": ("int got = knn_query(x, t, x, t_lo, t_hi, E, tau, 1, excl, k, idx + r * k, d2);",
                                   "int got = knn_query(x, t, x, t_lo, t_hi - 1, E, tau, 1, excl, k, idx + r * k, d2);"),
}


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site for {name} not found exactly once"
    csrc = tmp_path / "mutant.c"
    csrc.write_text(source.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", "-o", str(so), str(csrc), "-lm"],
                   check=True)
    lib = orc.load_library(str(so))
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(lib=lib)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
    assert caught, f"no pin fails for mutant {name}"
