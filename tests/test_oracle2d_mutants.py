"""The 2-D oracle's pins must catch plausible mistakes in it.

As for the 1-D oracle: each case copies csc2d_oracle.c, plants one mistake by
a textual substitution, compiles the copy and runs the pins of
test_oracle2d_pins against it; at least one must fail.  Mistakes are planted
only in the CPU oracle.
"""
import os
import subprocess

import pytest

from oracle import csc2d
from tests import test_oracle2d_pins as pins

PINS = [
    pins.test_crosscorr_and_norms_match_scipy,
    pins.test_dtx_matches_scipy_valid_correlation,
    pins.test_objective_matches_scipy_convolution,
    pins.test_beta_fresh_matches_definition,
    pins.test_greedy_beta_update_matches_fresh_residual,
    pins.test_band_schedule_border_updates_match_fresh_residual,
    pins.test_each_update_lowers_E_by_prop_A1,
    pins.test_one_row_image_is_the_1d_problem,
    pins.test_transposed_problem_has_transposed_optimum,
    pins.test_matches_fista_optimum,
    pins.test_matches_exhaustive_lasso,
    pins.test_kkt_at_solution,
    pins.test_bands_partition_and_phases_are_disjoint,
    pins.test_single_band_equals_greedy_trajectory,
]

MUTANTS = {
    "update_sign": ("-=\n                    Sk[(i - i0 + (h - 1)) * W2 + (j - j0 + (w - 1))] * delta;",
                    "+=\n                    Sk[(i - i0 + (h - 1)) * W2 + (j - j0 + (w - 1))] * delta;"),
    "row_lag_reversed": ("Sk[(i - i0 + (h - 1)) * W2", "Sk[(i0 - i + (h - 1)) * W2"),
    "column_lag_reversed": ("(j - j0 + (w - 1))] * delta;", "(j0 - j + (w - 1))] * delta;"),
    "window_row_one_short": ("ihi = i0 + (h - 1),", "ihi = i0 + (h - 2),"),
    "window_column_one_short": ("jhi = j0 + (w - 1);", "jhi = j0 + (w - 2);"),
    "own_entry_not_skipped": ("if (k == k0 && i == i0 && j == j0)\n                    continue;",
                              "if (0)\n                    continue;"),
    "norm_dropped": ("const double zp = sh(s->beta[e], s->lam) / s->n[k];",
                     "const double zp = sh(s->beta[e], s->lam);"),
    "crosscorr_column_lag_flipped": ("const int v2 = v + db;", "const int v2 = v - db;"),
    "dtx_row_flipped": ("R[((i64)p * H + i + u) * W + j + v];",
                        "R[((i64)p * H + i + h - 1 - u) * W + j + v];"),
    "band_start_truncated": ("return (i64)m * Hz / M;", "return (i64)m * (Hz / M);"),
    "phase_count_one_short": ("i64 c = 1 + (need + hmin - 1) / hmin;",
                              "i64 c = (need + hmin - 1) / hmin;"),
    "objective_half_dropped": ("return 0.5 * sq + lam * l1;", "return sq + lam * l1;"),
    "threshold_not_shrunk": ("double a = fabs(u) - lam;", "double a = fabs(u) - 0.5 * lam;"),
    "argmax_keeps_first_coordinate": ("if (d > best) {", "if (d > best && best < 0.0) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path, monkeypatch):
    src = open(os.path.join(os.path.dirname(csc2d.__file__), "csc2d_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not found"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant2d.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                           "-o", so, str(path), "-lm"])
    monkeypatch.setattr(csc2d, "_lib", csc2d.bind(so))
    caught = []
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake {name!r}"
