"""The pins must catch plausible mistakes in the oracle.

Each case copies the oracle's C source, plants one mistake by a textual
substitution, compiles the copy into a temporary library and runs the pins
of test_oracle_pins against it: at least one must fail.  Mistakes are only
ever planted in the CPU oracle, never in GPU code.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

PINS = [
    pins.test_norms_and_crosscorr_match_numpy_correlate,
    pins.test_dtx_matches_fft_correlation,
    pins.test_objective_matches_numpy_convolution,
    pins.test_beta_fresh_matches_definition,
    pins.test_greedy_beta_update_matches_fresh_residual,
    pins.test_phase_schedule_border_updates_match_fresh_residual,
    pins.test_closed_form_for_non_overlapping_atoms,
    pins.test_matches_fista_optimum,
    pins.test_matches_exhaustive_lasso,
    pins.test_kkt_at_solution,
    pins.test_segments_partition_and_phases_are_disjoint,
    pins.test_single_segment_equals_greedy_trajectory,
    pins.test_kkt_report_at_zero_and_after_one_coordinate,
    pins.test_one_update_per_sweep_reaches_greedy_optimum,
]

MUTANTS = {
    "beta_update_sign": ("s->beta[(i64)k * s->Tz + t] -= Sk[t - t0 + (L - 1)] * delta;",
                         "s->beta[(i64)k * s->Tz + t] += Sk[t - t0 + (L - 1)] * delta;"),
    "beta_update_lag_reversed": ("-= Sk[t - t0 + (L - 1)] * delta;",
                                 "-= Sk[t0 - t + (L - 1)] * delta;"),
    "own_entry_not_skipped": ("            if (k == k0 && t == t0)\n                continue;\n"
                              "            s->beta",
                              "            s->beta"),
    "window_one_short": ("i64 lo = t0 - (L - 1), hi = t0 + (L - 1);",
                         "i64 lo = t0 - (L - 1), hi = t0 + (L - 2);"),
    "norm_dropped": ("return orc_soft_threshold(s->beta[(i64)k * s->Tz + t], s->lam) / s->n[k];",
                     "return orc_soft_threshold(s->beta[(i64)k * s->Tz + t], s->lam);"),
    "objective_half_dropped": ("return 0.5 * sq + lam * l1;", "return sq + lam * l1;"),
    "crosscorr_lag_reversed": ("int u = tau + lag;", "int u = tau - lag;"),
    "dtx_convolution_not_correlation": (
        "acc += (double)D[((i64)k * P + p) * L + tau] * (double)X[(i64)p * T + t + tau];",
        "acc += (double)D[((i64)k * P + p) * L + tau] * (double)X[(i64)p * T + t + L - 1 - tau];"),
    "threshold_not_shrunk": ("double a = fabs(u) - lam;", "double a = fabs(u) - 0.5 * lam;"),
    "segment_start_truncated": ("return (i64)m * Tz / M;", "return (i64)m * (Tz / M);"),
    "phase_count_one_short": ("i64 c = 1 + (need + wmin - 1) / wmin;",
                              "i64 c = (need + wmin - 1) / wmin;"),
    "argmax_keeps_first_coordinate": ("if (d > best) {", "if (d > best && best < 0.0) {"),
    "schedule_skips_last_segment": ("for (int m = p; m < M && !stop; m += c)",
                                    "for (int m = p; m < M - 1 && !stop; m += c)"),
    "random_never_picks_last_segment": ("% (uint64_t)M);", "% (uint64_t)(M > 1 ? M - 1 : 1));"),
    "kkt_branches_swapped": ("if (z == 0.0) {\n                double e = fabs(b) - lam;",
                             "if (z != 0.0) {\n                double e = fabs(b) - lam;"),
    "kkt_excess_without_abs": ("double e = fabs(b) - lam;", "double e = b - lam;"),
    "l1_without_abs": ("l1 += fabs(Z[i]);", "l1 += Z[i];"),
    "norm_not_squared": ("                s += d * d;", "                s += fabs(d);"),
    "schedule_stops_with_one_update_left": ("if (!stop && in_sweep == 0) {",
                                            "if (!stop && in_sweep <= 1) {"),
    "random_mode_trusts_stale_dz": ("if (local_argmax(&s, 0, Tz, &kk, &tt, &zz) < eps) {",
                                    "if (local_argmax(&s, 0, Tz, &kk, &tt, &zz) < eps || 1) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path, monkeypatch):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "csc_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not found"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                           "-o", so, str(path), "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle.bind(so))
    caught = []
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake {name!r}"
