"""Plant plausible mistakes in a copy of the oracle and check that the pins
in ``test_oracle_pins`` catch every one of them.

Each mutant is a textual edit of ``oracle/dd_oracle.c`` compiled into a
temporary library; the pins then run against it.  Mutants are chosen to stay
memory-safe (no out-of-range reads), so a caught mistake shows up as a
failed assertion or an oracle error status.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "dd_oracle.c")

MUTANTS = {
    "delay sign flipped": ("1.0 / (f_c * f_c) - 1.0 / (f_top * f_top)",
                           "1.0 / (f_top * f_top) - 1.0 / (f_c * f_c)"),
    "inverse square dropped": ("1.0 / (f_c * f_c) - 1.0 / (f_top * f_top)",
                               "1.0 / f_c - 1.0 / f_top"),
    "channels ascend from the top": ("double f_c = f_top - (double)c * df;",
                                     "double f_c = f_top + (double)c * df;"),
    "channel index off by one": ("double f_c = f_top - (double)c * df;",
                                 "double f_c = f_top - (double)(c + 1) * df;"),
    "floor instead of round": ("double x = round(dm[d] * dT);", "double x = floor(dm[d] * dT);"),
    "sampling time multiplied": ("/ (f_top * f_top)) / t_samp;", "/ (f_top * f_top)) * t_samp * 1e8;"),
    "constant in ms units": ("ORACLE_KDM = 4.148808e3;", "ORACLE_KDM = 4.148808e6;"),
    "delay table transposed in the sum": (
        "const uint8_t *row = (const uint8_t *)block + (int64_t)c * pitch +\n"
        "                               delays[(int64_t)c * ndm + d];",
        "const uint8_t *row = (const uint8_t *)block + (int64_t)c * pitch +\n"
        "                               delays[((int64_t)d * nchan + c) % ((int64_t)nchan * ndm)];"),
    "last channel dropped": ("for (int32_t c = 0; c < nchan; ++c) {\n"
                             "          const uint8_t",
                             "for (int32_t c = 0; c < nchan - 1; ++c) {\n"
                             "          const uint8_t"),
    "half exponent bias off": ("e - 25", "e - 24"),
    "sample std (N-1) for real rows": ("sigma[d] = sqrt(q / (double)n);",
                                       "sigma[d] = sqrt(q / (double)(n - 1));"),
    "finaliser divides by N-1": ("sigma[d] = sqrt((double)(unsigned __int128)num) / dn;",
                                 "sigma[d] = sqrt((double)(unsigned __int128)num) / (dn - 1);"),
    "mean from first sample only": ("mean[d] = (double)(int64_t)s1 / dn;",
                                    "mean[d] = (double)row[0];"),
    "threshold not strict": ("if (snr > thr) {", "if (snr >= thr) {"),
    "snr without the mean": ("double snr = (v - mean[d]) / sigma[d];",
                             "double snr = v / sigma[d];"),
}


def _all_pins():
    calls = []
    for g in pins.GEOMS[:2]:
        calls.append(lambda g=g: pins.test_delay_table_matches_exact_rational_evaluation(g))
    calls += [pins.test_delay_table_invariants, pins.test_delay_table_known_maxshift_values,
              pins.test_adjacent_channel_delay_matches_channel_smear_formula,
              pins.test_dm_max_closed_form_gives_one_sample_smear]
    for dt in ("u8", "f16", "f32"):
        for seed in (0, 1, 2):
            calls.append(lambda dt=dt, seed=seed:
                         pins.test_dedisperse_matches_numpy_gather_on_tiny_random_blocks(dt, seed))
    calls += [pins.test_dm_zero_row_is_plain_channel_sum, pins.test_linearity,
              pins.test_impulse_response_pins_direction_and_indexing,
              pins.test_injected_on_grid_pulse_adds_amp_times_nchan_and_peaks_at_truth,
              pins.test_int_stats_match_numpy_and_exact_finaliser,
              pins.test_float_stats_match_numpy]
    for kind in ("int", "float"):
        calls.append(lambda kind=kind: pins.test_detect_matches_numpy_mask_in_dm_time_order(kind))
    calls += [pins.test_detect_threshold_is_strict_and_capacity_truncates_in_order]
    return calls


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor missing: " + name
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared",
                    "-fPIC", str(mutated), "-o", str(lib), "-lm"], check=True)
    oracle._use_library(str(lib))
    try:
        caught = None
        for pin in _all_pins():
            try:
                pin()
            except (AssertionError, RuntimeError) as e:  # the pin noticed
                caught = e
                break
        assert caught is not None, "no pin caught: " + name
    finally:
        oracle._use_library(None)
