"""Plant plausible mistakes in a copy of ``oracle/approx.py`` (subband
dedispersion, time binning, the incorrect-dedispersion curve) and check that
the pins in ``test_oracle_approx_pins`` catch every one of them."""
import importlib.util
import os

import pytest

import oracle
from tests import test_oracle_approx_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "approx.py")

MUTANTS = {
    "step-1 delays not relative to the subband": (
        "(T[c0:c1][:, self.nominal] - T[c0][self.nominal])", "(T[c0:c1][:, self.nominal])"),
    "step-2 delays at the nominal trial": (
        "self.d2 = [T[self.first][:, g0:g1].astype(np.int32) for g0, g1 in self.groups]",
        "self.d2 = [np.repeat(T[self.first][:, [g0 + (g1 - g0 - 1) // 2]], g1 - g0, axis=1)"
        ".astype(np.int32) for g0, g1 in self.groups]"),
    "nominal trial is the first of its group": (
        "self.nominal = [g0 + (g1 - g0 - 1) // 2 for g0, g1 in self.groups]",
        "self.nominal = [g0 for g0, g1 in self.groups]"),
    "curve constant off by ten": ("zeta = 6.91e-3 * abs(ddm)", "zeta = 6.91e-2 * abs(ddm)"),
    "curve without the sqrt(pi)/2": ("return math.sqrt(math.pi) / 2 * math.erf(zeta) / zeta",
                                     "return math.erf(zeta) / zeta"),
    "diagonal DM without the factor 2": (
        "/ (2.0 * k_dm * chan_width_mhz)", "/ (k_dm * chan_width_mhz)"),
    "diagonal DM at the band top": ("f_bot = f_top_mhz - (nchan - 1) * chan_width_mhz",
                                    "f_bot = f_top_mhz"),
    "downfactor already from one diagonal DM": (
        "while 2 * k <= max_factor and dm >= 2 * k * dm_diag:",
        "while 2 * k <= max_factor and dm >= k * dm_diag:"),
    "binning averages instead of summing": ("x = x[:, 0:2 * n:2] + x[:, 1:2 * n:2]",
                                            "x = (x[:, 0:2 * n:2] + x[:, 1:2 * n:2]) // 2"),
    "8-bit binning rounds down": ("x = (x[:, 0:2 * n:2] + x[:, 1:2 * n:2] + 1) // 2",
                                  "x = (x[:, 0:2 * n:2] + x[:, 1:2 * n:2]) // 2"),
    "8-bit binning keeps the even samples": (
        "x = (x[:, 0:2 * n:2] + x[:, 1:2 * n:2] + 1) // 2", "x = x[:, 0:2 * n:2]"),
    "8-bit binned rows from the full-rate block": (
        "src = decimate_mean8(block, nsamp_in, f)", "src = block[:, :nsamp_in // f]"),
    "binned delays at the full-rate sampling time": (
        "delay_table(nchan, f_top_mhz, chan_width_mhz, t_samp_s * f, dms[idx])",
        "delay_table(nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms[idx])"),
}


def load_mutant(name, tmp_path):
    old, new = MUTANTS[name] if name else ("", "")
    src = open(SRC).read()
    assert not name or src.count(old) == 1, name
    pkg = tmp_path / "mutpkg"
    pkg.mkdir()
    (pkg / "approx.py").write_text((src.replace(old, new) if name else src).replace("from . import dedisperse",
                                                                "from oracle import dedisperse")
                                   .replace("from . import delay_table",
                                            "from oracle import delay_table"))
    spec = importlib.util.spec_from_file_location("approx_mutant", pkg / "approx.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pin_calls():
    calls = [pins.test_curve_limits, pins.test_subband_tables,
             pins.test_subband_exact_at_nominal_trials_and_degenerate_sizes,
             pins.test_diagonal_dm_is_one_sample_per_channel_at_the_band_bottom,
             pins.test_binning_factors_follow_the_doubling_ranges,
             pins.test_decimate_sums_adjacent_samples,
             pins.test_decimate_mean8_rounds_half_up_within_half_a_count_per_level,
             pins.test_mean8_binned_rows_keep_the_pulse_snr_of_summed_binning,
             pins.test_binned_rows_full_rate_exact_and_flux_conserved,
             pins.test_binned_rows_gather_a_dispersed_pulse]
    calls += [lambda d=d, w=w: pins.test_brute_force_smearing_matches_analytic_curve(d, w)
              for d, w in ((1.0, 5.0), (3.0, 5.0))]
    calls += [lambda o=o: pins.test_subband_loss_follows_analytic_curve_per_subband(o)
              for o in (-6, 3)]
    return calls


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_approx_pins_catch_planted_mistake(name, tmp_path, monkeypatch):
    oracle.build()
    mod = load_mutant(name, tmp_path)
    monkeypatch.setattr(pins, "approx", mod)
    caught = []
    for call in _pin_calls():
        try:
            call()
        except Exception as e:  # an assertion or an error both count
            caught.append(type(e).__name__)
    assert caught, f"no pin caught: {name}"


def test_unmodified_copy_passes_every_pin(tmp_path, monkeypatch):
    """Control: the same loading path without a mutation fails nothing."""
    oracle.build()
    monkeypatch.setattr(pins, "approx", load_mutant(None, tmp_path))
    for call in _pin_calls():
        call()
