"""Pins of the subband oracle (``oracle/approx.py``) and of the analytic S/N
loss curve it is checked with.

* The thesis's incorrect-dedispersion curve (Sec. 3.6) against the brute-force
  oracle on a Gaussian pulse dispersed with exact (unrounded) delays: a pin
  of the curve's transcription and of the brute-force sum at once.
* Subband dedispersion (Sec. 2.1.3) equals the brute-force sum exactly at the
  nominal trials, for one channel per subband and for one trial per group.
* Away from the nominal trials its peak loss follows the same curve applied
  to each subband (bandwidth of the subband, DM error = trial - nominal).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import approx
import synth

K_DM = 4.148808e3  # MHz^2 pc^-1 cm^3 s (Sec. 1.2.1)


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def gaussian_pulse_block(nchan, f_top, df, t_samp, dm, fwhm_ms, nsamp, t0_s):
    """Unit-height Gaussian pulse dispersed with the exact cold-plasma delay."""
    t = np.arange(nsamp) * t_samp
    f = f_top - np.arange(nchan) * df
    tau = K_DM * dm * (f ** -2 - f_top ** -2)
    sig = fwhm_ms * 1e-3 / (2 * math.sqrt(2 * math.log(2)))
    return np.exp(-0.5 * ((t[None, :] - t0_s - tau[:, None]) / sig) ** 2).astype(np.float32)


BAND = dict(nchan=256, f_top=416.0, bw=16.0, t_samp=51.2e-6)


def test_curve_limits():
    assert approx.smearing_peak_ratio(0.0, 16, 0.4, 1.0) == 1.0
    # small zeta: 1 - zeta^2 / 3; large zeta: sqrt(pi) / (2 zeta)
    z = 1e-3
    ddm = z * 1.0 * 0.4 ** 3 / (6.91e-3 * 16)
    assert approx.smearing_peak_ratio(ddm, 16, 0.4, 1.0) == pytest.approx(1 - z * z / 3, rel=1e-9)
    ddm = 50 * 1.0 * 0.4 ** 3 / (6.91e-3 * 16)
    assert approx.smearing_peak_ratio(ddm, 16, 0.4, 1.0) == pytest.approx(
        math.sqrt(math.pi) / 100, rel=1e-9)


@pytest.mark.parametrize("ddm,width_ms", [(0.5, 5.0), (1.0, 5.0), (3.0, 5.0), (5.0, 5.0),
                                          (1.0, 2.0), (2.0, 2.0)])
def test_brute_force_smearing_matches_analytic_curve(ddm, width_ms):
    b = BAND
    df = b["bw"] / b["nchan"]
    dm = 50.0
    blk = gaussian_pulse_block(b["nchan"], b["f_top"], df, b["t_samp"], dm, width_ms, 6000, 0.05)
    delays, _ = oracle.delay_table(b["nchan"], b["f_top"], df, b["t_samp"],
                                   np.array([dm, dm + ddm]))
    D = oracle.dedisperse(blk, delays)
    measured = D[1].max() / D[0].max()
    f_centre = (b["f_top"] - b["bw"] / 2 + df / 2) / 1000
    predicted = approx.smearing_peak_ratio(ddm, b["bw"], f_centre, width_ms)
    assert measured == pytest.approx(predicted, abs=0.01)


def geometry(nchan=256, ndm=96, step=0.5):
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = 16.0 / nchan
    wl.dms = synth.dm_grid(0.0, step, ndm)
    return wl


def test_subband_exact_at_nominal_trials_and_degenerate_sizes():
    wl = geometry()
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                    wl.dms)
    rng = np.random.default_rng(4)
    block = synth.random_block(rng, wl.nchan, mx + 3000, "u8")
    brute = oracle.dedisperse(block, delays)
    for cps, dpg in ((32, 16), (16, 7), (64, 32)):
        tb = approx.SubbandTables(delays, cps, dpg)
        out = approx.subband_dedisperse(block, delays, cps, dpg)
        # the step delays reach at most the nominal trials' span, so the
        # output may run a little longer than the brute-force one
        assert out.shape[1] == block.shape[1] - tb.maxshift
        n = min(out.shape[1], brute.shape[1])
        assert np.array_equal(out[tb.nominal, :n], brute[tb.nominal, :n])
        assert not np.array_equal(out[:, :n], brute[:, :n])  # other trials are approximate
    for cps, dpg in ((1, 16), (32, 1)):
        out = approx.subband_dedisperse(block, delays, cps, dpg)
        n = min(out.shape[1], brute.shape[1])
        assert np.array_equal(out[:, :n], brute[:, :n])


def test_subband_tables():
    wl = geometry(nchan=100, ndm=50)
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                   wl.dms)
    tb = approx.SubbandTables(delays, 32, 16)
    assert tb.first == [0, 32, 64, 96] and [t.shape[0] for t in tb.d1] == [32, 32, 32, 4]
    assert tb.groups == [(0, 16), (16, 32), (32, 48), (48, 50)]
    assert tb.nominal == [7, 23, 39, 48]
    for s, c0 in enumerate(tb.first):
        assert np.all(tb.d1[s][0] == 0) and np.all(np.diff(tb.d1[s], axis=0) >= 0)
    assert np.array_equal(tb.d2[1], delays[tb.first][:, 16:32])


@pytest.mark.parametrize("offset", [-6, -3, 3, 6])
def test_subband_loss_follows_analytic_curve_per_subband(offset):
    """A pulse at trial nominal + offset: the subband sum spreads each
    subband by the DM error (offset trials) over the subband's bandwidth."""
    b = BAND
    nchan, cps, dpg, width = b["nchan"], 32, 16, 0.5
    df = b["bw"] / nchan
    dms = synth.dm_grid(40.0, 0.5, 48)
    tb_probe = approx.SubbandTables(np.zeros((nchan, 48), dtype=np.int32), cps, dpg)
    nominal = tb_probe.nominal[1]
    d = nominal + offset
    blk = gaussian_pulse_block(nchan, b["f_top"], df, b["t_samp"], dms[d], width, 9000, 0.08)
    delays, _ = oracle.delay_table(nchan, b["f_top"], df, b["t_samp"], dms)
    brute = oracle.dedisperse(blk, delays)
    sub = approx.subband_dedisperse(blk, delays, cps, dpg)
    measured = sub[d].max() / brute[d].max()
    ddm = dms[d] - dms[nominal]
    f_centres = [(b["f_top"] - (c0 + cps / 2 - 0.5) * df) / 1000 for c0 in tb_probe.first]
    predicted = np.mean([approx.smearing_peak_ratio(ddm, cps * df, f, width) for f in f_centres])
    assert predicted < 0.97  # a visible loss
    assert measured == pytest.approx(predicted, abs=0.03)


# ---------------------------------------------------------------- time binning

def test_diagonal_dm_is_one_sample_per_channel_at_the_band_bottom():
    for name in ("full_block_u8", "lband_f32", "single_beam_f32"):
        wl = synth.workload(name)
        dd = approx.diagonal_dm(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s)
        for m in (1, 2, 4):
            delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                           wl.t_samp_s, np.array([m * dd]))
            step = int(delays[-1, 0] - delays[-2, 0])
            assert abs(step - m) <= 1, (name, m, step)


def test_binning_factors_follow_the_doubling_ranges():
    f = approx.binning_factors(np.array([0, 10, 19.9, 20, 39.9, 40, 79, 80, 1000.0]), 10.0, 8)
    assert f.tolist() == [1, 1, 1, 2, 2, 4, 4, 8, 8]


def test_decimate_sums_adjacent_samples():
    rng = np.random.default_rng(8)
    b = rng.integers(0, 256, size=(3, 1000), dtype=np.uint8)
    for f in (1, 2, 4, 16):
        d = approx.decimate(b, 1000, f)
        n = 1000 // f
        assert np.array_equal(d, b[:, :n * f].astype(np.int64).reshape(3, n, f).sum(axis=2))
    x = rng.standard_normal((2, 999)).astype(np.float32)
    d = approx.decimate(x, 999, 4)
    ref = x[:, :996].astype(np.float64).reshape(2, 249, 4).sum(axis=2)
    assert d.dtype == np.float32 and np.allclose(d, ref, rtol=0, atol=1e-5)


def test_decimate_mean8_rounds_half_up_within_half_a_count_per_level():
    """8-bit binning against the exact mean of each f-sample block (numpy
    reshape-sum / f): every halving rounds a half-integer up, so the result
    never falls below the exact mean and exceeds it by at most half a count
    per level; one level gives exactly 0 or 1/2; a constant stays put."""
    rng = np.random.default_rng(12)
    b = rng.integers(0, 256, size=(3, 4096), dtype=np.uint8)
    b[0, :64] = 255  # the top of the range stays in 8 bits
    for f in (1, 2, 4, 8, 16):
        d = approx.decimate_mean8(b, 4096, f)
        assert d.dtype == np.uint8 and d.shape == (3, 4096 // f)
        exact = b.astype(np.float64).reshape(3, 4096 // f, f).sum(axis=2) / f
        dev = d.astype(np.float64) - exact
        levels = f.bit_length() - 1
        assert dev.min() >= 0 and dev.max() <= levels / 2, (f, dev.min(), dev.max())
        if f == 2:
            assert set(np.unique(dev).tolist()) == {0.0, 0.5}
    assert np.all(d[0, :64 // 16] == 255)
    c = np.full((2, 1000), 77, dtype=np.uint8)
    assert np.all(approx.decimate_mean8(c, 1000, 8) == 77)
    with pytest.raises(ValueError):
        approx.decimate_mean8(np.zeros((1, 8), dtype=np.float32), 8, 2)


def test_mean8_binned_rows_keep_the_pulse_snr_of_summed_binning():
    """Noise of 16 counts rms plus a dispersed pulse: the 8-bit binned rows
    are the summed rows divided by f up to the rounding (at most half a count
    per level and channel), so each row's peak S/N agrees with the summed
    rows' within 1%, at the summed rows' peak sample; the full-rate rows are
    identical."""
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=128, ndm=160)
    wl.dms = synth.dm_grid(0.0, 1.0, 160)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                    wl.dms)
    nsamp = (2 * mx + 8192) // 64 * 64
    rng = np.random.default_rng(4)
    z = 128 + 16 * rng.standard_normal((wl.nchan, nsamp))
    for d in (10, 70, 120, 159):
        for c in range(wl.nchan):
            z[c, mx + 2000 * (d % 4) + 500 + delays[c, d]:][:16] += 24
    block = np.clip(np.rint(z), 0, 255).astype(np.uint8)
    args = (block, wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, 8)
    rs, fac, ls = approx.binned_dedisperse(*args)
    r8, fac8, l8 = approx.binned_dedisperse(*args, mode="mean8")
    assert np.array_equal(fac, fac8) and np.array_equal(ls, l8)
    assert set(fac.tolist()) == {1, 2, 4, 8}
    for d in range(wl.ndm):
        if fac[d] == 1:
            assert np.array_equal(rs[d], r8[d])
            continue
        dev = r8[d].astype(np.float64) - rs[d] / fac[d]
        levels = int(fac[d]).bit_length() - 1
        assert dev.min() >= 0 and dev.max() <= wl.nchan * levels / 2, d
    for d in (10, 70, 120, 159):
        snr_s = (rs[d] - rs[d].mean()) / rs[d].std()
        snr_8 = (r8[d] - r8[d].mean()) / r8[d].std()
        t = int(np.argmax(snr_s))
        assert snr_s[t] > 8, (d, snr_s[t])
        assert abs(snr_8[t] / snr_s[t] - 1) < 0.01, (d, fac[d], snr_s[t], snr_8[t])
    with pytest.raises(ValueError):
        approx.binned_dedisperse(block.astype(np.float32), *args[1:], mode="mean8")


def test_binned_rows_full_rate_exact_and_flux_conserved():
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=128, ndm=160)
    wl.dms = synth.dm_grid(0.0, 1.0, 160)
    dd = approx.diagonal_dm(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                    wl.dms)
    nsamp = (2 * mx + 4096) // 64 * 64
    rng = np.random.default_rng(3)
    block = np.zeros((wl.nchan, nsamp), dtype=np.uint8)
    block[:, mx + 64:nsamp - mx - 64] = rng.integers(0, 256, size=(wl.nchan, nsamp - 2 * mx - 128))
    rows, fac, lens = approx.binned_dedisperse(block, wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                               wl.t_samp_s, wl.dms, 8)
    assert set(fac.tolist()) == {1, 2, 4, 8} and dd * 2 <= wl.dms[-1]
    brute = oracle.dedisperse(block, delays)
    for d in range(wl.ndm):
        if fac[d] == 1:  # the full-rate trials' own maxshift: rows may run longer
            n = min(lens[d], brute.shape[1])
            assert np.array_equal(rows[d][:n], brute[d, :n])
        # every sample of the signal is added exactly once at any rate
        assert int(rows[d].astype(np.int64).sum()) == int(brute[d].astype(np.int64).sum()), d
        assert lens[d] >= nsamp // fac[d] - (mx // fac[d] + 1)


def test_binned_rows_gather_a_dispersed_pulse():
    """A 16-sample pulse on trial d's track: at any rate the row's peak
    collects most of it (f samples per bin), which a wrong delay scale (f)
    or a misaligned bin would spread over many bins."""
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=128, ndm=160)
    wl.dms = synth.dm_grid(0.0, 1.0, 160)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                    wl.dms)
    nsamp = (2 * mx + 4096) // 64 * 64
    for d in (10, 70, 120, 159):
        block = np.zeros((wl.nchan, nsamp), dtype=np.uint8)
        for c in range(wl.nchan):  # amplitude 3 on the track (uint8 block)
            block[c, mx + 500 + delays[c, d]:mx + 516 + delays[c, d]] = 3
        rows, fac, _ = approx.binned_dedisperse(block, wl.nchan, wl.f_top_mhz,
                                                wl.chan_width_mhz, wl.t_samp_s, wl.dms, 8)
        total = int(block.astype(np.int64).sum())  # the pulse: 16 samples x nchan x 3
        assert total == 16 * wl.nchan * 3
        peak = int(rows[d].max())
        assert peak >= 0.75 * wl.nchan * 3 * min(fac[d], 16), (d, fac[d], peak)
