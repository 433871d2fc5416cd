"""Pins for the CPU oracle against facts that do not come from the oracle.

Each group names what fixes the expected value: exact rational arithmetic,
closed forms printed in the thesis, numpy library routines, impulse
responses, injected pulses, and brute force on tiny blocks.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
K = GOLDEN["dispersion_constant_mhz2_s"]["value"]

GEOMS = [
    # name, nchan, f_top, df, t_samp, dms
    ("single_beam", 64, 416.0, 0.25, 100e-6, synth.dm_grid(0, 1.0, 64)),
    ("full_block", 1024, 416.0, 16.0 / 1024, 51.2e-6, synth.dm_grid(0, 0.1, 2048)),
    ("lband", 4096, 1500.0, 300.0 / 4096, 64e-6, synth.dm_grid(0, 0.1, 4096)),
]


def _round_half_away(q: Fraction) -> int:
    return int(math.floor(q + Fraction(1, 2))) if q >= 0 else -int(math.floor(-q + Fraction(1, 2)))


# ----------------------------------------------------------------- delays

@pytest.mark.parametrize("geom", GEOMS[:2], ids=lambda g: g[0])
def test_delay_table_matches_exact_rational_evaluation(geom):
    """Sec. 2.1.1 deltaT equation evaluated in exact rationals (from the same
    double inputs) agrees with the double-precision table except within
    1e-9 of a rounding tie."""
    name, nchan, f_top, df, ts, dms = geom
    tab, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    Kf, ft, dff, tsf = Fraction(K), Fraction(f_top), Fraction(df), Fraction(ts)
    rng = np.random.default_rng(5)
    chans = np.unique(np.concatenate([[0, 1, nchan - 1], rng.integers(0, nchan, 40)]))
    ds = np.unique(np.concatenate([[0, 1, dms.size - 1], rng.integers(0, dms.size, 40)]))
    mismatches = 0
    for c in chans:
        fc = ft - int(c) * dff
        dT = Kf * (1 / (fc * fc) - 1 / (ft * ft)) / tsf
        for d in ds:
            x = Fraction(float(dms[d])) * dT
            exact = _round_half_away(x)
            if exact != tab[c, d]:
                frac = x - math.floor(x)
                assert abs(frac - Fraction(1, 2)) < Fraction(1, 10 ** 9), (c, d, float(x))
                mismatches += 1
    assert mismatches <= 2


def test_delay_table_invariants():
    """Delays are relative to the band top (Sec. 2.1.1): channel 0 and DM 0
    give 0; lower frequencies and larger DMs never give smaller delays."""
    for name, nchan, f_top, df, ts, dms in GEOMS:
        tab, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
        assert tab.shape == (nchan, dms.size)
        assert np.all(tab[0] == 0)
        assert np.all(tab[:, 0] == 0)
        assert np.all(np.diff(tab, axis=0) >= 0)
        assert np.all(np.diff(tab, axis=1) >= 0)
        assert mx == tab.max() == tab[-1, -1]


def test_delay_table_known_maxshift_values():
    """Maximum delays of the three workload geometries, worked out by hand
    from the deltaT equation: K*DM_max*(f_lo^-2 - f_top^-2)/t_samp."""
    expect = {"single_beam": 1212, "full_block": 7813, "lband": 6634}
    for name, nchan, f_top, df, ts, dms in GEOMS:
        _, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
        assert mx == expect[name], name


def test_adjacent_channel_delay_matches_channel_smear_formula():
    """Sec. 2.5: a channel of width dv at v smears a pulse over
    dt = 2 K DM dv / v^3.  The delay step between adjacent channels must be
    that smear (in samples) to within rounding (+-1) and the curvature of
    v^-2 over one channel."""
    factor = GOLDEN["channel_smear_factor"]["value"]
    for name, nchan, f_top, df, ts, dms in GEOMS:
        tab, _ = oracle.delay_table(nchan, f_top, df, ts, dms)
        for c in (1, nchan // 3, nchan // 2, nchan - 1):
            for d in (dms.size // 4, dms.size - 1):
                fmid = f_top - (c - 0.5) * df
                smear = factor * K * dms[d] * df / fmid ** 3 / ts
                step = int(tab[c, d]) - int(tab[c - 1, d])
                curvature = 3 * K * dms[d] * df ** 2 / fmid ** 4 / ts
                assert abs(step - smear) <= 1.0 + curvature, (name, c, d, step, smear)


def test_dm_max_closed_form_gives_one_sample_smear():
    """Sec. 6.3: DM_max = dt f0^3 / (8300 df) keeps the smear within one
    channel to one sample at the band bottom f0; at that DM the delay step
    between the two lowest channels is 1 sample to within rounding."""
    c8300 = GOLDEN["dm_max_one_sample_smear_constant"]["value"]
    for name, nchan, f_top, df, ts, _ in GEOMS:
        f0 = f_top - (nchan - 1) * df
        dm_max = ts * f0 ** 3 / (c8300 * df)
        tab, _ = oracle.delay_table(nchan, f_top, df, ts, np.array([dm_max, 4 * dm_max]))
        step1 = int(tab[-1, 0]) - int(tab[-2, 0])
        step4 = int(tab[-1, 1]) - int(tab[-2, 1])
        assert step1 in (0, 1, 2), (name, step1)
        assert 3 <= step4 <= 5, (name, step4)


def test_delay_table_rejects_bad_geometry():
    with pytest.raises(RuntimeError):
        oracle.delay_table(64, 10.0, 0.25, 1e-4, [1.0])  # band bottom below 0
    with pytest.raises(RuntimeError):
        oracle.delay_table(64, 416.0, 0.25, 1e-4, [-1.0])
    with pytest.raises(RuntimeError):
        oracle.delay_table(64, 416.0, 0.25, 0.0, [1.0])


# ------------------------------------------------------------ dedispersion

def _numpy_gather(block, delays, nsamp_out):
    """Second formulation: fancy-index gather then numpy sum over channels."""
    nchan, ndm = delays.shape
    t = np.arange(nsamp_out)
    idx = delays.T[:, :, None] + t[None, None, :]          # [ndm][nchan][t]
    c = np.arange(nchan)[None, :, None]
    vals = block[c, idx]
    if block.dtype == np.uint8:
        return vals.astype(np.int64).sum(axis=1)
    return vals.astype(np.float64).sum(axis=1)


@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dedisperse_matches_numpy_gather_on_tiny_random_blocks(dtype, seed):
    rng = np.random.default_rng(100 + seed)
    nchan = int(rng.integers(1, 38))
    ndm = int(rng.integers(1, 20))
    nsamp = int(rng.integers(40, 300))
    f_top = float(rng.uniform(300, 1500))
    df = float(rng.uniform(0.01, 0.5)) * 300 / max(nchan, 1) / 10
    ts = float(rng.uniform(20e-6, 200e-6))
    dms = np.sort(rng.uniform(0, 30, ndm))
    delays, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    if mx >= nsamp:
        nsamp = mx + 37
    pitch = nsamp + int(rng.integers(0, 9))
    block = synth.random_block(rng, nchan, nsamp, dtype, pitch)
    nout = nsamp - mx
    got = oracle.dedisperse(block, delays, nsamp_in=nsamp)
    ref = _numpy_gather(block, delays, nout)
    if dtype == "u8":
        assert got.dtype == np.int32
        assert np.array_equal(got, ref)
    else:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1, nchan))


def test_dm_zero_row_is_plain_channel_sum():
    """With DM 0 every delay is 0, so the row is the channel sum (Sec. 2.1.1)."""
    rng = np.random.default_rng(3)
    wl = synth.workload("single_beam_f32")
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    for dtype in ("u8", "f32"):
        block = synth.random_block(rng, wl.nchan, 2000, dtype)
        d = oracle.dedisperse(block, delays[:, :1], nsamp_out=2000 - mx)
        if dtype == "u8":
            assert np.array_equal(d[0], block[:, :2000 - mx].astype(np.int64).sum(axis=0))
        else:
            np.testing.assert_allclose(d[0], block[:, :2000 - mx].astype(np.float64).sum(axis=0),
                                       rtol=1e-13, atol=1e-12)


def test_linearity():
    rng = np.random.default_rng(4)
    wl = synth.workload("single_beam_f32")
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    x = rng.integers(0, 128, size=(64, 3000), dtype=np.uint8)
    y = rng.integers(0, 128, size=(64, 3000), dtype=np.uint8)
    assert np.array_equal(oracle.dedisperse(x + y, delays),
                          oracle.dedisperse(x, delays) + oracle.dedisperse(y, delays))
    # multiples of 2^-10 below 2^6: 2x - 3y is exact in f32 and every sum is
    # exact in double, so linearity holds bit for bit
    xf = (np.round(rng.standard_normal((64, 3000)) * 1024) / 1024).astype(np.float32)
    yf = (np.round(rng.standard_normal((64, 3000)) * 1024) / 1024).astype(np.float32)
    lhs = oracle.dedisperse((2 * xf - 3 * yf).astype(np.float32), delays)
    rhs = 2 * oracle.dedisperse(xf, delays) - 3 * oracle.dedisperse(yf, delays)
    assert np.array_equal(lhs, rhs)


def test_impulse_response_pins_direction_and_indexing():
    """A single unit sample at (c0, s) appears in row d exactly at output
    time t = s - delay(c0, d): the sum reads forward in time along the
    dispersion track (Sec. 2.1.1)."""
    wl = synth.workload("single_beam_f32")
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = 3000
    nout = nsamp - mx
    for c0, s in [(0, 5), (63, 1300), (17, 900), (40, 2999)]:
        block = np.zeros((wl.nchan, nsamp), dtype=np.uint8)
        block[c0, s] = 1
        D = oracle.dedisperse(block, delays)
        for d in range(wl.ndm):
            t = s - int(delays[c0, d])
            expect = np.zeros(nout, dtype=np.int32)
            if 0 <= t < nout:
                expect[t] = 1
            assert np.array_equal(D[d], expect), (c0, s, d)


def test_injected_on_grid_pulse_adds_amp_times_nchan_and_peaks_at_truth():
    """A boxcar pulse placed on the track of DM trial d_p adds exactly
    A*nchan at (d_p, t0 .. t0+w-1); the best S/N sits there."""
    wl = synth.workload("single_beam_f32")
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, pulses = synth.make_block(wl, seed=1, delays=delays)
    (p,) = pulses
    assert p.dm_idx == 30 and p.width == 4
    noise = block.copy()
    for c in range(wl.nchan):
        s = p.t0 + delays[c, p.dm_idx]
        noise[c, s:s + p.width] -= np.float32(p.amp)
    Ds = oracle.dedisperse(block, delays)
    Dn = oracle.dedisperse(noise, delays)
    diff = Ds[p.dm_idx, p.t0:p.t0 + p.width] - Dn[p.dm_idx, p.t0:p.t0 + p.width]
    np.testing.assert_allclose(diff, p.amp * wl.nchan, atol=1e-4)
    mean, sigma = oracle.stats(Ds)
    snr = (Ds - mean[:, None]) / sigma[:, None]
    d_best, t_best = np.unravel_index(np.argmax(snr), snr.shape)
    assert d_best == p.dm_idx
    assert p.t0 <= t_best < p.t0 + p.width
    # amplitude 5 per channel in unit noise over 64 channels: the pulse adds
    # 5*64 = 320 against a noise rms of sqrt(64) = 8 measured on the pulse-free
    # row (the pulse itself inflates the whole-row rms used by the detector)
    assert abs(Ds[p.dm_idx, t_best] - mean[p.dm_idx] - 320) < 5 * 8
    _, sig_n = oracle.stats(Dn)
    assert abs(sig_n[p.dm_idx] / 8 - 1) < 0.05


def test_functional_test_snr_matches_thesis_closed_form():
    """Sec. 2.4 functional test: top-hat height a = 8/sqrt(1024) in N(0,1)
    noise over 1024 channels is recovered at S/N a*sqrt(N_c) = 8 at its DM.
    (t_samp is not printed; 1 ms is used; DM trials around the pulse DM.)"""
    ft = GOLDEN["functional_test"]
    nchan = ft["nchan"]
    f_top = ft["f_centre_mhz"] + ft["bandwidth_mhz"] / 2
    df = ft["bandwidth_mhz"] / nchan
    ts = 1e-3
    dms = ft["pulse_dm"] + ft["dm_step"] * np.arange(-16, 16)
    delays, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    nsamp = mx + 3000
    rng = np.random.default_rng(11)
    block = rng.standard_normal((nchan, nsamp), dtype=np.float32)
    w = 64
    for t0 in (200, 900, 1600, 2300):
        synth.add_pulse(block, delays[:, 16], synth.Pulse(16, t0, w, ft["pulse_height"]))
    D = oracle.dedisperse(block, delays)
    on = np.zeros(D.shape[1], dtype=bool)
    for t0 in (200, 900, 1600, 2300):
        on[t0:t0 + w] = True
    # S/N against the pulse-free noise of the dedispersed row
    mu_off, sd_off = D[16, ~on].mean(), D[16, ~on].std()
    snrs = (D[16, on] - mu_off) / sd_off
    # each in-pulse sample has S/N 8 +- 1 (unit noise); mean over 256 samples
    assert abs(np.mean(snrs) - ft["integrated_snr"]) < 0.5
    # off-pulse noise in a dedispersed row is N(0, nchan)
    assert abs(np.std(D[0, 2400:2900]) / math.sqrt(nchan) - 1) < 0.1


def test_dedispersed_noise_has_sigma_sqrt_nchan():
    rng = np.random.default_rng(8)
    wl = synth.workload("single_beam_f32")
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block = rng.standard_normal((wl.nchan, wl.nsamp), dtype=np.float32)
    mean, sigma = oracle.stats(oracle.dedisperse(block, delays))
    assert np.all(np.abs(mean) < 0.3)
    assert np.all(np.abs(sigma / 8.0 - 1) < 0.05)


def test_dedisperse_rejects_out_of_range_delays():
    block = np.zeros((4, 100), dtype=np.uint8)
    delays = np.array([[0], [10], [20], [30]], dtype=np.int32)
    with pytest.raises(RuntimeError):
        oracle.dedisperse(block, delays, nsamp_out=71)
    assert oracle.dedisperse(block, delays, nsamp_out=70).shape == (1, 70)
    assert oracle.dedisperse(block, delays, nsamp_out=0).shape == (1, 0)


# ---------------------------------------------------------------- stats

def test_int_stats_match_numpy_and_exact_finaliser():
    rng = np.random.default_rng(21)
    D = rng.integers(-(2 ** 31), 2 ** 31 - 1, size=(6, 5000), dtype=np.int64).astype(np.int32)
    D[1] = rng.integers(0, 300000, 5000)
    D[2] = 7                                   # constant row: sigma 0
    D[3, ::2] = 10
    D[3, 1::2] = 16                            # two values equally often: sigma 3
    mean, sigma = oracle.stats(D)
    for d in range(D.shape[0]):
        row = [int(v) for v in D[d]]
        n = len(row)
        s1 = sum(row)
        s2 = sum(v * v for v in row)
        assert mean[d] == s1 / n                        # correctly rounded S1/N
        assert sigma[d] == math.sqrt(float(n * s2 - s1 * s1)) / n
    np.testing.assert_allclose(mean, D.astype(np.float64).mean(axis=1), rtol=1e-12)
    np.testing.assert_allclose(sigma, D.astype(np.float64).std(axis=1), rtol=1e-9)
    assert sigma[2] == 0.0 and mean[2] == 7.0
    assert sigma[3] == 3.0 and mean[3] == 13.0


def test_float_stats_match_numpy():
    rng = np.random.default_rng(22)
    D = rng.standard_normal((5, 7777)) * 40 + 1000
    mean, sigma = oracle.stats(D)
    np.testing.assert_allclose(mean, D.mean(axis=1), rtol=1e-14)
    np.testing.assert_allclose(sigma, D.std(axis=1), rtol=1e-12)


# ----------------------------------------------------------- candidates

@pytest.mark.parametrize("kind", ["int", "float"])
def test_detect_matches_numpy_mask_in_dm_time_order(kind):
    rng = np.random.default_rng(31)
    if kind == "int":
        D = rng.integers(0, 1000, size=(9, 3000)).astype(np.int32)
        D[4] = 5
    else:
        D = rng.standard_normal((9, 3000))
        D[4] = 5.0
    mean, sigma = oracle.stats(D)
    assert sigma[4] == 0.0
    for nsig in (1.5, 2.5, 3.5):
        cands, total = oracle.detect(D, mean, sigma, nsig)
        snr = np.full(D.shape, -np.inf)
        ok = sigma > 0
        snr[ok] = (D[ok].astype(np.float64) - mean[ok, None]) / sigma[ok, None]
        d_idx, t_idx = np.nonzero(snr > nsig)
        assert total == d_idx.size
        assert np.array_equal(cands["dm_idx"], d_idx)
        assert np.array_equal(cands["t"], t_idx)
        assert np.array_equal(cands["value"], D[d_idx, t_idx].astype(np.float32))
        assert np.array_equal(cands["snr"], snr[d_idx, t_idx].astype(np.float32))
        assert not np.any(cands["dm_idx"] == 4)


def test_detect_threshold_is_strict_and_capacity_truncates_in_order():
    D = np.array([[0, 0, 0, 4]], dtype=np.int32)   # mean 1, sigma sqrt(3)
    mean, sigma = oracle.stats(D)
    snr_top = (4 - 1) / math.sqrt(3)
    c, tot = oracle.detect(D, mean, sigma, np.float32(snr_top) - 1e-6)
    assert tot == 1 and c[0]["t"] == 3
    c, tot = oracle.detect(D, mean, sigma, np.float32(2.0))
    assert tot == 0
    # mean 0, sigma 1 exactly: samples at snr == nsigma are not candidates
    D = np.array([[-1, 1, -1, 1]], dtype=np.int32)
    mean, sigma = oracle.stats(D)
    assert mean[0] == 0.0 and sigma[0] == 1.0
    assert oracle.detect(D, mean, sigma, 1.0)[1] == 0
    assert oracle.detect(D, mean, sigma, 0.999)[1] == 2
    rng = np.random.default_rng(2)
    D = rng.integers(0, 100, size=(4, 500)).astype(np.int32)
    mean, sigma = oracle.stats(D)
    full, tot = oracle.detect(D, mean, sigma, 1.0)
    part, tot2 = oracle.detect(D, mean, sigma, 1.0, capacity=17)
    assert tot == tot2 and tot > 17
    assert np.array_equal(part, full[:17])


def test_false_alarm_count_on_dedispersed_noise():
    """Sec. 1.5.1: chance events above S/N_min in Gaussian noise.  The printed
    integral drops the Gaussian's normalisation; the one-sided tail
    Q(x) = erfc(x/sqrt 2)/2 per sample is used.  Expected count
    nDM * nsamp * Q(3)."""
    rng = np.random.default_rng(41)
    wl = synth.workload("single_beam_f32")
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block = rng.standard_normal((wl.nchan, wl.nsamp), dtype=np.float32)
    D = oracle.dedisperse(block, delays)
    mean, sigma = oracle.stats(D)
    _, total = oracle.detect(D, mean, sigma, 3.0, capacity=0)
    expect = D.size * 0.5 * math.erfc(3.0 / math.sqrt(2))
    assert 0.75 * expect < total < 1.25 * expect


def test_realtime_op_rate_accounting_matches_thesis():
    """Sec. 3.9 (for the benchmark of Sec. 3.8.3): 138e9 ops/s is beams x samples/s x channels x DM trials."""
    r = GOLDEN["realtime_op_rate"]
    ops = r["n_beams"] * r["samples_per_s"] * r["nchan"] * r["n_dm"]
    assert abs(ops / r["ops_per_s"] - 1) < 0.01
    assert r["samples_per_s"] == 1 / 51.2e-6


# -------------------------------------------------------- f16 storage error

@pytest.mark.parametrize("name,nsamp,rows", [
    ("single_beam_f32", None, None),
    ("lband_f32", 2048, [0, 1, 2048, 4094, 4095]),
])
def test_f16_storage_error_within_half_precision_bound(name, nsamp, rows):
    """Storing the input in f16 (round to nearest even, unit roundoff 2^-11)
    moves each sum by at most sum_c |f16(I) - I| <= 2^-11 sum_c |I| plus
    2^-25 per channel for values in the subnormal range.  Both sides run
    through the FP64 oracle, so this is the storage error alone, apart from
    any accumulation error of a kernel; its max and 99th percentile (relative
    to sum_c |I|) are printed for the record."""
    wl = synth.workload(name)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    if nsamp is not None:
        wl = synth.scaled(wl, nsamp=mx + nsamp)
    block32, _ = synth.make_block(wl, seed=1, delays=delays)
    block16 = block32.astype(np.float16)
    d = delays if rows is None else delays[:, rows]
    nout = wl.nsamp - mx
    D32 = oracle.dedisperse(block32, d, nsamp_out=nout)
    D16 = oracle.dedisperse(block16, d, nsamp_out=nout)
    # f16 -> f32 widening is exact, so the oracle must read both forms alike
    assert np.array_equal(D16, oracle.dedisperse(block16.astype(np.float32), d, nsamp_out=nout))
    scale = oracle.dedisperse(np.abs(block32), d, nsamp_out=nout)
    cast_err = oracle.dedisperse(np.abs(block16.astype(np.float32) - block32), d, nsamp_out=nout)
    diff = np.abs(D16 - D32)
    assert np.all(diff <= cast_err * (1 + 1e-12))
    assert np.all(cast_err <= 2.0 ** -11 * scale + wl.nchan * 2.0 ** -25)
    rel = diff / scale
    print(f"\n{name} f16 storage: relative error max {rel.max():.3e} "
          f"p99 {np.percentile(rel, 99):.3e}")
    assert rel.max() > 0  # the cast does move the sums
