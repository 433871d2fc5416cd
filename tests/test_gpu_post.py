"""GPU: post-processing (include/dd_post.h) against the oracle (oracle/post.py).

Median filter and boxcar search are compared exactly (a median is one of its
inputs; boxcar sums are exact int64 for int rows and follow the same float
adds in the same order for float rows; every threshold decision is taken in
the same double expression on both sides).  Detrending is compared within the
bound derived from its float output: the GPU forms r = y - a - b t from a
line evaluated in double once per 16 samples and split into an integer part
and a float remainder, then multiplies by 1/s in float, so each output
carries a few float roundings of |y|, |a + b t| and |b| (16 samples) and of
|z| itself.  Int rows fit the line from exact sums; float rows sum 16-sample
chunks pairwise in float (4 roundings of the chunk's magnitude), and the
intercept's sensitivity to the two sums is at most 7 times the row's mean
magnitude, so a and b t carry at most 28 float roundings of max|y|.  With
u = 2^-24:
    |z_gpu - z| <= 64 u (|z| + (max|y| + |a| + |b| n + 1) / s).
A series whose least-squares residual is at the rounding level (two float
samples, say) has no stable normalisation and is only tested for int rows,
where the residual is decided exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import post
import paper_1401_8258_gb300 as dd
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rows_of(seed, nrows, ncols, dtype, pitch=None, **kw):
    rng = np.random.default_rng(seed)
    full = synth.series_rows(rng, nrows, ncols, dtype, pitch=pitch, **kw)
    return full, full[:, :ncols]


# ------------------------------------------------------------------ median

@pytest.mark.parametrize("dtype", ["i32", "f32"])
@pytest.mark.parametrize("ncols", [1, 2, 7, 4095, 4096, 4097, 10001])
def test_median_matches_oracle_exactly(dtype, ncols):
    full, x = rows_of(ncols, 5, ncols, dtype, pitch=ncols + 3, level=50, noise=20, pulses=3,
                      pulse_amp=8)
    d_in = dev(full)
    for width in (1, 3, 5, 7, 9, 15):
        out = torch.full((5, ncols + 1), -7, dtype=d_in.dtype, device=DEV)  # odd pitch
        dd._native.dd_median_filter(d_in, full.shape[1], 0 if dtype == "i32" else 1, 5, ncols,
                                    width, out, out.shape[1])
        got = out.cpu().numpy()
        assert np.array_equal(got[:, :ncols], post.median_filter(x, width)), width
        assert np.all(got[:, ncols:] == -7)  # nothing written past ncols


def test_median_of_dedispersed_rows_and_wrapper():
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=256, nsamp=9000, ndm=40)
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, 3, delays)
    D = oracle.dedisperse(block, delays)
    for width in (5, 7):
        got = dd.median_filter(dev(D), width).cpu().numpy()
        assert np.array_equal(got, post.median_filter(D, width))


def test_median_argument_errors():
    x = torch.zeros((2, 100), dtype=torch.int32, device=DEV)
    o = torch.zeros_like(x)
    for width in (0, 2, 17):
        with pytest.raises(dd.DDError):
            dd._native.dd_median_filter(x, 100, 0, 2, 100, width, o, 100)
    with pytest.raises(dd.DDError):  # in place is refused
        dd._native.dd_median_filter(x, 100, 0, 2, 100, 5, x, 100)
    with pytest.raises(dd.DDError):
        dd._native.dd_median_filter(x, 100, 7, 2, 100, 5, o, 100)


# ----------------------------------------------------------------- detrend

def check_detrend(x, z_gpu, coef_gpu):
    z, coef = post.detrend(x)
    n = x.shape[1]
    u = 2.0 ** -24
    for r in range(x.shape[0]):
        a, b, s = coef[r]
        if s == 0:
            assert coef_gpu[r, 2] == 0 and not z_gpu[r].any(), r
            continue
        scale = (np.abs(x[r].astype(np.float64)).max() + abs(a) + abs(b) * n + 1) / s
        err = np.abs(z_gpu[r].astype(np.float64) - z[r])
        assert np.all(err <= 64 * u * (np.abs(z[r]) + scale)), (r, err.max(), scale)
        span = s + abs(b) * n
        assert coef_gpu[r, 0] == pytest.approx(a, rel=1e-6, abs=64 * u * span)
        assert coef_gpu[r, 1] == pytest.approx(b, rel=1e-6, abs=64 * u * span / n)
        assert coef_gpu[r, 2] == pytest.approx(s, rel=64 * u * (1 + abs(b) * n / s))


@pytest.mark.parametrize("dtype", ["i32", "f32"])
@pytest.mark.parametrize("ncols,slope", [(1, 0.0), (3, 1.0), (33, 0.3), (4099, 0.02),
                                         (57723, 0.001), (20000, 5.0),
                                         (73729, 0.01)])
def test_detrend_matches_oracle_within_bound(dtype, ncols, slope):
    level = 130000.0 if dtype == "i32" else 3.0
    full, x = rows_of(ncols + 1, 6, ncols, dtype, pitch=ncols + (4 if ncols % 2 else 0),
                      level=level, noise=500.0, slope=slope * 500, pulses=2, pulse_amp=10)
    d_in = dev(full)
    out, coef = dd.detrend(d_in[:, :ncols], coef=True)
    check_detrend(x, out.cpu().numpy(), coef.cpu().numpy())


def test_detrend_exact_line_and_in_place():
    t = np.arange(5000, dtype=np.int64)
    x = np.stack([3 + 2 * t, -7 * t + 11, np.full(5000, 9)]).astype(np.int32)
    out, coef = dd.detrend(dev(x), coef=True)
    assert not out.cpu().numpy().any()
    c = coef.cpu().numpy()
    assert np.array_equal(c[:, 2], np.zeros(3))
    assert np.allclose(c[:, 1], [2, -7, 0]) and np.allclose(c[:, 0], [3, 11, 9])
    two = np.array([[5, 9], [-3, 100]], dtype=np.int32)  # two samples: always a line
    out, coef = dd.detrend(dev(two), coef=True)
    assert not out.cpu().numpy().any() and not coef.cpu().numpy()[:, 2].any()
    # float rows in place (out is the input)
    full, xf = rows_of(9, 4, 7000, "f32", level=2.0, noise=1.0, slope=0.001)
    buf = dev(xf)
    out, coef = dd.detrend(buf, out=buf, coef=True)
    assert out.data_ptr() == buf.data_ptr()
    check_detrend(xf, buf.cpu().numpy(), coef.cpu().numpy())


# ------------------------------------------------------------------ boxcar

def run_boxcar(rows, mean, sigma, nwidths, nsigma, capacity=1 << 18):
    m = None if mean is None else dev(np.asarray(mean, dtype=np.float64))
    s = None if sigma is None else dev(np.asarray(sigma, dtype=np.float64))
    return dd.boxcar_detect(dev(rows), nwidths, nsigma, mean=m, sigma=s, capacity=capacity)


def assert_pulses_equal(got, ref):
    assert got.shape == ref.shape
    for f in ("dm_idx", "t", "width", "snr", "value"):
        assert np.array_equal(got[f], ref[f]), f


@pytest.mark.parametrize("nwidths", [1, 4, 8, 12])
def test_boxcar_int_rows_from_dedispersion_exact(nwidths):
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=256, nsamp=12000, ndm=24)
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, 11, delays)
    D = oracle.dedisperse(block, delays)
    mean, sigma = oracle.stats(D)
    for nsig in (3.0, 5.0):
        got, total = run_boxcar(D, mean, sigma, nwidths, nsig)
        ref = post.boxcar_detect(D, mean, sigma, nwidths, nsig)
        assert total == ref.size
        assert_pulses_equal(got, ref)


@pytest.mark.parametrize("ncols", [1, 3, 100, 4095, 4096, 4097, 9000])
@pytest.mark.parametrize("nwidths", [1, 3, 9, 12])
def test_boxcar_float_rows_exact(ncols, nwidths):
    _, x = rows_of(ncols * 7 + nwidths, 5, ncols, "f32", noise=1.0, pulses=4, pulse_amp=1.5,
                   pulse_width=(1, 300))
    got, total = run_boxcar(x, None, None, nwidths, 3.0)
    ref = post.boxcar_detect(x, None, None, nwidths, 3.0)
    assert total == ref.size
    assert_pulses_equal(got, ref)


def test_boxcar_statistics_rules_and_overflow():
    _, x = rows_of(5, 6, 6000, "i32", level=1000, noise=30, pulses=5, pulse_amp=4)
    mean = np.array([1000.0, 1000.0, 1000.0, np.inf, 1000.0, -np.inf])
    sigma = np.array([30.0, 0.0, np.nan, 30.0, -1.0, 30.0])
    got, total = run_boxcar(x, mean, sigma, 6, 3.5)
    ref = post.boxcar_detect(x, mean, sigma, 6, 3.5)
    assert set(ref["dm_idx"]) == {0}
    assert total == ref.size
    assert_pulses_equal(got, ref)
    # capacity below the total: DD_ERR_OVERFLOW, the first `capacity` written
    mean = np.full(6, 1000.0)
    sigma = np.full(6, 30.0)
    ref = post.boxcar_detect(x, mean, sigma, 6, 2.5)
    cap = ref.size // 3
    got, total = run_boxcar(x, mean, sigma, 6, 2.5, capacity=cap)
    assert total == ref.size and got.size == cap
    assert_pulses_equal(got, ref[:cap])


def test_boxcar_argument_errors():
    x = torch.zeros((2, 100), dtype=torch.float32, device=DEV)
    ws = torch.empty(dd._native.dd_boxcar_workspace_bytes(2, 100), dtype=torch.uint8, device=DEV)
    p = torch.empty((4, 24), dtype=torch.uint8, device=DEV)
    for nw in (0, 13):
        with pytest.raises(dd.DDError):
            dd._native.dd_boxcar_detect(x, 100, 1, 2, 100, None, None, nw, 3.0, ws, ws.numel(), p,
                                        4)
    with pytest.raises(dd.DDError):  # short workspace
        dd._native.dd_boxcar_detect(x, 100, 1, 2, 100, None, None, 3, 3.0, ws, 8, p, 4)
    with pytest.raises(dd.DDError):
        dd._native.dd_boxcar_detect(x, 100, 1, 2, 100, None, None, 3, float("nan"), ws,
                                    ws.numel(), p, 4)


# ------------------------------------------------------------------- chain

def test_post_chain_after_dd_run():
    """dd_run -> median(5) -> detrend -> boxcar, against the oracle chain
    on the same block: the median is exact, detrending within its bound, and
    the boxcar pulses agree wherever the decision is not within float noise
    of the threshold or of a tie between widths."""
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=512, nsamp=20000, ndm=64)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as plan:
        delays = plan.delays()
        block, _ = synth.make_block(wl, 21, delays)
        ref_delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                           wl.t_samp_s, wl.dms)
        assert np.array_equal(delays, ref_delays)
        D_gpu = plan.run(dev(block), 6.0)[0]
    D = oracle.dedisperse(block, ref_delays)
    assert np.array_equal(D_gpu.cpu().numpy(), D)
    m_gpu = dd.median_filter(D_gpu, 5)
    m = post.median_filter(D, 5)
    assert np.array_equal(m_gpu.cpu().numpy(), m)
    z_gpu, coef = dd.detrend(m_gpu, coef=True)
    check_detrend(m, z_gpu.cpu().numpy(), coef.cpu().numpy())
    got, total = dd.boxcar_detect(z_gpu, 8, 4.0, capacity=1 << 18)
    assert got.size == total
    z, _ = post.detrend(m)
    ref = post.boxcar_detect(z.astype(np.float32), None, None, 8, 4.0)
    # robust comparison: per (row, t) the oracle's largest S/N over widths
    sums = post.boxcar_sums(z.astype(np.float32), 8)
    best = np.full(z.shape, -np.inf)
    for j, s in enumerate(sums):
        snr = post.boxcar_snr(s, 1 << j, np.zeros(len(z)), np.ones(len(z)))
        best[:, :snr.shape[1]] = np.maximum(best[:, :snr.shape[1]], snr)
    # the two chains' normalised series differ by float rounding (bounded
    # above); a width-w S/N moves by at most sqrt(w) times that difference
    dz = np.abs(z_gpu.cpu().numpy().astype(np.float64) - z).max()
    near = np.abs(best - 4.0) <= np.sqrt(128) * dz + 1e-6
    g = {(int(a), int(b)) for a, b in zip(got["dm_idx"], got["t"])}
    r = {(int(a), int(b)) for a, b in zip(ref["dm_idx"], ref["t"])}
    for k in g ^ r:
        assert near[k], k
    assert len(g & r) > 0.9 * len(r) and len(r) > 10
