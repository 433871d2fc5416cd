"""Pins of the post-processing oracle (``oracle/post.py``) to facts that do not
come from the oracle itself: brute force written independently here, library
routines (scipy's median filter, numpy.polyfit), closed forms (a quadratic
residual, the top-hat pulse S/N of Sec. 1.5.1) and the Gaussian tail rate of
chance events.

Each pin is a function of the module under test, so that
``test_oracle_post_mutations`` can run them against mutated copies.
"""
import math

import numpy as np
import pytest

from oracle import post as P0


def rand_rows(rng, nrows, n, dtype):
    if dtype == np.int32:
        return rng.integers(-50, 200, size=(nrows, n)).astype(np.int32)
    return (rng.standard_normal((nrows, n)) * 30 + 5).astype(np.float32)


# ------------------------------------------------------------------ median

def pin_median_brute_force(P):
    rng = np.random.default_rng(1)
    for dtype in (np.int32, np.float32):
        for n in (1, 2, 5, 9, 23):
            x = rand_rows(rng, 3, n, dtype)
            for width in (1, 3, 5, 7, 15):
                h = width // 2
                got = P.median_filter(x, width)
                assert got.dtype == x.dtype
                for r in range(x.shape[0]):
                    for i in range(n):
                        win = [x[r, min(max(i + k, 0), n - 1)] for k in range(-h, h + 1)]
                        assert got[r, i] == sorted(win)[h], (dtype, n, width, r, i)


def pin_median_scipy(P):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    x = rand_rows(rng, 6, 300, np.int32)
    for width in (3, 5, 7, 11):
        ref = ndimage.median_filter(x, size=(1, width), mode="nearest")
        assert np.array_equal(P.median_filter(x, width), ref)


def pin_median_invariants(P):
    rng = np.random.default_rng(3)
    mono = np.sort(rand_rows(rng, 4, 64, np.int32), axis=1)
    const = np.full((2, 40), 7, dtype=np.int32)
    for width in (3, 5, 7):
        assert np.array_equal(P.median_filter(mono, width), mono)  # monotone rows pass through
        assert np.array_equal(P.median_filter(const, width), const)
        # spikes narrower than half the window vanish
        x = np.zeros((1, 50), dtype=np.float32)
        h = width // 2
        x[0, 20:20 + h] = 1000.0
        assert not P.median_filter(x, width).any()


# ----------------------------------------------------------------- detrend

def pin_detrend_polyfit_and_normal_equations(P):
    rng = np.random.default_rng(4)
    n = 1000
    t = np.arange(n, dtype=np.float64)
    for dtype in (np.int32, np.float32):
        x = rand_rows(rng, 3, n, dtype)
        x = (x.astype(np.float64) + (0.37 * t - 11.0)).astype(dtype)
        z, coef = P.detrend(x)
        for r in range(3):
            y = x[r].astype(np.float64)
            b, a = np.polyfit(t, y, 1)
            assert coef[r, 0] == pytest.approx(a, rel=1e-9, abs=1e-9)
            assert coef[r, 1] == pytest.approx(b, rel=1e-9, abs=1e-12)
            res = y - (a + b * t)
            assert coef[r, 2] == pytest.approx(np.sqrt(np.mean(res ** 2)), rel=1e-9)
            # residual orthogonal to 1 and t; unit variance after normalising
            assert abs(z[r].sum()) < 1e-7 * n
            assert abs((z[r] * t).sum()) < 1e-7 * n * n
            assert np.mean(z[r] ** 2) == pytest.approx(1.0, rel=1e-12)


def pin_detrend_closed_form(P):
    # y = c + d t + e q(t), q orthogonal to 1 and t: the residual is e q exactly
    n = 257
    t = np.arange(n, dtype=np.float64)
    tm = (n - 1) / 2
    q = (t - tm) ** 2
    q -= q.mean()
    for c, d, e in ((3.0, 0.5, 2.0), (-40.0, -1.25, -0.75)):
        y = (c + d * t + e * q).astype(np.float32).astype(np.float64)
        x = y.astype(np.float32)[None, :]
        z, coef = P.detrend(x)
        rms = np.sqrt(np.mean(q * q))
        # float32 input rounding sets the tolerance
        assert coef[0, 0] == pytest.approx(c, abs=1e-3)
        assert coef[0, 1] == pytest.approx(d, abs=1e-5)
        assert coef[0, 2] == pytest.approx(abs(e) * rms, rel=1e-5)
        assert np.allclose(z[0], np.sign(e) * q / rms, atol=1e-4)


def pin_detrend_exact_line(P):
    t = np.arange(100, dtype=np.int64)
    x = (3 + 2 * t).astype(np.int32)[None, :]
    z, coef = P.detrend(x)
    assert not z.any()
    assert coef[0, 2] == pytest.approx(0.0, abs=1e-9)
    assert coef[0, 1] == pytest.approx(2.0) and coef[0, 0] == pytest.approx(3.0)
    z1, c1 = P.detrend(np.array([[5]], dtype=np.int32))  # one sample: nothing left
    assert not z1.any() and c1[0, 0] == 5.0 and c1[0, 2] == 0.0


# ------------------------------------------------------------------ boxcar

def pin_boxcar_sums_direct(P):
    rng = np.random.default_rng(5)
    x = rand_rows(rng, 3, 70, np.int32)
    sums = P.boxcar_sums(x, 7)
    c = np.concatenate([np.zeros((3, 1), dtype=np.int64), np.cumsum(x, axis=1, dtype=np.int64)],
                       axis=1)
    for j, s in enumerate(sums):
        w = 1 << j
        assert s.shape == (3, 70 - w + 1)
        assert np.array_equal(s, c[:, w:] - c[:, :-w])
    xf = rand_rows(rng, 2, 300, np.float32)
    for j, s in enumerate(P.boxcar_sums(xf, 6)):
        w = 1 << j
        ref = np.array([[xf[r, i:i + w].astype(np.float64).sum() for i in range(300 - w + 1)]
                        for r in range(2)])
        assert s.dtype == np.float32
        assert np.allclose(s, ref, rtol=0, atol=w * 2e-6 * np.abs(xf).max() * 4)
    assert P.boxcar_sums(x[:, :3], 4)[2].shape == (3, 0)


def pin_boxcar_top_hat(P):
    # a top-hat of height h and width W on a quiet series: at its start the
    # matched width W gives S/N = h sqrt(W) (fixed height: S/N grows as
    # sqrt(W)), and it beats every other width
    for W, t0 in ((1, 10), (4, 33), (16, 100), (64, 7)):
        for h in (1.0, 2.5):
            x = np.zeros((1, 400), dtype=np.float32)
            x[0, t0:t0 + W] = h
            nsig = 0.5 * h * math.sqrt(W)
            p = P.boxcar_detect(x, None, None, 8, nsig)
            at = p[p["t"] == t0]
            assert at.size == 1 and at["width"][0] == W
            assert at["snr"][0] == pytest.approx(h * math.sqrt(W), rel=1e-6)
            assert at["value"][0] == pytest.approx(h * W)
            # with a mean and sigma: (S - w mean)/(sigma sqrt w)
            q = P.boxcar_detect(x * 3 + 2, np.array([2.0]), np.array([3.0]), 8, nsig)
            assert np.array_equal(q["t"], p["t"]) and np.array_equal(q["width"], p["width"])
            assert np.allclose(q["snr"], p["snr"], rtol=1e-6)


def pin_boxcar_gaussian_tail(P):
    # chance events on N(0,1) noise: width w sums have sigma sqrt(w), so each
    # width alone exceeds 3 sigma at the normal tail rate Q(3)
    rng = np.random.default_rng(6)
    n = 400000
    x = rng.standard_normal((1, n)).astype(np.float32)
    q3 = 0.5 * math.erfc(3 / math.sqrt(2))
    for j in range(4):
        w = 1 << j
        s = P.boxcar_sums(x, j + 1)[j]
        snr = P.boxcar_snr(s, w, np.zeros(1), np.ones(1))
        frac = np.mean(snr > 3.0)
        sd = math.sqrt(q3 * (1 - q3) / s.size) * math.sqrt(w)  # correlated neighbours
        assert abs(frac - q3) < 6 * sd, (w, frac, q3)
    one = P.boxcar_detect(x, None, None, 1, 3.0)
    assert one.size == int(np.sum(x[0].astype(np.float64) > 3.0))


def pin_boxcar_rules(P):
    x = np.zeros((3, 32), dtype=np.int32)
    x[:, 5] = 10
    mean, sigma = np.zeros(3), np.array([1.0, 0.0, np.nan])
    p = P.boxcar_detect(x, mean, sigma, 3, 10.0)  # strict: snr 10 at width 1 is not > 10
    # width 2 from t=4 or 5: 10/sqrt(2) < 10; only rows with finite sigma > 0 count
    assert p.size == 0
    p = P.boxcar_detect(x, mean, sigma, 3, 4.0)
    assert set(p["dm_idx"]) == {0}
    # every boxcar that covers sample 5: t in 2..5 for widths up to 4
    assert list(p["t"]) == [2, 3, 4, 5]
    assert list(p["width"]) == [4, 4, 2, 1]  # largest S/N: 10/sqrt(w) with the smallest w covering
    assert np.all(np.diff(p["t"]) > 0)


PINS = [pin_median_brute_force, pin_median_scipy, pin_median_invariants,
        pin_detrend_polyfit_and_normal_equations, pin_detrend_closed_form, pin_detrend_exact_line,
        pin_boxcar_sums_direct, pin_boxcar_top_hat, pin_boxcar_gaussian_tail, pin_boxcar_rules]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_post_oracle_pin(pin):
    pin(P0)
