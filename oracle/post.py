"""CPU oracle for the post-processing of dedispersed series.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg use it; the
CUDA library neither imports nor links it.  Plain numpy, float64 wherever the
thesis leaves the precision open, written from the thesis:

* ``median_filter`` -- Sec. 3.5, median filtering: each value is replaced by
  the median of the window of ``width`` samples centred on it.
* ``detrend``       -- Sec. 3.5, detrending and normalisation: a least-squares
  line is fitted to each series (first pass), subtracted while the standard
  deviation of what remains is formed (second pass), and the series is divided
  by it (third pass).
* ``boxcar_detect`` -- Sec. 1.5.1 (single-pulse S/N and the smoothing that
  approaches optimal detection): the series is smoothed by successively adding
  adjacent groups of samples, widths 1, 2, 4, ..., and every width is
  thresholded at n sigma, the noise of a w-sample sum being sqrt(w) sigma.

Readings where the text is silent (each listed in the design notes):
median windows at the ends of a series repeat the end sample; widths are odd;
the detrending line is fitted over t = 0 .. n-1 and the standard deviation is
the population one (1/n), a series whose residual is exactly zero becomes
zeros; boxcar sums of width 2w are S_2w[t] = S_w[t] + S_w[t + w] (one add per
level, in this order, so float series round identically everywhere), the S/N
of width w at t is (S_w[t] - w mean) / (sigma sqrt(w)) in IEEE double with
the threshold strict, and each (series, t) with some width above threshold is
reported once, at its largest S/N (smallest width on ties).

Pins (``tests/test_oracle_post_pins.py``): brute force with Python's
``sorted`` and scipy's median filter, ``numpy.polyfit`` and the orthogonality
of the residual to 1 and t, a closed-form quadratic residual, direct window
sums, the top-hat pulse S/N of Sec. 1.5.1 and the Gaussian tail rate of false
events.
"""
from __future__ import annotations

import numpy as np
from numpy.lib.stride_tricks import sliding_window_view

PULSE_DTYPE = np.dtype([("dm_idx", np.int32), ("t", np.int32), ("width", np.int32),
                        ("snr", np.float32), ("value", np.float64)])

MAX_MEDIAN_WIDTH = 15
MAX_BOXCAR_WIDTHS = 12


def _rows(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x)
    if x.ndim != 2 or x.dtype not in (np.dtype(np.int32), np.dtype(np.float32)):
        raise ValueError("rows must be a 2-D int32 or float32 array")
    return x


def median_filter(x: np.ndarray, width: int) -> np.ndarray:
    """Sec. 3.5 median filtering of each row (window centred on the sample).

    ``width`` is odd, 1 .. 15; the window of a sample near either end of a
    row repeats that end sample.  The median of an odd number of values is
    one of them, so the result has the row's dtype exactly."""
    x = _rows(x)
    if width < 1 or width % 2 == 0 or width > MAX_MEDIAN_WIDTH:
        raise ValueError("width must be odd, 1..15")
    h = width // 2
    padded = np.pad(x, ((0, 0), (h, h)), mode="edge")
    windows = sliding_window_view(padded, width, axis=1)
    return np.sort(windows, axis=-1)[..., h].astype(x.dtype)


def detrend(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sec. 3.5 detrending and normalisation of each row, in three passes.

    Pass 1 fits y ~ a + b t (t = 0 .. n-1) by least squares; pass 2 forms the
    residual r = y - a - b t and its population standard deviation s; pass 3
    returns r / s (zeros where s == 0).  Returns (z as float64 [nrows][n],
    coefficients [nrows][3] = a, b, s)."""
    x = _rows(x)
    nrows, n = x.shape
    y = x.astype(np.float64)
    t = np.arange(n, dtype=np.float64)
    coef = np.zeros((nrows, 3))
    z = np.zeros((nrows, n))
    for r in range(nrows):
        # pass 1: regression parameters about the means of t and y
        t_mean = t.mean()
        y_mean = y[r].mean()
        stt = np.sum((t - t_mean) ** 2)
        b = np.sum((t - t_mean) * (y[r] - y_mean)) / stt if stt > 0 else 0.0
        a = y_mean - b * t_mean
        # pass 2: subtract the line, standard deviation of the remainder
        res = y[r] - (a + b * t)
        s = np.sqrt(np.mean(res * res))
        # pass 3: normalise
        if s > 0:
            z[r] = res / s
        coef[r] = a, b, s
    return z, coef


def boxcar_sums(x: np.ndarray, nwidths: int) -> list[np.ndarray]:
    """S_w for w = 1, 2, 4, ..., 2^(nwidths-1): S_1 = x, S_2w[t] = S_w[t] +
    S_w[t + w], t = 0 .. n - 2w.  int32 rows sum in int64 (exact), float32
    rows in float32 in exactly this order."""
    x = _rows(x)
    if nwidths < 1 or nwidths > MAX_BOXCAR_WIDTHS:
        raise ValueError("nwidths must be 1..12")
    s = x.astype(np.int64) if x.dtype == np.int32 else x.copy()
    sums = [s]
    for j in range(1, nwidths):
        half = 1 << (j - 1)
        if s.shape[1] <= half:
            s = s[:, :0]
        else:
            s = s[:, :-half] + s[:, half:]
        sums.append(s)
    return sums


def boxcar_snr(sum_w: np.ndarray, w: int, mean: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """(S_w - w mean) / (sigma sqrt(w)) in IEEE double, per row."""
    num = sum_w.astype(np.float64) - w * mean[:, None]
    return num / (sigma[:, None] * np.sqrt(np.float64(w)))


def boxcar_detect(x: np.ndarray, mean: np.ndarray | None, sigma: np.ndarray | None,
                  nwidths: int, nsigma: float) -> np.ndarray:
    """Single-pulse search over boxcar widths (Sec. 1.5.1).

    ``mean`` / ``sigma``: float64 per row (None: 0 and 1, as after
    ``detrend``).  Rows whose sigma is not finite and positive, or whose mean
    is not finite, give nothing.
    Returns PULSE_DTYPE records ordered by (dm_idx, t): for each (row, t) with
    some width w (t + w <= n) whose S/N exceeds ``nsigma``, the width with the
    largest S/N (smallest on ties), that S/N (rounded to float32) and S_w."""
    x = _rows(x)
    nrows, n = x.shape
    mean = np.zeros(nrows) if mean is None else np.asarray(mean, dtype=np.float64)
    sigma = np.ones(nrows) if sigma is None else np.asarray(sigma, dtype=np.float64)
    thr = np.float64(np.float32(nsigma))
    sums = boxcar_sums(x, nwidths)
    best = np.full((nrows, n), -np.inf)
    best_w = np.zeros((nrows, n), dtype=np.int32)
    best_v = np.zeros((nrows, n))
    ok = np.isfinite(sigma) & (sigma > 0) & np.isfinite(mean)
    with np.errstate(divide="ignore", invalid="ignore"):
        for j, s in enumerate(sums):
            w = 1 << j
            m = s.shape[1]
            if m == 0:
                continue
            snr = boxcar_snr(s, w, mean, sigma)
            hit = (snr > thr) & ok[:, None]
            better = hit & (snr > best[:, :m])
            best[:, :m] = np.where(better, snr, best[:, :m])
            best_w[:, :m] = np.where(better, w, best_w[:, :m])
            best_v[:, :m] = np.where(better, s.astype(np.float64), best_v[:, :m])
    rows, ts = np.nonzero(best_w > 0)
    out = np.zeros(rows.size, dtype=PULSE_DTYPE)
    out["dm_idx"] = rows
    out["t"] = ts
    out["width"] = best_w[rows, ts]
    out["snr"] = best[rows, ts].astype(np.float32)
    out["value"] = best_v[rows, ts]
    return out
