/*
 * dd_post.h -- C ABI of libdd's post-processing of dedispersed time series
 * (A. Magro 2013: Sec. 3.5 "signal post-processing"; Sec. 1.5.1 single-pulse
 * S/N and boxcar smoothing).
 *
 * Every call takes "rows": a device array [nrows][pitch] holding one
 * dedispersed series per DM trial, int32 (DD_ROWS_I32, the output of 8-bit
 * dedispersion) or IEEE float (DD_ROWS_F32), time fastest; only the first
 * ncols elements of each row are read.  Pitches are in elements.  Pointers
 * are device pointers unless stated; the caller owns every buffer.  Work is
 * queued on `stream` (a cudaStream_t, NULL for the default stream) on the
 * calling thread's current device; calls are asynchronous unless stated.
 * Argument errors are reported before anything is queued.  Return values are
 * dd_status codes (dd.h).
 */
#ifndef DD_POST_H
#define DD_POST_H

#include <stdint.h>

#include "dd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { DD_ROWS_I32 = 0, DD_ROWS_F32 = 1 } dd_rows_type;

/* Median filtering (Sec. 3.5, windowed median): out[r][t] is the median of
 * the `width` values in[r][clamp(t + k, 0, ncols - 1)], k = -h .. h,
 * width = 2h + 1 (odd, 1 .. 15; the thesis uses 5 or 7).  Near either end
 * of a row the window repeats the end sample.  The result is one of the
 * inputs, so it is exact for both row types (NaN inputs give unspecified
 * results).  out: [nrows][out_pitch] of the same type; it must not overlap
 * `in`.  DD_ERR_ARG: null pointer, width even or out of range, a pitch below
 * ncols, overlapping buffers; DD_ERR_SIZE: nrows < 1, ncols < 1 or
 * ncols > 2^31 - 1; DD_ERR_DTYPE: unknown rows_type. */
int dd_median_filter(const void *in, int64_t in_pitch, int32_t rows_type, int32_t nrows,
                     int64_t ncols, int32_t width, void *out, int64_t out_pitch, void *stream);

/* Detrending and normalisation (Sec. 3.5): per row, the least-squares line
 * a + b t over t = 0 .. ncols-1, the residual r = y - a - b t, its population
 * standard deviation s = sqrt(mean(r^2)), and out = r / s as float (all
 * zeros when s == 0, which includes ncols == 1).  The line is fitted from
 * exact 128-bit integer sums for DD_ROWS_I32 rows (a residual that is exactly
 * zero gives s == 0 exactly) and from double sums about the row's first value
 * for DD_ROWS_F32 rows; out is formed in float, so it agrees with the exact
 * result to within a few float roundings of |r| + |a| + |b| ncols, divided
 * by s.  out: float [nrows][out_pitch]; it may be `in` itself for
 * DD_ROWS_F32 rows with out_pitch == in_pitch, otherwise it must not overlap
 * `in`.  coef: double [nrows][3] = (a, b, s) per row, or NULL.
 * DD_ERR_SIZE also for ncols > 2^24 (the exact integer sums' range). */
int dd_detrend(const void *in, int64_t in_pitch, int32_t rows_type, int32_t nrows, int64_t ncols,
               float *out, int64_t out_pitch, double *coef, void *stream);

/* One single-pulse detection: DM trial (row), boxcar start sample, boxcar
 * width in samples, its S/N (rounded to float) and the boxcar sum S_w[t]. */
typedef struct {
  int32_t dm_idx;
  int32_t t;
  int32_t width;
  float snr;
  double value;
} dd_pulse;

/* Bytes of device workspace dd_boxcar_detect needs for nrows x ncols. */
int dd_boxcar_workspace_bytes(int32_t nrows, int64_t ncols, int64_t *bytes);

/* Boxcar single-pulse search (Sec. 1.5.1: the series is smoothed by
 * successively adding adjacent samples, which approaches optimal detection
 * for pulses of unknown width, and each smoothing is thresholded).
 *   S_1[t] = x[t];  S_2w[t] = S_w[t] + S_w[t + w]       (w = 1, 2, 4, ...)
 * for widths w = 2^j, j < nwidths (1 .. 12), t + w <= ncols.  Sums are exact
 * int64 for DD_ROWS_I32 rows and float, in exactly this order, for
 * DD_ROWS_F32 rows, so both are reproducible bit for bit.  The S/N of (t, w)
 * is (S_w[t] - w mean) / (sigma sqrt(w)) evaluated in IEEE double (each
 * operation correctly rounded, in this order), with mean / sigma the row's
 * (device double[nrows]; NULL: 0 and 1, e.g. after dd_detrend).  Every
 * (row, t) where some width's S/N exceeds nsigma (strictly) gives one pulse,
 * at the width with the largest S/N (the smallest width on ties); rows whose
 * sigma is not finite and positive, or whose mean is not finite, give none.
 * Pulses are written to `pulses` (device, `capacity` entries, may be NULL
 * when capacity == 0) in (dm_idx, t) order; *count (host) receives the total
 * found.  workspace: device, at least dd_boxcar_workspace_bytes(nrows, ncols)
 * bytes, no alignment beyond 16 bytes needed, contents not preserved; work
 * on one workspace must not overlap in time.  Synchronises `stream` once.
 * Returns DD_ERR_OVERFLOW when the total exceeds capacity (the first
 * capacity pulses are still written); DD_ERR_ARG for nwidths out of range,
 * a non-finite nsigma or a short workspace; DD_ERR_SIZE for nrows < 1,
 * ncols < 1 or ncols > 2^31 - 1. */
int dd_boxcar_detect(const void *rows, int64_t pitch, int32_t rows_type, int32_t nrows,
                     int64_t ncols, const double *mean, const double *sigma, int32_t nwidths,
                     float nsigma, void *workspace, int64_t workspace_bytes, dd_pulse *pulses,
                     int64_t capacity, int64_t *count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DD_POST_H */
