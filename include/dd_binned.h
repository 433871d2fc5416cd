/*
 * dd_binned.h -- C ABI of libdd's time-binned dedispersion: past the
 * diagonal DM the higher DM ranges are dedispersed from the series
 * downfactored by 2, 4, ... (A. Magro 2013, Sec. 2.1.1 on the diagonal DM
 * and the downfactoring procedure of Sec. 2.1.2).
 *
 * Diagonal DM (the DM whose sweep across one channel at the bottom of the
 * band is one sample): DM_diag = t_samp f_bot^3 / (2 K df), f_bot = f_top -
 * (nchan - 1) df, K = 4.148808e3, in double, f_bot^3 as f_bot*f_bot*f_bot.
 * Trial d gets the downfactor 1 below 2 DM_diag, else the largest power of
 * two f <= max_factor with DM_d >= f DM_diag.  A trial with downfactor f is
 * dedispersed from the block binned by f -- adjacent samples summed in pairs,
 * log2(f) times: b[c][t] = a[c][2t] + a[c][2t+1] -- with the delays of
 * dd_plan_create at sampling time f t_samp, over the trials that share f:
 *   out[d][t] = sum_c B_f[c][t + delay_f(c, d)],  t < nsamp_out(d),
 *   nsamp_out(d) = floor(nsamp_in / f) - (largest delay_f of those trials).
 * Each output sample of such a row covers f input samples.  u8 input: the
 * binned series are integer sums carried in float (exact below 2^24, hence
 * DD_ERR_RANGE when nchan * 255 * max_factor >= 2^24) and every row is int32;
 * f16/f32 input: float rows (float pair sums, float accumulation).
 *
 * DD_BIN_MEAN_U8 (u8 input only; a variant, not in the thesis): the binned
 * series stay 8-bit -- each halving takes the pair's mean rounded half up,
 * b[c][t] = (a[c][2t] + a[c][2t+1] + 1) >> 1 -- so the binned trials run
 * through the 8-bit kernel like the full-rate ones.  A binned row is then
 * the summed row divided by f plus a rounding term between 0 and
 * nchan * log2(f) / 2 counts; rows stay exact int32 sums of the 8-bit
 * series.  Only the binning differs; downfactors, delays and lengths are
 * those of DD_BIN_SUM.
 */
#ifndef DD_BINNED_H
#define DD_BINNED_H

#include <stdint.h>

#include "dd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_binned dd_binned; /* opaque; owns one plan per downfactor and the binned series */

typedef enum {
  DD_BIN_SUM = 0,     /* pair sums (the thesis's downfactoring) */
  DD_BIN_MEAN_U8 = 1  /* 8-bit pair means rounded half up (u8 input) */
} dd_bin_mode;

/* Geometry and DM list as for dd_plan_create, with the DM list
 * non-decreasing (so each downfactor covers consecutive trials; DD_ERR_ARG
 * otherwise); max_factor a power of two in 1..64; mode a dd_bin_mode
 * (DD_ERR_ARG otherwise; DD_BIN_MEAN_U8 with f16/f32 input: DD_ERR_DTYPE). */
int dd_binned_create(dd_binned **out, int32_t nchan, double f_top_mhz, double chan_width_mhz,
                     double t_samp_s, const double *dm_list, int32_t ndm, int32_t in_dtype,
                     int32_t max_factor, int32_t mode, int32_t device);
int dd_binned_destroy(dd_binned *b);

int dd_binned_diagonal_dm(const dd_binned *b, double *dm_diag);

/* Per trial, host arrays of ndm entries (either may be NULL): its downfactor
 * and its output length for a block of nsamp_in samples (DD_ERR_SIZE when
 * some trial would have no output). */
int dd_binned_rows(const dd_binned *b, int64_t nsamp_in, int32_t *factor, int64_t *nsamp_out);

/* Dedisperse one block (device, [nchan][pitch_elems] of the dtype, first
 * nsamp_in samples of each row read) on `stream`: row d of out (device,
 * [ndm][out_pitch], int32 for u8 input, float otherwise) gets its
 * nsamp_out(d) samples; the rest of the row is not written.  out_pitch must
 * cover the longest row (DD_ERR_ARG).  The first call for a given nsamp_in
 * grows the binned-series workspace (about nchan x nsamp_in x 4 bytes for
 * DD_BIN_SUM, nchan x nsamp_in bytes for DD_BIN_MEAN_U8) and synchronises
 * the device; later calls are asynchronous. */
int dd_binned_execute(dd_binned *b, const void *block, int64_t nsamp_in, int64_t pitch_elems,
                      void *out, int64_t out_pitch, void *stream);

/* Kernel launches queued by this object since creation. */
int dd_binned_launch_count(const dd_binned *b, int64_t *launches);

/* Synchronise `stream` and return DD_ERR_DEVICE_TIMEOUT if a bounded wait
 * of any launch of this object ran out since the last call (clearing it),
 * else DD_OK -- dd_sync for the plans inside. */
int dd_binned_sync(dd_binned *b, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DD_BINNED_H */
