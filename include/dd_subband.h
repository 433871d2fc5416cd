/*
 * dd_subband.h -- C ABI of libdd's subband dedispersion: the two-step
 * approximation of the brute-force sum (A. Magro 2013, Sec. 2.1.3).
 *
 * The trial DMs fall into groups of `dms_per_group` consecutive trials, each
 * represented by one nominal trial (its middle one; the lower middle one for
 * an even group).  With T[c][d] the brute-force delay table of dd_plan_create
 * and c_s the first channel of subband s (`chans_per_subband` adjacent
 * channels; the last subband may be narrower):
 *   step 1  SB[n][s][t] = sum_{c in s} I[c][t + T[c][n] - T[c_s][n]]
 *           (each subband dedispersed at the nominal trials only);
 *   step 2  out[d][t]  = sum_s SB[n(d)][s][t + T[c_s][d]]
 *           (the subband series dedispersed as channels at every trial of
 *           the nominal's group).
 * At a nominal trial the result equals the brute-force sum exactly; at the
 * others each subband keeps its nominal trial's internal delays, which
 * smears a pulse as a DM error of (trial - nominal) over one subband's
 * bandwidth would (the incorrect-dedispersion curve of Sec. 3.6).  The work
 * drops from nchan * ndm adds per sample to about
 *   nchan * ndm / dms_per_group + (nchan / chans_per_subband) * ndm.
 *
 * Output length: nsamp_out = nsamp_in - maxshift with maxshift = D1 + D2,
 * D1 the largest step-1 delay and D2 the largest step-2 delay (it can be
 * slightly below the brute-force maxshift: the step-1 delays reach only the
 * nominal trials).  Types as for dd_execute: u8 input gives int32 output
 * (exact integer sums: the step-1 series kept as 16-bit integers when
 * chans_per_subband * 255 <= 65535, else carried through float, which is
 * exact below 2^24, hence DD_ERR_RANGE when nchan * 255 >= 2^24), f16/f32
 * input gives float (step-1 series kept in float).
 */
#ifndef DD_SUBBAND_H
#define DD_SUBBAND_H

#include <stdint.h>

#include "dd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_subband dd_subband; /* opaque; owns its step plans and workspace */

/* Geometry and DM list as for dd_plan_create; chans_per_subband >= 1,
 * dms_per_group >= 1 (1 and 1 reduce to the brute-force sum).  Builds one
 * plan per subband (step 1) and one per group (step 2) on `device`. */
int dd_subband_create(dd_subband **out, int32_t nchan, double f_top_mhz, double chan_width_mhz,
                      double t_samp_s, const double *dm_list, int32_t ndm, int32_t in_dtype,
                      int32_t chans_per_subband, int32_t dms_per_group, int32_t device);
int dd_subband_destroy(dd_subband *s);

/* maxshift = D1 + D2 (above); nsamp_out = nsamp_in - maxshift. */
int dd_subband_max_delay(const dd_subband *s, int32_t *maxshift);

/* Host copy of the nominal trial of each group: nominal[0 .. ngroups), with
 * ngroups = ceil(ndm / dms_per_group) (either pointer may be NULL). */
int dd_subband_nominal(const dd_subband *s, int32_t *nominal, int32_t *ngroups);

/* Subband dedispersion of one block on `stream`: block and pitch as for
 * dd_execute (device, [nchan][pitch_elems], the first nsamp_in samples of
 * each row read); out: device [ndm][nsamp_out], int32 for u8 input, float
 * otherwise, every element written.  The first call for a given nsamp_in
 * grows the step-1 workspace (nominal trials x subbands x samples x 4 bytes)
 * and synchronises the device; later calls are asynchronous.  Kernel
 * selection follows dd_execute (staged kernels where the layout allows). */
int dd_subband_execute(dd_subband *s, const void *block, int64_t nsamp_in, int64_t pitch_elems,
                       void *out, void *stream);

/* Kernel launches queued by this object since creation. */
int dd_subband_launch_count(const dd_subband *s, int64_t *launches);

/* Synchronise `stream` and return DD_ERR_DEVICE_TIMEOUT if a bounded wait
 * of any launch of this object ran out since the last call (clearing it),
 * else DD_OK -- dd_sync for the step plans inside. */
int dd_subband_sync(dd_subband *s, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DD_SUBBAND_H */
