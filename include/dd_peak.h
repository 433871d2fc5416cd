/*
 * dd_peak.h -- add-pipe throughput probes (measurement support, not part of
 * the dedispersion path).
 *
 * The brute-force dedispersion sum (Sec. 2.1.1) costs one add per
 * (channel, DM trial, sample); its roofline is therefore the rate at which
 * an SM retires 32-bit adds.  dd_measure_add_peak runs one instruction form
 * in eight independent chains per thread on every SM of `device` and reports
 * the rate both in operations per second and per clock per SM (cycles read
 * inside the kernel).  A two-lane form (DD_PEAK_FADD2, DD_PEAK_IADD3) counts
 * two operations per instruction.  Returns 0, or DD_PEAK_ERR on a CUDA
 * error.  Allocates and frees a few kilobytes of device memory; synchronous.
 */
#ifndef DD_PEAK_H
#define DD_PEAK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DD_PEAK_FADD = 0,      /* add.rn.f32 */
  DD_PEAK_FADD2 = 1,     /* add.rn.f32x2 (two f32 adds per instruction) */
  DD_PEAK_IADD = 2,      /* add.u32 */
  DD_PEAK_IADD3 = 3,     /* two dependent add.u32, fusable into one three-input add */
  DD_PEAK_IMAD = 4,      /* mad.lo.u32 */
  DD_PEAK_LOP3 = 5,      /* lop3.b32 */
  DD_PEAK_PRMT = 6,      /* prmt.b32 */
  DD_PEAK_HADD2 = 7,     /* add.rn.f16x2 */
  DD_PEAK_FADD_F16 = 8,  /* add.rn.f32.f16 (f16 operand into an f32 sum) */
  DD_PEAK_PRMT_IADD = 9, /* byte unpack (prmt) feeding a 32-bit add */
  DD_PEAK_LOP3_IADD = 10 /* byte mask (and) feeding a 32-bit add */
};

#define DD_PEAK_ERR (-4)

int dd_measure_add_peak(int32_t kind, int32_t device, double *ops_per_s,
                        double *ops_per_clk_per_sm);

#ifdef __cplusplus
}
#endif

#endif /* DD_PEAK_H */
