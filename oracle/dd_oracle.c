/*
 * dd_oracle.c -- plain CPU oracle for brute-force incoherent dedispersion
 * followed by per-DM-trial normalisation and n-sigma candidate extraction.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists so that the tests, the smoke
 * check and the timed CPU baseline have an obviously correct, slow reference
 * to compare the CUDA library against.  The CUDA library never calls, links
 * or includes anything from here, and nothing here is taken from it: the
 * delay rule, the half-precision decoder, the statistics and the candidate
 * rule are each written out below from the thesis text.
 *
 * Thesis passages followed (A. Magro, "A Real-Time, GPU-Based, Non-Imaging
 * Back-End for Radio Telescopes", 2013):
 *   - dispersion constant D = 4.148808e3 MHz^2 pc^-1 cm^3 s       (Sec. 1.2.1, dispersion equation)
 *   - delay between two frequencies, k_DM * DM * (f1^-2 - f2^-2)  (Sec. 1.2.1, dispersion relationship equation)
 *   - direct dedispersion D[d][t] = sum_c A[c][t + dt(d,c)]       (Sec. 2.1.1, brute-force equation)
 *   - discretised delay dT(c), dt(d,c) = round(DM(d) dT(c))       (Sec. 2.1.1, deltaT equation)
 *   - valid output length = nsamp - maxshift (overlap carry)      (Sec. 3.4, Dedispersion)
 *   - normalisation of the dedispersed series                      (Sec. 3.5, Detrending and Normalisation)
 *   - n-sigma thresholding into (time, DM, intensity) triplets     (Sec. 3.6, Detection and Candidate Selection)
 *
 * Readings where the text is silent (each is also listed in the design notes):
 *   - channel c has frequency f_top - c*df (df > 0): channel 0 is the band top,
 *     so its delay is 0 for every DM;
 *   - round() is round-half-away-from-zero (C99 round);
 *   - the expression is evaluated in IEEE double, left to right, as
 *       dT = K * (1/(f_c*f_c) - 1/(f_top*f_top)) / t_samp ;  delay = round(DM * dT)
 *     with no fused multiply-add (compile with -ffp-contract=off);
 *   - "normalisation" is mean / population standard deviation (1/N) per DM
 *     row, no detrending; a candidate is snr = (D - mean)/sigma > nsigma
 *     (strict), rows with sigma == 0 give no candidates; candidates are listed
 *     in (dm index, time) order.
 *
 * Accumulation: u8 input is summed in int64 (exact) and stored as int32;
 * f16 and f32 input is widened exactly to double and summed in double in
 * channel order c = 0 .. nchan-1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Dispersion constant in MHz^2 pc^-1 cm^3 s (Sec. 1.2.1). */
static const double ORACLE_KDM = 4.148808e3;

enum { OR_U8 = 0, OR_F16 = 1, OR_F32 = 2 };
enum { OR_OK = 0, OR_EARG = -1, OR_ERANGE = -2, OR_ENOMEM = -3 };

typedef struct {
  int32_t dm_idx;
  int32_t t;
  float value;
  float snr;
} oracle_candidate;

/* ------------------------------------------------------------------ delays */

/* Discretised dispersion delay table, Sec. 2.1.1 (deltaT equation).
 * delays[c*ndm + d] = round(dm[d] * dT(c)),
 * dT(c) = K * ((f_top - c*df)^-2 - f_top^-2) / t_samp. */
int32_t oracle_delay_table(int32_t nchan, double f_top, double df, double t_samp,
                           const double *dm, int32_t ndm, int32_t *delays,
                           int32_t *maxshift) {
  if (nchan < 1 || ndm < 1 || !dm || !delays || !maxshift) return OR_EARG;
  if (!(df > 0.0) || !(t_samp > 0.0) || !(f_top - (double)(nchan - 1) * df > 0.0))
    return OR_EARG;
  for (int32_t d = 0; d < ndm; ++d)
    if (!(dm[d] >= 0.0) || !isfinite(dm[d])) return OR_EARG;
  int32_t mx = 0;
  for (int32_t c = 0; c < nchan; ++c) {
    double f_c = f_top - (double)c * df;
    double dT = ORACLE_KDM * (1.0 / (f_c * f_c) - 1.0 / (f_top * f_top)) / t_samp;
    for (int32_t d = 0; d < ndm; ++d) {
      double x = round(dm[d] * dT);
      if (!(x <= 2147483647.0)) return OR_ERANGE;
      int32_t v = (int32_t)x;
      delays[(int64_t)c * ndm + d] = v;
      if (v > mx) mx = v;
    }
  }
  *maxshift = mx;
  return OR_OK;
}

/* ---------------------------------------------------------- half decoding */

/* IEEE 754 binary16 -> double, exact (every half is a double). */
static double oracle_half_to_double(uint16_t h) {
  int sign = (h >> 15) & 1;
  int e = (h >> 10) & 0x1f;
  int m = h & 0x3ff;
  double v;
  if (e == 0)
    v = ldexp((double)m, -24); /* subnormal: m * 2^-24 */
  else if (e == 31)
    v = (m == 0) ? INFINITY : NAN;
  else
    v = ldexp((double)(m + 1024), e - 25); /* (1 + m/1024) * 2^(e-15) */
  return sign ? -v : v;
}

/* ----------------------------------------------------------- dedispersion */

/* Brute-force dedispersion, Sec. 2.1.1:
 *   D[d][t] = sum_{c=0}^{nchan-1} A[c][t + delays[c][d]],  0 <= t < nsamp_out.
 * Loop order d -> c -> t.  block is [nchan][pitch] with time fastest.
 * out is int32 [ndm][nsamp_out] for u8 input, double [ndm][nsamp_out] else.
 * nthreads <= 0 uses the OpenMP default. */
int32_t oracle_dedisperse(int32_t dtype, const void *block, int32_t nchan,
                          int64_t nsamp_in, int64_t pitch, const int32_t *delays,
                          int32_t ndm, int64_t nsamp_out, void *out,
                          int32_t nthreads) {
  if (!block || !delays || !out || nchan < 1 || ndm < 1 || nsamp_out < 0 ||
      pitch < nsamp_in)
    return OR_EARG;
  if (dtype != OR_U8 && dtype != OR_F16 && dtype != OR_F32) return OR_EARG;
  for (int64_t i = 0; i < (int64_t)nchan * ndm; ++i)
    if (delays[i] < 0 || (int64_t)delays[i] + nsamp_out > nsamp_in) return OR_ERANGE;
  if (nsamp_out == 0) return OR_OK;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
  nthreads = 1;
#endif
  int32_t status = OR_OK;
#pragma omp parallel num_threads(nthreads)
  {
    void *acc = malloc((size_t)nsamp_out * 8);
    if (!acc) {
#pragma omp atomic write
      status = OR_ENOMEM;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t d = 0; d < ndm; ++d) {
      if (!acc) continue;
      if (dtype == OR_U8) {
        int64_t *a = (int64_t *)acc;
        memset(a, 0, (size_t)nsamp_out * 8);
        for (int32_t c = 0; c < nchan; ++c) {
          const uint8_t *row = (const uint8_t *)block + (int64_t)c * pitch +
                               delays[(int64_t)c * ndm + d];
          for (int64_t t = 0; t < nsamp_out; ++t) a[t] += row[t];
        }
        int32_t *o = (int32_t *)out + (int64_t)d * nsamp_out;
        for (int64_t t = 0; t < nsamp_out; ++t) {
          if (a[t] > 2147483647LL) {
#pragma omp atomic write
            status = OR_ERANGE;
          }
          o[t] = (int32_t)a[t];
        }
      } else {
        double *a = (double *)out + (int64_t)d * nsamp_out;
        memset(a, 0, (size_t)nsamp_out * 8);
        for (int32_t c = 0; c < nchan; ++c) {
          int64_t off = (int64_t)c * pitch + delays[(int64_t)c * ndm + d];
          if (dtype == OR_F32) {
            const float *row = (const float *)block + off;
            for (int64_t t = 0; t < nsamp_out; ++t) a[t] += (double)row[t];
          } else {
            const uint16_t *row = (const uint16_t *)block + off;
            for (int64_t t = 0; t < nsamp_out; ++t) a[t] += oracle_half_to_double(row[t]);
          }
        }
      }
    }
    free(acc);
  }
  return status;
}

/* ------------------------------------------------------------- statistics */

/* Per-DM mean and population standard deviation of integer rows
 * (Sec. 3.5 normalisation).  Exact integer sums S1 = sum D, S2 = sum D^2,
 * then one written finaliser in double:
 *   mean  = S1 / N
 *   sigma = sqrt( (double)(N*S2 - S1*S1) ) / N
 * where N*S2 - S1^2 >= 0 is formed exactly in 128-bit integers and converted
 * to double with round-to-nearest-even. */
int32_t oracle_stats_i32(const int32_t *D, int32_t ndm, int64_t n, double *mean,
                         double *sigma) {
  if (!D || !mean || !sigma || ndm < 1 || n < 1) return OR_EARG;
  for (int32_t d = 0; d < ndm; ++d) {
    const int32_t *row = D + (int64_t)d * n;
    __int128 s1 = 0, s2 = 0;
    for (int64_t t = 0; t < n; ++t) {
      s1 += row[t];
      s2 += (__int128)((int64_t)row[t] * (int64_t)row[t]);
    }
    __int128 num = (__int128)n * s2 - s1 * s1;
    double dn = (double)n;
    mean[d] = (double)(int64_t)s1 / dn;
    sigma[d] = sqrt((double)(unsigned __int128)num) / dn;
  }
  return OR_OK;
}

/* Per-DM mean and population standard deviation of real rows, two-pass in
 * double: mean = sum D / N, sigma = sqrt(sum (D - mean)^2 / N). */
int32_t oracle_stats_f64(const double *D, int32_t ndm, int64_t n, double *mean,
                         double *sigma) {
  if (!D || !mean || !sigma || ndm < 1 || n < 1) return OR_EARG;
  for (int32_t d = 0; d < ndm; ++d) {
    const double *row = D + (int64_t)d * n;
    double s = 0.0;
    for (int64_t t = 0; t < n; ++t) s += row[t];
    double mu = s / (double)n;
    double q = 0.0;
    for (int64_t t = 0; t < n; ++t) q += (row[t] - mu) * (row[t] - mu);
    mean[d] = mu;
    sigma[d] = sqrt(q / (double)n);
  }
  return OR_OK;
}

/* ------------------------------------------------------------- candidates */

/* n-sigma thresholding into (DM, time, intensity) triplets, Sec. 3.6.
 * snr = ((double)D - mean[d]) / sigma[d]; a candidate iff sigma[d] > 0 and
 * snr > nsigma.  Candidates are written in (d, t) order, at most capacity of
 * them; *total receives the number found. */
static int32_t oracle_detect_any(int is_int, const void *Dv, int32_t ndm, int64_t n,
                                 const double *mean, const double *sigma,
                                 float nsigma, oracle_candidate *cands,
                                 int64_t capacity, int64_t *total) {
  if (!Dv || !mean || !sigma || !total || ndm < 1 || n < 0 || capacity < 0)
    return OR_EARG;
  if (capacity > 0 && !cands) return OR_EARG;
  int64_t k = 0;
  double thr = (double)nsigma;
  for (int32_t d = 0; d < ndm; ++d) {
    if (!(sigma[d] > 0.0)) continue;
    for (int64_t t = 0; t < n; ++t) {
      double v = is_int ? (double)((const int32_t *)Dv)[(int64_t)d * n + t]
                        : ((const double *)Dv)[(int64_t)d * n + t];
      double snr = (v - mean[d]) / sigma[d];
      if (snr > thr) {
        if (k < capacity) {
          cands[k].dm_idx = d;
          cands[k].t = (int32_t)t;
          cands[k].value = (float)v;
          cands[k].snr = (float)snr;
        }
        ++k;
      }
    }
  }
  *total = k;
  return OR_OK;
}

int32_t oracle_detect_i32(const int32_t *D, int32_t ndm, int64_t n, const double *mean,
                          const double *sigma, float nsigma, oracle_candidate *cands,
                          int64_t capacity, int64_t *total) {
  return oracle_detect_any(1, D, ndm, n, mean, sigma, nsigma, cands, capacity, total);
}

int32_t oracle_detect_f64(const double *D, int32_t ndm, int64_t n, const double *mean,
                          const double *sigma, float nsigma, oracle_candidate *cands,
                          int64_t capacity, int64_t *total) {
  return oracle_detect_any(0, D, ndm, n, mean, sigma, nsigma, cands, capacity, total);
}

/* Number of OpenMP threads the oracle would use by default. */
int32_t oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
