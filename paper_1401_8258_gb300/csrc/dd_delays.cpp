// dd_delays.cpp -- host-side discretised dispersion delays and status strings.
//
// Compiled by the host C++ compiler with -ffp-contract=off so that every
// multiply and add below rounds on its own (no fused multiply-add), on x86-64
// and on aarch64 alike.
#include <cmath>
#include <cstdint>

#include "dd.h"

namespace {

// Dispersion constant in MHz^2 pc^-1 cm^3 s (Sec. 1.2.1, dispersion equation).
constexpr double kDispersionConstant = 4.148808e3;

}  // namespace

// Sec. 2.1.1, deltaT equation:
//   dT(c)      = K * ((f_top - c*df)^-2 - f_top^-2) / t_samp
//   delay(c,d) = round(DM_d * dT(c))        (round half away from zero)
// Channel 0 is the band top (delay 0); channel c sits c*df below it.
extern "C" int dd_compute_delays(int32_t nchan, double f_top_mhz, double chan_width_mhz,
                                 double t_samp_s, const double *dm_list, int32_t ndm,
                                 int32_t *delays_out, int32_t *maxshift_out) {
  if (nchan < 1 || ndm < 1 || !dm_list || !delays_out || !maxshift_out) return DD_ERR_ARG;
  if (!(chan_width_mhz > 0.0) || !(t_samp_s > 0.0) || !std::isfinite(f_top_mhz) ||
      !std::isfinite(chan_width_mhz) || !std::isfinite(t_samp_s))
    return DD_ERR_ARG;
  const double f_bottom = f_top_mhz - static_cast<double>(nchan - 1) * chan_width_mhz;
  if (!(f_bottom > 0.0)) return DD_ERR_ARG;
  for (int32_t d = 0; d < ndm; ++d)
    if (!std::isfinite(dm_list[d]) || !(dm_list[d] >= 0.0)) return DD_ERR_ARG;

  const double inv_top_sq = 1.0 / (f_top_mhz * f_top_mhz);
  int32_t largest = 0;
  for (int32_t c = 0; c < nchan; ++c) {
    const double f_c = f_top_mhz - static_cast<double>(c) * chan_width_mhz;
    const double per_dm = kDispersionConstant * (1.0 / (f_c * f_c) - inv_top_sq) / t_samp_s;
    int32_t *row = delays_out + static_cast<int64_t>(c) * ndm;
    for (int32_t d = 0; d < ndm; ++d) {
      const double shift = std::round(dm_list[d] * per_dm);
      if (!(shift <= 2147483647.0)) return DD_ERR_RANGE;
      row[d] = static_cast<int32_t>(shift);
      if (row[d] > largest) largest = row[d];
    }
  }
  *maxshift_out = largest;
  return DD_OK;
}

extern "C" const char *dd_status_string(int status) {
  switch (status) {
    case DD_OK: return "ok";
    case DD_ERR_ARG: return "invalid argument";
    case DD_ERR_SIZE: return "size out of range";
    case DD_ERR_DTYPE: return "unknown input dtype";
    case DD_ERR_CUDA: return "CUDA runtime error";
    case DD_ERR_OOM: return "out of memory";
    case DD_ERR_OVERFLOW: return "more candidates than capacity";
    case DD_ERR_DEVICE_TIMEOUT: return "bounded device wait ran out";
    case DD_ERR_RANGE: return "value out of representable range";
    default: return "unknown status";
  }
}
