// dd_subband.cu -- subband dedispersion (Sec. 2.1.3) as two brute-force
// passes over derived delay tables, each run by the library's dedispersion
// kernels through plans built with dd_plan_create_from_delays:
//   step 1: one plan per subband (its channels x the nominal trials), rows
//           written interleaved as SB[n][s][t] (dd_execute_pitched);
//   step 2: one plan per DM group (the subbands as channels x the group's
//           trials), reading SB[n] as a float block.
// For u8 input the step-1 sums (int32) are converted to float in place
// before step 2 and the float result back to int32 after it; both
// conversions are exact (|values| < 2^24).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <vector>

#include "dd.h"
#include "dd_subband.h"

struct dd_subband {
  int32_t device = 0, nchan = 0, ndm = 0, dtype = 0;
  int32_t cps = 0, dpg = 0, nsub = 0, ngroups = 0;
  std::vector<int32_t> first;    // first channel of each subband
  std::vector<int32_t> nominal;  // nominal trial of each group
  std::vector<dd_plan *> step1;  // per subband
  std::vector<dd_plan *> step2;  // per group
  std::vector<int32_t> shift1, shift2;
  int32_t D1 = 0, D2 = 0;
  void *d_sb = nullptr;  // step-1 series [ngroups][nsub][L1pad], 4-byte elements
  size_t sb_bytes = 0;
  int64_t launches = 0;
};

namespace {

constexpr int kConvThreads = 256;

// In-place int32 -> float over rows [nrows][pitch] (first ncols of each).
__global__ void to_float_rows(int32_t *p, int64_t nrows, int64_t ncols, int64_t pitch) {
  const int64_t n = nrows * ncols;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int32_t *q = p + (i / ncols) * pitch + i % ncols;
    *reinterpret_cast<float *>(q) = static_cast<float>(*q);  // exact below 2^24
  }
}

// In-place float -> int32 (values are integers below 2^24).
__global__ void to_int_rows(float *p, int64_t n) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    reinterpret_cast<int32_t *>(p)[i] = __float2int_rn(p[i]);
  }
}

unsigned conv_grid(int64_t n) {
  const int64_t b = (n + kConvThreads - 1) / kConvThreads;
  return static_cast<unsigned>(std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16));
}

int elem_bytes(int32_t dtype) { return dtype == DD_U8 ? 1 : (dtype == DD_F16 ? 2 : 4); }

void destroy(dd_subband *s) {
  for (dd_plan *p : s->step1) dd_plan_destroy(p);
  for (dd_plan *p : s->step2) dd_plan_destroy(p);
  if (s->d_sb) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaFree(s->d_sb);
    cudaSetDevice(prev);
  }
  delete s;
}

}  // namespace

extern "C" int dd_subband_create(dd_subband **out, int32_t nchan, double f_top_mhz,
                                 double chan_width_mhz, double t_samp_s, const double *dm_list,
                                 int32_t ndm, int32_t in_dtype, int32_t chans_per_subband,
                                 int32_t dms_per_group, int32_t device) {
  if (!out) return DD_ERR_ARG;
  *out = nullptr;
  if (in_dtype != DD_U8 && in_dtype != DD_F16 && in_dtype != DD_F32) return DD_ERR_DTYPE;
  if (nchan < 1 || ndm < 1 || !dm_list || chans_per_subband < 1 || dms_per_group < 1 ||
      device < 0)
    return DD_ERR_ARG;
  if (in_dtype == DD_U8 && static_cast<int64_t>(nchan) * 255 >= (1 << 24)) return DD_ERR_RANGE;
  std::vector<int32_t> T;
  try {
    T.resize(static_cast<size_t>(nchan) * ndm);
  } catch (...) {
    return DD_ERR_OOM;
  }
  int32_t mx = 0;
  int st = dd_compute_delays(nchan, f_top_mhz, chan_width_mhz, t_samp_s, dm_list, ndm, T.data(),
                             &mx);
  if (st != DD_OK) return st;
  auto at = [&](int32_t c, int32_t d) { return T[static_cast<size_t>(c) * ndm + d]; };

  dd_subband *s = new (std::nothrow) dd_subband();
  if (!s) return DD_ERR_OOM;
  s->device = device;
  s->nchan = nchan;
  s->ndm = ndm;
  s->dtype = in_dtype;
  s->cps = chans_per_subband;
  s->dpg = dms_per_group;
  try {
    for (int32_t c = 0; c < nchan; c += chans_per_subband) s->first.push_back(c);
    for (int32_t g0 = 0; g0 < ndm; g0 += dms_per_group) {
      const int32_t g1 = std::min(ndm, g0 + dms_per_group);
      s->nominal.push_back(g0 + (g1 - g0 - 1) / 2);
    }
    s->nsub = static_cast<int32_t>(s->first.size());
    s->ngroups = static_cast<int32_t>(s->nominal.size());
    const int32_t nnom = s->ngroups;
    // step 1: subband s, delays T[c][n] - T[c_s][n] over its channels
    for (int32_t k = 0; k < s->nsub; ++k) {
      const int32_t c0 = s->first[k], nc = std::min(chans_per_subband, nchan - c0);
      std::vector<int32_t> tab(static_cast<size_t>(nc) * nnom);
      for (int32_t c = 0; c < nc; ++c)
        for (int32_t n = 0; n < nnom; ++n)
          tab[static_cast<size_t>(c) * nnom + n] = at(c0 + c, s->nominal[n]) - at(c0, s->nominal[n]);
      dd_plan *p = nullptr;
      st = dd_plan_create_from_delays(&p, nc, nnom, tab.data(), in_dtype, device);
      if (st != DD_OK) break;
      s->step1.push_back(p);
      int32_t m = 0;
      dd_plan_max_delay(p, &m);
      s->shift1.push_back(m);
      s->D1 = std::max(s->D1, m);
    }
    // step 2: group g, delays T[c_s][d] over the subbands
    for (int32_t g = 0; st == DD_OK && g < s->ngroups; ++g) {
      const int32_t g0 = g * dms_per_group, gn = std::min(dms_per_group, ndm - g0);
      std::vector<int32_t> tab(static_cast<size_t>(s->nsub) * gn);
      for (int32_t k = 0; k < s->nsub; ++k)
        for (int32_t d = 0; d < gn; ++d)
          tab[static_cast<size_t>(k) * gn + d] = at(s->first[k], g0 + d);
      dd_plan *p = nullptr;
      st = dd_plan_create_from_delays(&p, s->nsub, gn, tab.data(), DD_F32, device);
      if (st != DD_OK) break;
      s->step2.push_back(p);
      int32_t m = 0;
      dd_plan_max_delay(p, &m);
      s->shift2.push_back(m);
      s->D2 = std::max(s->D2, m);
    }
  } catch (...) {
    st = DD_ERR_OOM;
  }
  if (st != DD_OK) {
    destroy(s);
    return st;
  }
  *out = s;
  return DD_OK;
}

extern "C" int dd_subband_destroy(dd_subband *s) {
  if (s) destroy(s);
  return DD_OK;
}

extern "C" int dd_subband_max_delay(const dd_subband *s, int32_t *maxshift) {
  if (!s || !maxshift) return DD_ERR_ARG;
  *maxshift = s->D1 + s->D2;
  return DD_OK;
}

extern "C" int dd_subband_nominal(const dd_subband *s, int32_t *nominal, int32_t *ngroups) {
  if (!s) return DD_ERR_ARG;
  if (ngroups) *ngroups = s->ngroups;
  if (nominal) std::copy(s->nominal.begin(), s->nominal.end(), nominal);
  return DD_OK;
}

extern "C" int dd_subband_launch_count(const dd_subband *s, int64_t *launches) {
  if (!s || !launches) return DD_ERR_ARG;
  int64_t n = s->launches;
  for (dd_plan *p : s->step1) {
    int64_t k = 0;
    dd_plan_launch_count(p, &k);
    n += k;
  }
  for (dd_plan *p : s->step2) {
    int64_t k = 0;
    dd_plan_launch_count(p, &k);
    n += k;
  }
  *launches = n;
  return DD_OK;
}

extern "C" int dd_subband_execute(dd_subband *s, const void *block, int64_t nsamp_in,
                                  int64_t pitch_elems, void *out, void *stream) {
  if (!s || !block || !out) return DD_ERR_ARG;
  const int64_t maxshift = static_cast<int64_t>(s->D1) + s->D2;
  if (nsamp_in <= maxshift || pitch_elems < nsamp_in) return DD_ERR_SIZE;
  const int64_t nsamp_out = nsamp_in - maxshift;
  if (nsamp_out > INT32_MAX) return DD_ERR_SIZE;
  const int64_t L1 = nsamp_in - s->D1;
  const int64_t L1pad = (L1 + 3) / 4 * 4;  // 16-byte float rows for the step-2 block
  const size_t need = static_cast<size_t>(s->ngroups) * s->nsub * L1pad * 4;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return DD_ERR_CUDA;
  if (cudaSetDevice(s->device) != cudaSuccess) return DD_ERR_CUDA;
  struct Restore {
    int dev;
    ~Restore() { cudaSetDevice(dev); }
  } restore{prev};
  if (need > s->sb_bytes) {
    cudaDeviceSynchronize();  // the old workspace may still be in use
    if (s->d_sb) cudaFree(s->d_sb);
    s->d_sb = nullptr;
    s->sb_bytes = 0;
    if (cudaMalloc(&s->d_sb, need) != cudaSuccess) return DD_ERR_OOM;
    s->sb_bytes = need;
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned char *blk = static_cast<const unsigned char *>(block);
  const int eb = elem_bytes(s->dtype);
  int32_t *sb = static_cast<int32_t *>(s->d_sb);
  // step 1: subband k at the nominal trials, rows (n, k) of SB
  for (int32_t k = 0; k < s->nsub; ++k) {
    const void *bk = blk + static_cast<size_t>(s->first[k]) * pitch_elems * eb;
    const int r = dd_execute_pitched(s->step1[k], bk, L1 + s->shift1[k], pitch_elems,
                                     sb + k * L1pad, static_cast<int64_t>(s->nsub) * L1pad, stream);
    if (r != DD_OK) return r;
  }
  if (s->dtype == DD_U8) {
    const int64_t rows = static_cast<int64_t>(s->ngroups) * s->nsub;
    to_float_rows<<<conv_grid(rows * L1), kConvThreads, 0, st>>>(sb, rows, L1, L1pad);
    ++s->launches;
  }
  // step 2: group g from its nominal's SB block, rows g0 .. of out
  const float *sbf = reinterpret_cast<const float *>(sb);
  for (int32_t g = 0; g < s->ngroups; ++g) {
    const float *bg = sbf + static_cast<size_t>(g) * s->nsub * L1pad;
    float *og = static_cast<float *>(out) + static_cast<size_t>(g) * s->dpg * nsamp_out;
    const int r = dd_execute_pitched(s->step2[g], bg, nsamp_out + s->shift2[g], L1pad, og,
                                     nsamp_out, stream);
    if (r != DD_OK) return r;
  }
  if (s->dtype == DD_U8) {
    const int64_t n = static_cast<int64_t>(s->ndm) * nsamp_out;
    to_int_rows<<<conv_grid(n), kConvThreads, 0, st>>>(static_cast<float *>(out), n);
    ++s->launches;
  }
  return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
}
