// dd_binned.cu -- time-binned dedispersion past the diagonal DM (Sec. 2.1.1,
// the downfactoring procedure of Sec. 2.1.2): one dd_plan per downfactor
// (its consecutive trials, sampling time f t_samp), run on the block binned
// by f.  The binned series are built level by level on the device (pairs of
// adjacent samples summed; u8 sums are exact integers held in float), the
// full-rate trials run on the block itself, and for u8 input the float rows
// of the binned trials are turned back into int32 in place (exact).  In the
// 8-bit mode the levels hold rounded pair means as bytes instead, and every
// downfactor runs through the 8-bit kernel.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <vector>

#include "dd.h"
#include "dd_binned.h"
#include "dd_internal.h"

namespace {

constexpr double kDispersion = 4.148808e3;  // MHz^2 pc^-1 cm^3 s (Sec. 1.2.1)
constexpr int kMaxLevels = 7;                // downfactors 1 .. 64
constexpr int kThreads = 256;

struct Range {
  int32_t factor = 1, d0 = 0, n = 0;  // trials d0 .. d0 + n - 1
  dd_plan *plan = nullptr;
  int32_t maxshift = 0;
};

}  // namespace

struct dd_binned {
  int32_t device = 0, nchan = 0, ndm = 0, dtype = 0, max_factor = 1, mode = DD_BIN_SUM;
  double dm_diag = 0.0;
  std::vector<int32_t> factor;  // per trial
  std::vector<Range> ranges;    // ascending factor
  void *d_bins = nullptr;       // binned series, levels 1.. back to back (float, or u8)
  size_t bins_bytes = 0;
  int64_t launches = 0;
};

namespace {

template <typename T> __device__ __forceinline__ float to_f(T x);
template <> __device__ __forceinline__ float to_f<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f<__half>(__half x) { return __half2float(x); }

// out[c][t] = in[c][2t] + in[c][2t+1] for t < n_out (u8: exact integer sum).
template <typename T>
__global__ void bin_pairs(const T *__restrict__ in, int64_t in_pitch, int32_t nchan, int64_t n_out,
                          float *__restrict__ out, int64_t out_pitch) {
  const int64_t n = static_cast<int64_t>(nchan) * n_out;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = i / n_out, t = i % n_out;
    const T *p = in + c * in_pitch + 2 * t;
    float v;
    if constexpr (sizeof(T) == 1) {
      v = static_cast<float>(static_cast<int32_t>(p[0]) + static_cast<int32_t>(p[1]));
    } else {
      v = to_f<T>(p[0]) + to_f<T>(p[1]);
    }
    out[c * out_pitch + t] = v;
  }
}

// out[c][t] = (in[c][2t] + in[c][2t+1] + 1) >> 1 for t < n_out: the pair's
// mean rounded half up, which stays in 0..255.
__global__ void bin_mean_u8(const uint8_t *__restrict__ in, int64_t in_pitch, int32_t nchan,
                            int64_t n_out, uint8_t *__restrict__ out, int64_t out_pitch) {
  for (int64_t c = blockIdx.y; c < nchan; c += gridDim.y) {
    const uint8_t *p = in + c * in_pitch;
    uint8_t *q = out + c * out_pitch;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n_out;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      const uint32_t a = p[2 * t], b = p[2 * t + 1];
      q[t] = static_cast<uint8_t>((a + b + 1u) >> 1);
    }
  }
}

// The same with 16-byte loads: thread v of row c makes outputs 8v .. 8v+7
// from input bytes 16v .. 16v+15; thread nvec makes the row's last n_out % 8
// outputs one by one.  Rows of `in` and `out` start on 16-byte boundaries.
// In each 32-bit word the even and odd bytes are added in 16-bit lanes
// (at most 511), halved, and the two results of a pair of words packed.
__global__ void bin_mean_u8_vec(const uint8_t *__restrict__ in, int64_t in_pitch, int32_t nchan,
                                int64_t n_out, uint8_t *__restrict__ out, int64_t out_pitch) {
  const int64_t nvec = n_out / 8;
  for (int64_t c = blockIdx.y; c < nchan; c += gridDim.y) {
    const uint8_t *p = in + c * in_pitch;
    uint8_t *q = out + c * out_pitch;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v <= nvec;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      if (v < nvec) {
        const uint4 w = *reinterpret_cast<const uint4 *>(p + 16 * v);
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
        uint32_t m[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          m[i] = (((x[i] & 0x00ff00ffu) + ((x[i] >> 8) & 0x00ff00ffu) + 0x00010001u) >> 1) &
                 0x00ff00ffu;
        uint2 r;
        r.x = __byte_perm(m[0], m[1], 0x6420);
        r.y = __byte_perm(m[2], m[3], 0x6420);
        *reinterpret_cast<uint2 *>(q + 8 * v) = r;
      } else {
        for (int64_t t = 8 * nvec; t < n_out; ++t) {
          const uint32_t a = p[2 * t], b = p[2 * t + 1];
          q[t] = static_cast<uint8_t>((a + b + 1u) >> 1);
        }
      }
    }
  }
}

// In-place float -> int32 over rows [nrows][pitch] (first ncols of each);
// the values are integers below 2^24.
__global__ void rows_to_int(float *p, int64_t nrows, int64_t ncols, int64_t pitch) {
  const int64_t n = nrows * ncols;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float *q = p + (i / ncols) * pitch + i % ncols;
    *reinterpret_cast<int32_t *>(q) = __float2int_rn(*q);
  }
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return static_cast<unsigned>(std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 32));
}

int level_of(int32_t f) {
  int k = 0;
  while ((1 << k) < f) ++k;
  return k;
}

// Length and 16-byte-padded pitch (in elements of esize bytes) of binning
// level k (k >= 1).
inline int64_t level_len(int64_t nsamp_in, int k) { return nsamp_in >> k; }
inline int64_t level_pitch(int64_t nsamp_in, int k, int esize) {
  const int64_t per = 16 / esize;
  return (level_len(nsamp_in, k) + per - 1) / per * per;
}

void destroy(dd_binned *b) {
  for (Range &r : b->ranges) dd_plan_destroy(r.plan);
  if (b->d_bins) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaFree(b->d_bins);
    cudaSetDevice(prev);
  }
  delete b;
}

}  // namespace

extern "C" int dd_binned_create(dd_binned **out, int32_t nchan, double f_top_mhz,
                                double chan_width_mhz, double t_samp_s, const double *dm_list,
                                int32_t ndm, int32_t in_dtype, int32_t max_factor,
                                int32_t mode, int32_t device) {
  if (!out) return DD_ERR_ARG;
  *out = nullptr;
  if (in_dtype != DD_U8 && in_dtype != DD_F16 && in_dtype != DD_F32) return DD_ERR_DTYPE;
  if (mode != DD_BIN_SUM && mode != DD_BIN_MEAN_U8) return DD_ERR_ARG;
  if (mode == DD_BIN_MEAN_U8 && in_dtype != DD_U8) return DD_ERR_DTYPE;
  if (nchan < 1 || ndm < 1 || !dm_list || device < 0 || !(chan_width_mhz > 0) ||
      !(t_samp_s > 0))
    return DD_ERR_ARG;
  if (max_factor < 1 || max_factor > (1 << (kMaxLevels - 1)) || (max_factor & (max_factor - 1)))
    return DD_ERR_ARG;
  for (int32_t d = 1; d < ndm; ++d)
    if (!(dm_list[d] >= dm_list[d - 1])) return DD_ERR_ARG;
  if (mode == DD_BIN_SUM && in_dtype == DD_U8 &&
      static_cast<int64_t>(nchan) * 255 * max_factor >= (1 << 24))
    return DD_ERR_RANGE;
  dd_binned *b = new (std::nothrow) dd_binned();
  if (!b) return DD_ERR_OOM;
  b->device = device;
  b->nchan = nchan;
  b->ndm = ndm;
  b->dtype = in_dtype;
  b->max_factor = max_factor;
  b->mode = mode;
  const double f_bot = f_top_mhz - (nchan - 1) * chan_width_mhz;
  b->dm_diag = t_samp_s * (f_bot * f_bot * f_bot) / (2.0 * kDispersion * chan_width_mhz);
  int st = DD_OK;
  try {
    b->factor.resize(ndm);
    for (int32_t d = 0; d < ndm; ++d) {
      int32_t k = 1;
      while (2 * k <= max_factor && dm_list[d] >= 2 * k * b->dm_diag) k *= 2;
      b->factor[d] = k;
    }
    for (int32_t d = 0; d < ndm;) {  // factors are non-decreasing along the list
      Range r;
      r.factor = b->factor[d];
      r.d0 = d;
      while (d < ndm && b->factor[d] == r.factor) ++d;
      r.n = d - r.d0;
      b->ranges.push_back(r);
    }
    for (Range &r : b->ranges) {
      const int32_t level_dtype = mode == DD_BIN_MEAN_U8 ? DD_U8 : DD_F32;
      st = dd_plan_create(&r.plan, nchan, f_top_mhz, chan_width_mhz, t_samp_s * r.factor,
                          dm_list + r.d0, r.n, r.factor == 1 ? in_dtype : level_dtype, device);
      if (st != DD_OK) break;
      dd_plan_max_delay(r.plan, &r.maxshift);
    }
  } catch (...) {
    st = DD_ERR_OOM;
  }
  if (st != DD_OK) {
    destroy(b);
    return st;
  }
  *out = b;
  return DD_OK;
}

extern "C" int dd_binned_destroy(dd_binned *b) {
  if (b) destroy(b);
  return DD_OK;
}

extern "C" int dd_binned_diagonal_dm(const dd_binned *b, double *dm_diag) {
  if (!b || !dm_diag) return DD_ERR_ARG;
  *dm_diag = b->dm_diag;
  return DD_OK;
}

extern "C" int dd_binned_rows(const dd_binned *b, int64_t nsamp_in, int32_t *factor,
                              int64_t *nsamp_out) {
  if (!b) return DD_ERR_ARG;
  for (const Range &r : b->ranges) {
    const int64_t n = nsamp_in / r.factor - r.maxshift;
    if (nsamp_out && n < 1) return DD_ERR_SIZE;
    for (int32_t d = r.d0; d < r.d0 + r.n; ++d) {
      if (factor) factor[d] = r.factor;
      if (nsamp_out) nsamp_out[d] = n;
    }
  }
  return DD_OK;
}

extern "C" int dd_binned_launch_count(const dd_binned *b, int64_t *launches) {
  if (!b || !launches) return DD_ERR_ARG;
  int64_t n = b->launches;
  for (const Range &r : b->ranges) {
    int64_t k = 0;
    dd_plan_launch_count(r.plan, &k);
    n += k;
  }
  *launches = n;
  return DD_OK;
}

extern "C" int dd_binned_sync(dd_binned *b, void *stream) {
  if (!b) return DD_ERR_ARG;
  int result = DD_OK;
  for (const Range &r : b->ranges) {
    const int st = dd_sync(r.plan, stream);
    if (st != DD_OK && result == DD_OK) result = st;
  }
  return result;
}

extern "C" int dd_binned_execute(dd_binned *b, const void *block, int64_t nsamp_in,
                                 int64_t pitch_elems, void *out, int64_t out_pitch, void *stream) {
  if (!b || !block || !out) return DD_ERR_ARG;
  if (pitch_elems < nsamp_in) return DD_ERR_SIZE;
  int64_t longest = 0;
  for (const Range &r : b->ranges) {
    const int64_t n = nsamp_in / r.factor - r.maxshift;
    if (n < 1) return DD_ERR_SIZE;
    longest = std::max(longest, n);
  }
  if (out_pitch < longest) return DD_ERR_ARG;
  const bool mean8 = b->mode == DD_BIN_MEAN_U8;
  const int es = mean8 ? 1 : 4;  // bytes per binned sample
  const int top = level_of(b->ranges.back().factor);
  // workspace: levels 1 .. top back to back, each a multiple of 16 bytes
  size_t need = 0;
  for (int k = 1; k <= top; ++k)
    need += static_cast<size_t>(b->nchan) * level_pitch(nsamp_in, k, es) * es;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(b->device) != cudaSuccess)
    return DD_ERR_CUDA;
  struct Restore {
    int dev;
    ~Restore() { cudaSetDevice(dev); }
  } restore{prev};
  if (need > b->bins_bytes) {
    cudaDeviceSynchronize();  // the old workspace may still be in use
    if (b->d_bins) cudaFree(b->d_bins);
    b->d_bins = nullptr;
    b->bins_bytes = 0;
    if (cudaMalloc(&b->d_bins, need) != cudaSuccess) return DD_ERR_OOM;
    b->bins_bytes = need;
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  char *level[kMaxLevels] = {};
  {
    char *p = static_cast<char *>(b->d_bins);
    for (int k = 1; k <= top; ++k) {
      level[k] = p;
      p += static_cast<size_t>(b->nchan) * level_pitch(nsamp_in, k, es) * es;
    }
  }
  // binned series, level by level
  for (int k = 1; k <= top; ++k) {
    const int64_t n = level_len(nsamp_in, k);
    const int64_t np = level_pitch(nsamp_in, k, es);
    if (mean8) {
      const uint8_t *src = k > 1 ? reinterpret_cast<const uint8_t *>(level[k - 1])
                                 : static_cast<const uint8_t *>(block);
      const int64_t sp = k > 1 ? level_pitch(nsamp_in, k - 1, es) : pitch_elems;
      uint8_t *dst = reinterpret_cast<uint8_t *>(level[k]);
      const unsigned gy = static_cast<unsigned>(std::min<int32_t>(b->nchan, 65535));
      if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (sp & 15) == 0) {
        const int64_t nvec = n / 8 + 1;  // the last thread of a row takes the ragged end
        const dim3 g(static_cast<unsigned>(std::min<int64_t>((nvec + kThreads - 1) / kThreads, 64)),
                     gy);
        bin_mean_u8_vec<<<g, kThreads, 0, st>>>(src, sp, b->nchan, n, dst, np);
      } else {
        const dim3 g(static_cast<unsigned>(std::min<int64_t>((n + kThreads - 1) / kThreads, 64)),
                     gy);
        bin_mean_u8<<<g, kThreads, 0, st>>>(src, sp, b->nchan, n, dst, np);
      }
    } else {
      float *dst = reinterpret_cast<float *>(level[k]);
      const unsigned g = grid_for(static_cast<int64_t>(b->nchan) * n);
      if (k > 1) {
        bin_pairs<float><<<g, kThreads, 0, st>>>(reinterpret_cast<const float *>(level[k - 1]),
                                                 level_pitch(nsamp_in, k - 1, es), b->nchan, n,
                                                 dst, np);
      } else if (b->dtype == DD_U8) {
        bin_pairs<uint8_t><<<g, kThreads, 0, st>>>(static_cast<const uint8_t *>(block),
                                                   pitch_elems, b->nchan, n, dst, np);
      } else if (b->dtype == DD_F16) {
        bin_pairs<__half><<<g, kThreads, 0, st>>>(static_cast<const __half *>(block),
                                                  pitch_elems, b->nchan, n, dst, np);
      } else {
        bin_pairs<float><<<g, kThreads, 0, st>>>(static_cast<const float *>(block), pitch_elems,
                                                 b->nchan, n, dst, np);
      }
    }
    ++b->launches;
  }
  // every downfactor's plan at once: the staged 8-bit ones share persistent
  // launches (all of them in the 8-bit mode)
  const int nr = static_cast<int>(b->ranges.size());
  std::vector<dd_plan *> plans(nr);
  std::vector<const void *> src(nr);
  std::vector<void *> dst(nr);
  std::vector<int64_t> len(nr), pitch(nr), opitch(nr, out_pitch);
  for (int i = 0; i < nr; ++i) {
    const Range &r = b->ranges[i];
    plans[i] = r.plan;
    dst[i] = static_cast<char *>(out) + static_cast<size_t>(r.d0) * out_pitch * 4;
    if (r.factor == 1) {
      src[i] = block, len[i] = nsamp_in, pitch[i] = pitch_elems;
    } else {
      const int k = level_of(r.factor);
      src[i] = level[k], len[i] = level_len(nsamp_in, k), pitch[i] = level_pitch(nsamp_in, k, es);
    }
  }
  const int rc = execute_plans_pitched(plans.data(), nr, src.data(), len.data(), pitch.data(),
                                       dst.data(), opitch.data(), stream);
  if (rc != DD_OK) return rc;
  if (b->dtype == DD_U8 && !mean8) {
    for (int i = 0; i < nr; ++i) {
      const Range &r = b->ranges[i];
      if (r.factor == 1) continue;
      const int64_t n_out = nsamp_in / r.factor - r.maxshift;
      rows_to_int<<<grid_for(static_cast<int64_t>(r.n) * n_out), kThreads, 0, st>>>(
          static_cast<float *>(dst[i]), r.n, n_out, out_pitch);
      ++b->launches;
    }
  }
  return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
}
