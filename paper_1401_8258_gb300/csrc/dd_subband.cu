// dd_subband.cu -- subband dedispersion (Sec. 2.1.3): two brute-force
// passes over delay tables derived from the brute-force table, each one
// launch of a grouped kernel:
//   step 1: groups = subbands, channels = the subband's channels, trials =
//           the nominal trials; rows written interleaved as SB[n][s][t];
//   step 2: groups = DM groups, channels = the subbands (SB[n(g)] as a
//           block), trials = the group's trials.
// The grouped kernels stage, per CTA (group, 16 trials, time tile), each
// channel's input window in shared memory and add from there.  u8 input
// (chans_per_subband x 255 <= 65535): both steps on packed pairs of 16-bit
// sums, SB kept as uint16, output int32 (exact).  Float input, or u8 with
// wider subbands: step 1 stores float (exact for u8 below 2^24), step 2 adds
// the floats (u8: integer-valued, exact) and stores float or int32.
#include <cuda_fp16.h>
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
  // stacked tables for the grouped kernel: step 1 [nsub][cps][nnom] (rows
  // past a narrow last subband unused), step 2 [ngroups][nsub][dpg] (trials
  // past a short last group repeat its last trial)
  int32_t *d_tab1 = nullptr, *d_tab2 = nullptr;
  int32_t span1 = 0, span2 = 0;  // largest delay spread over kGroupTrials trials of a channel
  void *d_sb = nullptr;  // step-1 series [ngroups][nsub][L1pad], 4-byte elements
  size_t sb_bytes = 0;
  int64_t launches = 0;
};

namespace {

constexpr int kGroupThreads = 256;
constexpr int kGroupTrials = 16;   // trials per CTA (one accumulator each per thread)
constexpr int kGroupTile = 512;    // output samples per CTA (two per thread)
static_assert(kGroupTile == 2 * kGroupThreads, "a thread owns samples t and t + kGroupThreads");

template <typename T> struct GroupIn;
template <> struct GroupIn<uint8_t> {
  using acc = int32_t;
  static __device__ __forceinline__ int32_t add(int32_t a, uint8_t x) { return a + x; }
};
template <> struct GroupIn<__half> {
  using acc = float;
  static __device__ __forceinline__ float add(float a, __half x) { return a + __half2float(x); }
};
template <> struct GroupIn<float> {
  using acc = float;
  static __device__ __forceinline__ float add(float a, float x) { return a + x; }
};

template <typename A, typename O> __device__ __forceinline__ O store_as(A v);
template <> __device__ __forceinline__ float store_as<int32_t, float>(int32_t v) {
  return static_cast<float>(v);  // exact below 2^24
}
template <> __device__ __forceinline__ float store_as<float, float>(float v) { return v; }
template <> __device__ __forceinline__ int32_t store_as<float, int32_t>(float v) {
  return __float2int_rn(v);  // integer-valued sums below 2^24
}

// Grouped brute-force sum: for group g, trial j < ntr and t < nsamp_out,
//   out[g * og + j * oj + t] = sum_{c < nch(g)} in[g * ig + c * pitch + t + tab[g][c][j]]
// tab: [ngroups][tab_ch][ntr]; nch(g) = min(tab_ch, nch_total - g * tab_ch)
// (the last group of channels may be narrower); trials j >= ntr_g(g) are not
// stored.  Input samples at or past n_valid in a row are never read (they
// could only reach outputs t >= nsamp_out, which are not stored).  Grid:
// (time tiles, ceil(ntr / 16), ngroups).  Dynamic shared memory:
// min(tab_ch, 64) rows of kGroupTile + span elements.
template <typename TI, typename TO>
__global__ void __launch_bounds__(kGroupThreads, 2)  // two CTAs per SM: at most 128 registers
dd_grouped(const TI *__restrict__ in, int64_t pitch, int64_t ig, const int32_t *__restrict__ tab,
           int tab_ch, int nch_total, int ntr, int ntr_last, int span, int64_t n_valid,
           TO *__restrict__ out, int64_t og, int64_t oj, int64_t nsamp_out) {
  using A = typename GroupIn<TI>::acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TI *win = reinterpret_cast<TI *>(smem_raw);
  __shared__ int32_t s_del[64][kGroupTrials];  // delay relative to the window start
  __shared__ int32_t s_lo[64];
  const int g = blockIdx.z;
  const int j0 = blockIdx.y * kGroupTrials;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kGroupTile;
  const int nch = min(tab_ch, nch_total - g * tab_ch);
  const int ntr_g = g == gridDim.z - 1 ? ntr_last : ntr;
  const int W = kGroupTile + span;
  const TI *x = in + g * ig;
  const int32_t *tg = tab + static_cast<int64_t>(g) * tab_ch * ntr;
  A acc0[kGroupTrials], acc1[kGroupTrials];
#pragma unroll
  for (int j = 0; j < kGroupTrials; ++j) acc0[j] = acc1[j] = A(0);
  for (int c0 = 0; c0 < nch; c0 += 64) {
    const int nc = min(64, nch - c0);
    __syncthreads();
    if (threadIdx.x < nc) {  // window start of each channel = its smallest delay here
      const int c = c0 + threadIdx.x;
      int lo = INT32_MAX;
      for (int j = 0; j < kGroupTrials; ++j) {
        const int jj = min(j0 + j, ntr_g - 1);
        lo = min(lo, tg[static_cast<int64_t>(c) * ntr + jj]);
      }
      s_lo[threadIdx.x] = lo;
      for (int j = 0; j < kGroupTrials; ++j) {
        const int jj = min(j0 + j, ntr_g - 1);
        s_del[threadIdx.x][j] = tg[static_cast<int64_t>(c) * ntr + jj] - lo;
      }
    }
    __syncthreads();
    // windows: channel c, samples t0 + lo_c .. t0 + lo_c + W - 1, in blocks
    // of 8 channels; a thread issues the loads of a block (8 channels x 3
    // samples in flight) before adding the previous block from shared memory,
    // and stores them after, so each block's loads overlap the adds of the
    // one before; any rest of a wide window is copied directly
    constexpr int kUnroll = 8, kReach = 3;
    TI v[kUnroll][kReach];
    auto load_block = [&](int cb) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int r = 0; r < kReach; ++r) {
          const int c = cb + u, k = threadIdx.x + r * kGroupThreads;
          const int64_t tt = t0 + (c < nc ? s_lo[c] : 0) + k;
          v[u][r] = (c < nc && k < W && tt < n_valid)
                        ? x[static_cast<int64_t>(c0 + c) * pitch + tt] : TI(0);
        }
      }
    };
    auto store_block = [&](int cb) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int r = 0; r < kReach; ++r) {
          const int k = threadIdx.x + r * kGroupThreads;
          if (cb + u < nc && k < W) win[(cb + u) * W + k] = v[u][r];
        }
      }
      for (int u = 0; u < kUnroll && cb + u < nc; ++u) {
        const int c = cb + u;
        for (int k = threadIdx.x + kReach * kGroupThreads; k < W; k += kGroupThreads) {
          const int64_t tt = t0 + s_lo[c] + k;
          win[c * W + k] = tt < n_valid ? x[static_cast<int64_t>(c0 + c) * pitch + tt] : TI(0);
        }
      }
    };
    load_block(0);
    store_block(0);
    for (int cb = 0; cb < nc; cb += kUnroll) {
      const bool more = cb + kUnroll < nc;
      if (more) load_block(cb + kUnroll);  // in flight during the adds below
      __syncthreads();                     // block cb stored by every thread
      const int ce = min(cb + kUnroll, nc);
      for (int c = cb; c < ce; ++c) {
        const TI *w = win + c * W + threadIdx.x;
#pragma unroll
        for (int j = 0; j < kGroupTrials; ++j) {
          const int dl = s_del[c][j];
          acc0[j] = GroupIn<TI>::add(acc0[j], w[dl]);
          acc1[j] = GroupIn<TI>::add(acc1[j], w[dl + kGroupThreads]);
        }
      }
      if (more) store_block(cb + kUnroll);  // read only after the next barrier
    }
  }
  const int64_t ta = t0 + threadIdx.x, tb = ta + kGroupThreads;
#pragma unroll
  for (int j = 0; j < kGroupTrials; ++j) {
    if (j0 + j >= ntr_g) break;
    TO *o = out + g * og + static_cast<int64_t>(j0 + j) * oj;
    if (ta < nsamp_out) o[ta] = store_as<A, TO>(acc0[j]);
    if (tb < nsamp_out) o[tb] = store_as<A, TO>(acc1[j]);
  }
}

constexpr size_t kGroupSmemMax = 200 * 1024;

inline size_t grouped_smem(int tab_ch, int span, size_t esize) {
  return static_cast<size_t>(std::min(tab_ch, 64)) * (kGroupTile + span) * esize;
}

template <typename TI, typename TO>
cudaError_t launch_grouped(const TI *in, int64_t pitch, int64_t ig, const int32_t *tab, int tab_ch,
                           int nch_total, int ngroups, int ntr, int ntr_last, int span,
                           int64_t n_valid, TO *out, int64_t og, int64_t oj, int64_t nsamp_out,
                           cudaStream_t s) {
  const size_t smem = grouped_smem(tab_ch, span, sizeof(TI));
  cudaError_t e = cudaFuncSetAttribute(dd_grouped<TI, TO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>((nsamp_out + kGroupTile - 1) / kGroupTile),
                  static_cast<unsigned>((ntr + kGroupTrials - 1) / kGroupTrials),
                  static_cast<unsigned>(ngroups));
  dd_grouped<TI, TO><<<grid, kGroupThreads, smem, s>>>(in, pitch, ig, tab, tab_ch, nch_total, ntr,
                                                       ntr_last, span, n_valid, out, og, oj,
                                                       nsamp_out);
  return cudaGetLastError();
}

// The grouped sum for integer input (u8 blocks, u16 subband series) with
// packed pairs: each channel's window is staged as pair words, word i
// holding the window's samples i and i + kGroupThreads in its low and high
// 16 bits, so one shared load and one add serve both outputs (t and t + 256)
// of a thread for one trial.  The 16-bit halves are drained into 32-bit sums
// every `drain` channels (drain x the largest input sample <= 65535).  Same
// grid, tables, n_valid rule and stores as dd_grouped; dynamic shared memory
// min(tab_ch, 64) rows of kGroupThreads + span words.
template <typename TI, typename TO>
__global__ void __launch_bounds__(kGroupThreads, 2)
dd_grouped_pairs(const TI *__restrict__ in, int64_t pitch, int64_t ig,
                 const int32_t *__restrict__ tab, int tab_ch, int nch_total, int ntr, int ntr_last,
                 int span, int64_t n_valid, int drain, TO *__restrict__ out, int64_t og,
                 int64_t oj, int64_t nsamp_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *win = reinterpret_cast<uint32_t *>(smem_raw);
  __shared__ int32_t s_del[64][kGroupTrials];  // delay relative to the window start
  __shared__ int32_t s_lo[64];
  const int g = blockIdx.z;
  const int j0 = blockIdx.y * kGroupTrials;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kGroupTile;
  const int nch = min(tab_ch, nch_total - g * tab_ch);
  const int ntr_g = g == gridDim.z - 1 ? ntr_last : ntr;
  const int P = kGroupThreads + span;  // pair words per channel
  const TI *x = in + g * ig;
  const int32_t *tg = tab + static_cast<int64_t>(g) * tab_ch * ntr;
  uint32_t pk[kGroupTrials], lo32[kGroupTrials], hi32[kGroupTrials];
#pragma unroll
  for (int j = 0; j < kGroupTrials; ++j) pk[j] = lo32[j] = hi32[j] = 0u;
  int since = 0;  // channels added into pk since the last drain
  for (int c0 = 0; c0 < nch; c0 += 64) {
    const int nc = min(64, nch - c0);
    __syncthreads();
    if (threadIdx.x < nc) {  // window start of each channel = its smallest delay here
      const int c = c0 + threadIdx.x;
      int lo = INT32_MAX;
      for (int j = 0; j < kGroupTrials; ++j) {
        const int jj = min(j0 + j, ntr_g - 1);
        lo = min(lo, tg[static_cast<int64_t>(c) * ntr + jj]);
      }
      s_lo[threadIdx.x] = lo;
      for (int j = 0; j < kGroupTrials; ++j) {
        const int jj = min(j0 + j, ntr_g - 1);
        s_del[threadIdx.x][j] = tg[static_cast<int64_t>(c) * ntr + jj] - lo;
      }
    }
    __syncthreads();
    // pair words in blocks of 4 channels: a block's 16 loads are issued
    // before the previous block is added from shared memory and stored after
    // it, so the loads overlap the adds; any rest of a wide window is copied
    // directly
    constexpr int kU = 4;
    uint32_t va[kU][2], vb[kU][2];
    auto load_block = [&](int cb) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int c = cb + u, i = threadIdx.x + r * kGroupThreads;
          const bool live = c < nc && i < P;
          const TI *row = x + static_cast<int64_t>(c0 + (live ? c : 0)) * pitch;
          const int64_t ta = t0 + (live ? s_lo[c] : 0) + i, tb = ta + kGroupThreads;
          va[u][r] = live && ta < n_valid ? static_cast<uint32_t>(row[ta]) : 0u;
          vb[u][r] = live && tb < n_valid ? static_cast<uint32_t>(row[tb]) : 0u;
        }
      }
    };
    auto store_block = [&](int cb) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int i = threadIdx.x + r * kGroupThreads;
          if (cb + u < nc && i < P) win[(cb + u) * P + i] = va[u][r] | (vb[u][r] << 16);
        }
      }
      for (int u = 0; u < kU && cb + u < nc; ++u) {
        const int c = cb + u;
        const TI *row = x + static_cast<int64_t>(c0 + c) * pitch;
        for (int i = threadIdx.x + 2 * kGroupThreads; i < P; i += kGroupThreads) {
          const int64_t ta = t0 + s_lo[c] + i, tb = ta + kGroupThreads;
          const uint32_t a = ta < n_valid ? static_cast<uint32_t>(row[ta]) : 0u;
          const uint32_t b = tb < n_valid ? static_cast<uint32_t>(row[tb]) : 0u;
          win[c * P + i] = a | (b << 16);
        }
      }
    };
    load_block(0);
    store_block(0);
    for (int cb = 0; cb < nc; cb += kU) {
      const bool more = cb + kU < nc;
      if (more) load_block(cb + kU);  // in flight during the adds below
      __syncthreads();                // block cb stored by every thread
      const int ce = min(cb + kU, nc);
      for (int c = cb; c < ce; ++c) {
        const uint32_t *w = win + c * P + threadIdx.x;
#pragma unroll
        for (int j = 0; j < kGroupTrials; ++j) pk[j] += w[s_del[c][j]];
        if (++since == drain) {
#pragma unroll
          for (int j = 0; j < kGroupTrials; ++j) {
            lo32[j] += pk[j] & 0xffffu;
            hi32[j] += pk[j] >> 16;
            pk[j] = 0u;
          }
          since = 0;
        }
      }
      if (more) store_block(cb + kU);  // read only after the next barrier
    }
  }
  const int64_t ta = t0 + threadIdx.x, tb = ta + kGroupThreads;
#pragma unroll
  for (int j = 0; j < kGroupTrials; ++j) {
    if (j0 + j >= ntr_g) break;
    TO *o = out + g * og + static_cast<int64_t>(j0 + j) * oj;
    if (ta < nsamp_out) o[ta] = static_cast<TO>(lo32[j] + (pk[j] & 0xffffu));
    if (tb < nsamp_out) o[tb] = static_cast<TO>(hi32[j] + (pk[j] >> 16));
  }
}

inline size_t pairs_smem(int tab_ch, int span) {
  return static_cast<size_t>(std::min(tab_ch, 64)) * (kGroupThreads + span) * 4;
}

template <typename TI, typename TO>
cudaError_t launch_pairs(const TI *in, int64_t pitch, int64_t ig, const int32_t *tab, int tab_ch,
                         int nch_total, int ngroups, int ntr, int ntr_last, int span,
                         int64_t n_valid, int drain, TO *out, int64_t og, int64_t oj,
                         int64_t nsamp_out, cudaStream_t s) {
  const size_t smem = pairs_smem(tab_ch, span);
  cudaError_t e = cudaFuncSetAttribute(dd_grouped_pairs<TI, TO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>((nsamp_out + kGroupTile - 1) / kGroupTile),
                  static_cast<unsigned>((ntr + kGroupTrials - 1) / kGroupTrials),
                  static_cast<unsigned>(ngroups));
  dd_grouped_pairs<TI, TO><<<grid, kGroupThreads, smem, s>>>(in, pitch, ig, tab, tab_ch,
                                                             nch_total, ntr, ntr_last, span,
                                                             n_valid, drain, out, og, oj,
                                                             nsamp_out);
  return cudaGetLastError();
}

// Largest spread (max - min) of a channel's delays over any kGroupTrials
// consecutive trials of a group (the chunks the kernel stages together).
int32_t chunk_span(const std::vector<int32_t> &tab, int ngroups, int tab_ch, int ntr,
                   const std::vector<int32_t> &ntr_of) {
  int32_t span = 0;
  for (int g = 0; g < ngroups; ++g)
    for (int c = 0; c < tab_ch; ++c)
      for (int j0 = 0; j0 < ntr_of[g]; j0 += kGroupTrials) {
        int32_t lo = INT32_MAX, hi = INT32_MIN;
        for (int j = j0; j < std::min(ntr_of[g], j0 + kGroupTrials); ++j) {
          const int32_t v = tab[(static_cast<size_t>(g) * tab_ch + c) * ntr + j];
          lo = std::min(lo, v);
          hi = std::max(hi, v);
        }
        span = std::max(span, hi - lo);
      }
  return span;
}

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
  if (s->d_sb || s->d_tab1 || s->d_tab2) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaFree(s->d_sb);
    cudaFree(s->d_tab1);
    cudaFree(s->d_tab2);
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
  // stacked tables and spans for the grouped kernel (one launch per step)
  if (st == DD_OK) {
    try {
      const int32_t nnom = s->ngroups;
      std::vector<int32_t> t1(static_cast<size_t>(s->nsub) * chans_per_subband * nnom, 0);
      for (int32_t k = 0; k < s->nsub; ++k) {
        const int32_t c0 = s->first[k], nc = std::min(chans_per_subband, nchan - c0);
        for (int32_t c = 0; c < nc; ++c)
          for (int32_t n = 0; n < nnom; ++n)
            t1[(static_cast<size_t>(k) * chans_per_subband + c) * nnom + n] =
                at(c0 + c, s->nominal[n]) - at(c0, s->nominal[n]);
      }
      std::vector<int32_t> t2(static_cast<size_t>(s->ngroups) * s->nsub * dms_per_group, 0);
      std::vector<int32_t> ntr2(s->ngroups);
      for (int32_t g = 0; g < s->ngroups; ++g) {
        const int32_t g0 = g * dms_per_group, gn = std::min(dms_per_group, ndm - g0);
        ntr2[g] = gn;
        for (int32_t k = 0; k < s->nsub; ++k)
          for (int32_t d = 0; d < dms_per_group; ++d)  // past a short group: its last trial
            t2[(static_cast<size_t>(g) * s->nsub + k) * dms_per_group + d] =
                at(s->first[k], g0 + std::min(d, gn - 1));
      }
      std::vector<int32_t> ntr1(s->nsub, nnom);
      s->span1 = chunk_span(t1, s->nsub, chans_per_subband, nnom, ntr1);
      s->span2 = chunk_span(t2, s->ngroups, s->nsub, dms_per_group, ntr2);
      int prev = 0;
      cudaGetDevice(&prev);
      cudaSetDevice(device);
      cudaError_t e = cudaMalloc(&s->d_tab1, t1.size() * sizeof(int32_t));
      if (e == cudaSuccess) e = cudaMalloc(&s->d_tab2, t2.size() * sizeof(int32_t));
      if (e == cudaSuccess)
        e = cudaMemcpy(s->d_tab1, t1.data(), t1.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(s->d_tab2, t2.data(), t2.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      cudaSetDevice(prev);
      if (e != cudaSuccess) st = DD_ERR_OOM;
    } catch (...) {
      st = DD_ERR_OOM;
    }
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

extern "C" int dd_subband_sync(dd_subband *s, void *stream) {
  if (!s) return DD_ERR_ARG;
  int result = DD_OK;
  for (dd_plan *p : s->step1) {
    const int st = dd_sync(p, stream);
    if (st != DD_OK && result == DD_OK) result = st;
  }
  for (dd_plan *p : s->step2) {
    const int st = dd_sync(p, stream);
    if (st != DD_OK && result == DD_OK) result = st;
  }
  return result;
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
  float *sbf = reinterpret_cast<float *>(sb);
  const int64_t ldsb = static_cast<int64_t>(s->nsub) * L1pad;  // SB row pitch per nominal
  const int last = s->ndm - (s->ngroups - 1) * s->dpg;
  const int64_t max_sb = static_cast<int64_t>(s->cps) * 255;  // largest step-1 sum (u8)
  if (s->dtype == DD_U8 && max_sb <= 65535 && pairs_smem(s->cps, s->span1) <= kGroupSmemMax &&
      pairs_smem(s->nsub, s->span2) <= kGroupSmemMax) {
    // u8: both steps on packed pairs, the step-1 series kept as uint16
    uint16_t *sb16 = static_cast<uint16_t *>(s->d_sb);
    const int64_t ig = static_cast<int64_t>(s->cps) * pitch_elems;
    cudaError_t e = launch_pairs(static_cast<const uint8_t *>(block), pitch_elems, ig, s->d_tab1,
                                 s->cps, s->nchan, s->nsub, s->ngroups, s->ngroups, s->span1,
                                 nsamp_in, 65535 / 255, sb16, L1pad, ldsb, L1, st);
    if (e == cudaSuccess) {
      const int64_t og = static_cast<int64_t>(s->dpg) * nsamp_out;
      e = launch_pairs(static_cast<const uint16_t *>(sb16), L1pad, ldsb, s->d_tab2, s->nsub,
                       s->nsub * s->ngroups, s->ngroups, s->dpg, last, s->span2, L1,
                       static_cast<int>(65535 / max_sb), static_cast<int32_t *>(out), og,
                       nsamp_out, nsamp_out, st);
    }
    s->launches += 2;
    return e == cudaSuccess ? DD_OK : DD_ERR_CUDA;
  }
  if (grouped_smem(s->cps, s->span1, eb) <= kGroupSmemMax &&
      grouped_smem(s->nsub, s->span2, 4) <= kGroupSmemMax) {
    cudaError_t e;
    // step 1: group = subband k, rows (n, k) of SB, float
    const int64_t ig = static_cast<int64_t>(s->cps) * pitch_elems;
    if (s->dtype == DD_U8)
      e = launch_grouped(static_cast<const uint8_t *>(block), pitch_elems, ig, s->d_tab1, s->cps,
                         s->nchan, s->nsub, s->ngroups, s->ngroups, s->span1, nsamp_in, sbf,
                         L1pad, ldsb, L1, st);
    else if (s->dtype == DD_F16)
      e = launch_grouped(static_cast<const __half *>(block), pitch_elems, ig, s->d_tab1, s->cps,
                         s->nchan, s->nsub, s->ngroups, s->ngroups, s->span1, nsamp_in, sbf,
                         L1pad, ldsb, L1, st);
    else
      e = launch_grouped(static_cast<const float *>(block), pitch_elems, ig, s->d_tab1, s->cps,
                         s->nchan, s->nsub, s->ngroups, s->ngroups, s->span1, nsamp_in, sbf,
                         L1pad, ldsb, L1, st);
    // step 2: group g reads SB[g] ([nsub][L1pad]), rows g * dpg + j of out
    if (e == cudaSuccess) {
      const int64_t og = static_cast<int64_t>(s->dpg) * nsamp_out;
      if (s->dtype == DD_U8)
        e = launch_grouped(static_cast<const float *>(sbf), L1pad, ldsb, s->d_tab2, s->nsub,
                           s->nsub * s->ngroups, s->ngroups, s->dpg, last, s->span2, L1,
                           static_cast<int32_t *>(out), og, nsamp_out, nsamp_out, st);
      else
        e = launch_grouped(static_cast<const float *>(sbf), L1pad, ldsb, s->d_tab2, s->nsub,
                           s->nsub * s->ngroups, s->ngroups, s->dpg, last, s->span2, L1,
                           static_cast<float *>(out), og, nsamp_out, nsamp_out, st);
    }
    s->launches += 2;
    return e == cudaSuccess ? DD_OK : DD_ERR_CUDA;
  }
  // windows too wide for shared memory: one plan per subband and per group
  for (int32_t k = 0; k < s->nsub; ++k) {
    const void *bk = blk + static_cast<size_t>(s->first[k]) * pitch_elems * eb;
    const int r = dd_execute_pitched(s->step1[k], bk, L1 + s->shift1[k], pitch_elems,
                                     sb + k * L1pad, ldsb, stream);
    if (r != DD_OK) return r;
  }
  if (s->dtype == DD_U8) {
    const int64_t rows = static_cast<int64_t>(s->ngroups) * s->nsub;
    to_float_rows<<<conv_grid(rows * L1), kConvThreads, 0, st>>>(sb, rows, L1, L1pad);
    ++s->launches;
  }
  for (int32_t g = 0; g < s->ngroups; ++g) {
    const float *bg = sbf + static_cast<size_t>(g) * ldsb;
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
