// dd_detect.cu -- per-DM-trial normalisation and n-sigma candidate extraction
// (Sec. 3.5 normalisation, Sec. 3.6 thresholding into (DM, time, intensity)
// triplets), moved from the host onto the GPU.
//
// Passes over D[ndm][n]:
//   1. dd_stats_*      one CTA per DM row: exact integer sums (int32 rows) or
//                      shifted double sums (float rows), then mean and rms;
//                      and the row's candidate threshold (see dd_row_stats);
//   2. dd_count        per (row, 4096-sample chunk): number of samples with
//                      snr > nsigma, tested as D >= threshold;
//   3. dd_scan         exclusive prefix over the chunk counts in (row, chunk)
//                      order, plus the total;
//   4. dd_write        chunks with a non-zero count write their candidates
//                      in time order at their prefix offset.
// The candidate list is therefore ordered by (dm_idx, t) and independent of
// scheduling.  The predicate is evaluated identically in passes 2 and 4.
//
// Tiled variant (after the staged u8 kernel, which already added each row's
// exact sums and recorded the largest output of each 512-sample time tile):
//   1. dd_tile_count   one CTA per row: mean, rms and threshold from the sums
//                      (the same finaliser as dd_stats_i32); counts the
//                      candidates of the tiles whose maximum reaches the
//                      threshold -- the only tiles that can hold one -- and
//                      the row total;
//   2. dd_scan         exclusive prefix over the row totals;
//   3. dd_tile_write   rows with candidates write them tile by tile in time
//                      order at their prefix offset.
// Same statistics, predicate and (dm_idx, t) order as the passes above.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "dd_detect_dev.cuh"
#include "dd_internal.h"

namespace {

constexpr int kStatsThreads = 512;
constexpr int kCountThreads = 256;
constexpr int kPerThread = ddk::kDetectChunk / kCountThreads;  // 16 contiguous samples
constexpr int kScanThreads = 1024;

// Correctly rounded (round-to-nearest-even) conversion of an unsigned
// 128-bit integer to double.  Values below 2^64 use the hardware
// conversion; larger ones are cut to their top 64 bits with every dropped
// bit folded into bit 0 (a sticky bit below the rounding position, which
// leaves the nearest-even decision unchanged), converted, and rescaled by an
// exact power of two.
__device__ double u128_to_double_rn(unsigned __int128 v) {
  const unsigned long long hi = static_cast<unsigned long long>(v >> 64);
  const unsigned long long lo = static_cast<unsigned long long>(v);
  if (hi == 0) return __ull2double_rn(lo);
  const int drop = 64 - __clzll(static_cast<long long>(hi));
  const unsigned __int128 mask = (static_cast<unsigned __int128>(1) << drop) - 1;
  const unsigned long long top =
      static_cast<unsigned long long>(v >> drop) | static_cast<unsigned long long>((v & mask) != 0);
  return scalbn(__ull2double_rn(top), drop);
}

// Smallest int64 v in [INT32_MIN, INT32_MAX + 1] with snr_of(v) > thr, where
// INT32_MAX + 1 stands for "none".  snr_of is monotone non-decreasing in v
// (IEEE subtraction and division by sigma > 0 are monotone), so a bisection
// finds the exact boundary of the double-precision decision.
__device__ int64_t int_threshold(double mean, double sigma, double thr) {
  int64_t lo = INT32_MIN, hi = static_cast<int64_t>(INT32_MAX) + 1;
  if (snr_of(static_cast<double>(lo), mean, sigma) > thr) return lo;
  while (hi - lo > 1) {  // pred(lo) false, pred(hi) true
    const int64_t mid = lo + (hi - lo) / 2;
    if (snr_of(static_cast<double>(mid), mean, sigma) > thr) hi = mid; else lo = mid;
  }
  return hi;
}

// Statistics of an integer row from its exact sums S1 = sum D, S2 = sum D^2
// over N samples:
//   mean = S1 / N,  rms = sqrt((double)(N*S2 - S1^2)) / N
// (numerator exact in 128 bits, one rounding to double), and the row's
// integer candidate threshold (int_threshold_window, else the bisection).
// Called by all 32 lanes of one warp (each computes the same result).
__device__ dd_row_stats finish_i32(long long s1, unsigned __int128 s2, int64_t n, double thr) {
  const __int128 S1 = s1;
  const __int128 S2 = static_cast<__int128>(s2);
  const __int128 num = static_cast<__int128>(n) * S2 - S1 * S1;  // >= 0
  const double dn = __ll2double_rn(n);
  dd_row_stats st;
  st.mean = __ddiv_rn(__ll2double_rn(s1), dn);
  st.sigma = __ddiv_rn(__dsqrt_rn(u128_to_double_rn(static_cast<unsigned __int128>(num))), dn);
  st.any = st.sigma > 0.0;
  st.ithr = static_cast<int64_t>(INT32_MAX) + 1;
  if (st.any && !int_threshold_window(st.mean, st.sigma, thr, &st.ithr))  // uniform in the warp
    st.ithr = int_threshold(st.mean, st.sigma, thr);
  st.fthr = INFINITY;
  return st;
}

// One CTA per row: S1 = sum D, S2 = sum D^2 exactly, then finish_i32.
__global__ void __launch_bounds__(kStatsThreads)
dd_stats_i32(const int32_t *__restrict__ D, int64_t n, double thr,
             dd_row_stats *__restrict__ stats) {
  __shared__ long long s_s1[kStatsThreads];
  __shared__ unsigned __int128 s_s2[kStatsThreads];
  const int32_t *row = D + static_cast<int64_t>(blockIdx.x) * n;
  long long s1 = 0;
  unsigned __int128 s2 = 0;
  unsigned long long part = 0;
  int pending = 0;
  for (int64_t t = threadIdx.x; t < n; t += kStatsThreads) {
    const long long v = row[t];
    s1 += v;
    part += static_cast<unsigned long long>(v * v);  // < 2^62 each
    if (++pending == 3) {  // flush before two more terms could overflow 64 bits
      s2 += part;
      part = 0;
      pending = 0;
    }
  }
  s2 += part;
  s_s1[threadIdx.x] = s1;
  s_s2[threadIdx.x] = s2;
  __syncthreads();
  for (int w = kStatsThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_s1[threadIdx.x] += s_s1[threadIdx.x + w];
      s_s2[threadIdx.x] += s_s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    const dd_row_stats st = finish_i32(s_s1[0], s_s2[0], n, thr);
    if (threadIdx.x == 0) stats[blockIdx.x] = st;
  }
}

// One CTA per row of f32 values: double sums of (x - K) with K the row's
// first value, combined in a fixed tree order (deterministic), then
//   mean = K + S1/N,  rms = sqrt(max(S2/N - (S1/N)^2, 0)),
// and the row's float candidate threshold.
__global__ void __launch_bounds__(kStatsThreads)
dd_stats_f32(const float *__restrict__ D, int64_t n, double thr,
             dd_row_stats *__restrict__ stats) {
  __shared__ double s_s1[kStatsThreads];
  __shared__ double s_s2[kStatsThreads];
  const float *row = D + static_cast<int64_t>(blockIdx.x) * n;
  const double K = static_cast<double>(row[0]);
  double s1 = 0.0, s2 = 0.0;
  for (int64_t t = threadIdx.x; t < n; t += kStatsThreads) {
    const double x = static_cast<double>(row[t]) - K;
    s1 += x;
    s2 += x * x;
  }
  s_s1[threadIdx.x] = s1;
  s_s2[threadIdx.x] = s2;
  __syncthreads();
  for (int w = kStatsThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_s1[threadIdx.x] += s_s1[threadIdx.x + w];
      s_s2[threadIdx.x] += s_s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < 32) {  // one warp, every lane the same result
    const double dn = static_cast<double>(n);
    const double m1 = s_s1[0] / dn;
    const double var = s_s2[0] / dn - m1 * m1;
    dd_row_stats st;
    st.mean = K + m1;
    st.sigma = sqrt(var > 0.0 ? var : 0.0);
    st.any = st.sigma > 0.0;
    st.fthr = INFINITY;
    if (st.any && !float_threshold_window(st.mean, st.sigma, thr, &st.fthr))
      st.fthr = float_threshold(st.mean, st.sigma, thr);
    st.ithr = static_cast<int64_t>(INT32_MAX) + 1;
    if (threadIdx.x == 0) stats[blockIdx.x] = st;
  }
}

template <typename T>
__global__ void __launch_bounds__(kCountThreads)
dd_count(const T *__restrict__ D, int64_t n, int nchunks, const dd_row_stats *__restrict__ stats,
         int64_t *__restrict__ counts) {
  __shared__ int s_cnt[kCountThreads / 32];
  const int d = blockIdx.y;
  const int chunk = blockIdx.x;
  const dd_row_stats st = stats[d];
  const T *row = D + static_cast<int64_t>(d) * n;
  const int64_t t0 = static_cast<int64_t>(chunk) * ddk::kDetectChunk;
  int cnt = 0;
  // coalesced sweep: sample t0 + k*256 + tid
#pragma unroll 4
  for (int k = 0; k < kPerThread; ++k) {
    const int64_t t = t0 + k * kCountThreads + threadIdx.x;
    if (t < n) cnt += is_candidate(row[t], st) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int total = 0;
    for (int w = 0; w < kCountThreads / 32; ++w) total += s_cnt[w];
    counts[static_cast<int64_t>(d) * nchunks + chunk] = total;
  }
}

// Single-CTA exclusive scan of m counts (each thread owns a contiguous run).
__global__ void __launch_bounds__(kScanThreads)
dd_scan(const int64_t *__restrict__ counts, int64_t m, int64_t *__restrict__ offsets,
        int64_t *__restrict__ total) {
  __shared__ int64_t s_part[kScanThreads];
  const int64_t per = (m + kScanThreads - 1) / kScanThreads;
  const int64_t lo = threadIdx.x * per;
  const int64_t hi = lo + per < m ? lo + per : m;
  int64_t sum = 0;
  for (int64_t i = lo; i < hi; ++i) sum += counts[i];
  s_part[threadIdx.x] = sum;
  __syncthreads();
  // Hillis-Steele inclusive scan over the per-thread sums.
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const int64_t add = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0;
    __syncthreads();
    s_part[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t run = s_part[threadIdx.x] - sum;
  for (int64_t i = lo; i < hi; ++i) {
    offsets[i] = run;
    run += counts[i];
  }
  if (threadIdx.x == kScanThreads - 1) *total = s_part[kScanThreads - 1];
}

template <typename T>
__global__ void __launch_bounds__(kCountThreads, 4)  // 4 CTAs per SM: no spills
dd_write(const T *__restrict__ D, int64_t n, int nchunks, const dd_row_stats *__restrict__ stats,
         const int64_t *__restrict__ counts, const int64_t *__restrict__ offsets,
         dd_candidate *__restrict__ cands, int64_t capacity) {
  __shared__ int s_scan[kCountThreads];
  const int d = blockIdx.y;
  const int chunk = blockIdx.x;
  const int64_t slot = static_cast<int64_t>(d) * nchunks + chunk;
  if (counts[slot] == 0) return;  // uniform across the CTA
  const int64_t base = offsets[slot];
  if (base >= capacity) return;
  const dd_row_stats st = stats[d];
  const T *row = D + static_cast<int64_t>(d) * n;
  // thread owns samples [t0 + tid*16, +16) so that output order is time order
  const int64_t t0 = static_cast<int64_t>(chunk) * ddk::kDetectChunk + threadIdx.x * kPerThread;
  unsigned mask = 0;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int64_t t = t0 + k;
    if (t < n && is_candidate(row[t], st)) mask |= 1u << k;
  }
  const int mine = __popc(mask);
  s_scan[threadIdx.x] = mine;
  __syncthreads();
  for (int o = 1; o < kCountThreads; o <<= 1) {
    const int add = threadIdx.x >= o ? s_scan[threadIdx.x - o] : 0;
    __syncthreads();
    s_scan[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t idx = base + s_scan[threadIdx.x] - mine;
  while (mask) {
    const int k = __ffs(mask) - 1;
    mask &= mask - 1;
    if (idx < capacity) {
      const double v = static_cast<double>(row[t0 + k]);
      dd_candidate c;
      c.dm_idx = d;
      c.t = static_cast<int32_t>(t0 + k);
      c.value = static_cast<float>(v);
      c.snr = static_cast<float>(snr_of(v, st.mean, st.sigma));
      cands[idx] = c;
    }
    ++idx;
  }
}

// ---- tiled detection after the staged kernels ----

// One CTA per row d (int32 rows after the staged u8 kernel): statistics from
// rowsums[d], then the candidates of each tile whose maximum reaches the
// threshold; tilecount[d][*] and rowcount[d].
__global__ void __launch_bounds__(kTileThreads)
dd_tile_count(const int32_t *__restrict__ D, int64_t n, int ntiles, double thr,
              const long long *__restrict__ rowsums, const int32_t *__restrict__ tilemax,
              dd_row_stats *__restrict__ stats, int32_t *__restrict__ tilecount,
              int64_t *__restrict__ rowcount) {
  __shared__ dd_row_stats s_st;
  const int d = blockIdx.x;
  if (threadIdx.x < 32) {
    const unsigned long long s2 = static_cast<unsigned long long>(rowsums[2 * d + 1]);
    const dd_row_stats st = finish_i32(rowsums[2 * d], static_cast<unsigned __int128>(s2), n, thr);
    if (threadIdx.x == 0) s_st = st, stats[d] = st;
  }
  __syncthreads();
  const dd_row_stats st = s_st;
  const int32_t *tmax = tilemax + static_cast<int64_t>(d) * ntiles;
  count_row_tiles<int32_t, ddk::kTileSamples>(
      D + static_cast<int64_t>(d) * n, n, ntiles, st,
      [&](int tt) { return static_cast<int64_t>(tmax[tt]) >= st.ithr; },
      tilecount + static_cast<int64_t>(d) * ntiles, rowcount + d);
}

// One CTA per row d (float rows after the float kernels): the row's
// statistics and float threshold from its tiles' partials (row_stats_f32),
// then the candidates of the tiles whose maximum reaches the threshold.
template <int TILE>
__global__ void __launch_bounds__(kTileThreads, 4)  // 4 CTAs per SM: room for its FP64 state
dd_tile_count_f32(const float *__restrict__ D, int64_t n, int ntiles, double thr,
                  const float4 *__restrict__ tilestats, dd_row_stats *__restrict__ stats,
                  int32_t *__restrict__ tilecount, int64_t *__restrict__ rowcount) {
  const int d = blockIdx.x;
  const float4 *ts = tilestats + static_cast<int64_t>(d) * ntiles;
  const dd_row_stats st = row_stats_f32<TILE>(ts, n, ntiles, thr, __drcp_rn(static_cast<double>(n)));
  if (threadIdx.x == 0) stats[d] = st;
  count_row_tiles<float, TILE>(
      D + static_cast<int64_t>(d) * n, n, ntiles, st, [&](int tt) { return ts[tt].w >= st.fthr; },
      tilecount + static_cast<int64_t>(d) * ntiles, rowcount + d);
}

// One CTA per row with candidates: tiles of TILE samples in time order, each
// tile's candidates in time order, at rowoff[d] + (candidates of earlier
// tiles).
template <typename T, int TILE>
__global__ void __launch_bounds__(kTileThreads)
dd_tile_write(const T *__restrict__ D, int64_t n, int ntiles,
              const dd_row_stats *__restrict__ stats, const int32_t *__restrict__ tilecount,
              const int64_t *__restrict__ rowcount, const int64_t *__restrict__ rowoff,
              dd_candidate *__restrict__ cands, int64_t capacity) {
  const int d = blockIdx.x;
  if (rowcount[d] == 0) return;  // uniform across the CTA
  const int64_t run = rowoff[d];
  if (run >= capacity) return;
  write_row_tiles<T, TILE>(D + static_cast<int64_t>(d) * n, n, ntiles, stats[d],
                           tilecount + static_cast<int64_t>(d) * ntiles, run, d, cands, capacity);
}

// ---- the same for the staged 8-bit beams of a batch, in two launches ----

struct DetectLaunch {
  ddk::DetectBeam beams[ddk::kMaxDetectBeams];
  int32_t nbeams;
  double thr;
};

// (beam, row) of CTA `row` of a batched launch (rows of beam b start at
// beams[b].row_begin).
__device__ __forceinline__ int beam_of_row(const DetectLaunch &L, int row) {
  int b = 0;
  while (b + 1 < L.nbeams && row >= L.beams[b + 1].row_begin) ++b;
  return b;
}

// dd_tile_count for every row of every beam of the launch.
__global__ void __launch_bounds__(kTileThreads)
dd_tile_count_beams(const __grid_constant__ DetectLaunch L) {
  __shared__ dd_row_stats s_st;
  const ddk::DetectBeam &a = L.beams[beam_of_row(L, blockIdx.x)];
  const int d = blockIdx.x - a.row_begin;
  if (threadIdx.x < 32) {
    const unsigned long long s2 = static_cast<unsigned long long>(a.rowsums[2 * d + 1]);
    const dd_row_stats st =
        finish_i32(a.rowsums[2 * d], static_cast<unsigned __int128>(s2), a.n, L.thr);
    if (threadIdx.x == 0) s_st = st, a.stats[d] = st;
  }
  __syncthreads();
  const dd_row_stats st = s_st;
  const int32_t *tmax = a.tilemax + static_cast<int64_t>(d) * a.ntiles;
  count_row_tiles<int32_t, ddk::kTileSamples>(
      a.D + static_cast<int64_t>(d) * a.n, a.n, a.ntiles, st,
      [&](int tt) { return static_cast<int64_t>(tmax[tt]) >= st.ithr; },
      a.tilecount + static_cast<int64_t>(d) * a.ntiles, a.rowcount + d);
}

// dd_tile_write for every row of every beam of the launch; each row's
// offset in its beam's candidate list is the sum of the earlier rows'
// counts (added up by the row's own CTA, so no scan launch is needed), and
// the CTA of a beam's last row stores the beam's total.
__global__ void __launch_bounds__(kTileThreads)
dd_tile_write_beams(const __grid_constant__ DetectLaunch L) {
  const ddk::DetectBeam &a = L.beams[beam_of_row(L, blockIdx.x)];
  const int d = blockIdx.x - a.row_begin;
  const int64_t before = rows_before(a.rowcount, d);
  const int64_t mine = a.rowcount[d];
  if (d == a.ndm - 1 && threadIdx.x == 0) *a.total = before + mine;
  if (mine == 0 || before >= a.capacity) return;  // uniform across the CTA
  write_row_tiles<int32_t, ddk::kTileSamples>(a.D + static_cast<int64_t>(d) * a.n, a.n, a.ntiles,
                                              a.stats[d],
                                              a.tilecount + static_cast<int64_t>(d) * a.ntiles,
                                              before, d, a.cands, a.capacity);
}

}  // namespace

namespace ddk {

int launch_tiled_detect_beams(const DetectBeam *beams, int nbeams, float nsigma,
                              cudaStream_t stream, cudaError_t *err) {
  if (nbeams < 1 || nbeams > kMaxDetectBeams) {
    *err = cudaErrorInvalidValue;
    return -1;
  }
  DetectLaunch L;
  std::memset(&L, 0, sizeof(L));
  int rows = 0;
  for (int i = 0; i < nbeams; ++i) {
    L.beams[i] = beams[i];
    L.beams[i].row_begin = rows;
    rows += beams[i].ndm;
  }
  L.nbeams = nbeams;
  L.thr = static_cast<double>(nsigma);
  dd_tile_count_beams<<<rows, kTileThreads, 0, stream>>>(L);
  dd_tile_write_beams<<<rows, kTileThreads, 0, stream>>>(L);
  *err = cudaGetLastError();
  return *err == cudaSuccess ? 2 : -1;
}

int launch_stats(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma,
                 cudaStream_t stream, cudaError_t *err) {
  const double thr = static_cast<double>(nsigma);
  if (p->dtype == DD_U8)
    dd_stats_i32<<<p->ndm, kStatsThreads, 0, stream>>>(static_cast<const int32_t *>(out), nsamp_out,
                                                        thr, p->d_stats);
  else
    dd_stats_f32<<<p->ndm, kStatsThreads, 0, stream>>>(static_cast<const float *>(out), nsamp_out,
                                                        thr, p->d_stats);
  *err = cudaGetLastError();
  return *err == cudaSuccess ? 1 : -1;
}

int launch_candidates(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma,
                      dd_candidate *cands, int64_t capacity, cudaStream_t stream,
                      cudaError_t *err) {
  const int nchunks = static_cast<int>((nsamp_out + kDetectChunk - 1) / kDetectChunk);
  const int64_t m = static_cast<int64_t>(p->ndm) * nchunks;
  const dim3 grid(nchunks, p->ndm);
  (void)nsigma;  // already folded into the per-row thresholds
  int n = 0;
  if (p->dtype == DD_U8)
    dd_count<int32_t><<<grid, kCountThreads, 0, stream>>>(static_cast<const int32_t *>(out),
                                                          nsamp_out, nchunks, p->d_stats,
                                                          p->d_counts);
  else
    dd_count<float><<<grid, kCountThreads, 0, stream>>>(static_cast<const float *>(out), nsamp_out,
                                                        nchunks, p->d_stats, p->d_counts);
  ++n;
  dd_scan<<<1, kScanThreads, 0, stream>>>(p->d_counts, m, p->d_offsets, p->d_total);
  ++n;
  if (capacity > 0) {
    if (p->dtype == DD_U8)
      dd_write<int32_t><<<grid, kCountThreads, 0, stream>>>(
          static_cast<const int32_t *>(out), nsamp_out, nchunks, p->d_stats, p->d_counts,
          p->d_offsets, cands, capacity);
    else
      dd_write<float><<<grid, kCountThreads, 0, stream>>>(
          static_cast<const float *>(out), nsamp_out, nchunks, p->d_stats, p->d_counts,
          p->d_offsets, cands, capacity);
    ++n;
  }
  *err = cudaGetLastError();
  return *err == cudaSuccess ? n : -1;
}

int launch_tiled_detect(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma,
                        dd_candidate *cands, int64_t capacity, cudaStream_t stream,
                        cudaError_t *err) {
  const int ntiles = static_cast<int>(time_tiles(nsamp_out));
  const int32_t *D = static_cast<const int32_t *>(out);
  dd_tile_count<<<p->ndm, kTileThreads, 0, stream>>>(
      D, nsamp_out, ntiles, static_cast<double>(nsigma),
      reinterpret_cast<const long long *>(p->d_rowsums), p->d_tilemax, p->d_stats,
      p->d_tilecount, p->d_rowcount);
  dd_scan<<<1, kScanThreads, 0, stream>>>(p->d_rowcount, p->ndm, p->d_rowoff, p->d_total);
  int n = 2;
  if (capacity > 0) {
    dd_tile_write<int32_t, kTileSamples><<<p->ndm, kTileThreads, 0, stream>>>(
        D, nsamp_out, ntiles, p->d_stats, p->d_tilecount, p->d_rowcount, p->d_rowoff, cands,
        capacity);
    ++n;
  }
  *err = cudaGetLastError();
  return *err == cudaSuccess ? n : -1;
}

int launch_tiled_detect_f32(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma,
                            dd_candidate *cands, int64_t capacity, cudaStream_t stream,
                            cudaError_t *err) {
  const int ntiles = static_cast<int>(octet_tiles(nsamp_out));
  const float *D = static_cast<const float *>(out);
  dd_tile_count_f32<kOctetTileSamples><<<p->ndm, kTileThreads, 0, stream>>>(
      D, nsamp_out, ntiles, static_cast<double>(nsigma), p->d_tilestats, p->d_stats,
      p->d_tilecount, p->d_rowcount);
  dd_scan<<<1, kScanThreads, 0, stream>>>(p->d_rowcount, p->ndm, p->d_rowoff, p->d_total);
  int n = 2;
  if (capacity > 0) {
    dd_tile_write<float, kOctetTileSamples><<<p->ndm, kTileThreads, 0, stream>>>(
        D, nsamp_out, ntiles, p->d_stats, p->d_tilecount, p->d_rowcount, p->d_rowoff, cands,
        capacity);
    ++n;
  }
  *err = cudaGetLastError();
  return *err == cudaSuccess ? n : -1;
}

}  // namespace ddk

// ---------------------------------------------------------------------------
// dd_detect_noalloc: the detection passes above with their scratch (per-row
// statistics, per-chunk counts and offsets, the total) in one file-scope
// device array instead of plan-owned cudaMalloc memory, for callers that must
// not allocate (dd.h).  Every GPU that loads the library holds the array until
// the process exits.
namespace {

constexpr int32_t kNoAllocMaxRows = 16384;        // DM trials per call
constexpr int64_t kNoAllocMaxChunks = 1 << 18;    // rows x ceil(nsamp_out / 4096)
constexpr size_t kNoAllocStatsBytes = sizeof(dd_row_stats) * kNoAllocMaxRows;
constexpr size_t kNoAllocChunkBytes = sizeof(int64_t) * kNoAllocMaxChunks;
constexpr size_t kNoAllocBytes = kNoAllocStatsBytes + 2 * kNoAllocChunkBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
struct NoAllocSlot {
  unsigned long long ctx_id = 0;  // context the address belongs to (0: none yet)
  void *addr = nullptr;
};
NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices];

// Unique id of the calling thread's current context (cuCtxGetCurrent +
// cuCtxGetId through the runtime's driver entry points, so that the library
// needs no link against the driver library); 0 if it cannot be read.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void **);
  using GetId = int (*)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device (the host-side
// symbol is only a stand-in, not a device address).  It is looked up with
// cudaGetSymbolAddress on the first call on a device and again whenever the
// device's context has been re-created since (e.g. by cudaDeviceReset), or on
// every call if the context id cannot be read.  Returns nullptr on failure.
void *noalloc_scratch(int device) {
  if (device < 0 || device >= kNoAllocMaxDevices) return nullptr;
  // no context may be current yet on this thread (id 0): the lookup below
  // makes the device's primary context current, and its id is read after it
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocSlot &slot = g_noalloc_slot[device];
  if (ctx == 0 || slot.ctx_id != ctx || !slot.addr) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return nullptr;
    slot.addr = ptr;
    slot.ctx_id = current_context_id();
  }
  return slot.addr;
}

}  // namespace

extern "C" int dd_detect_noalloc(const void *out, int32_t in_dtype, int32_t ndm, int64_t nsamp_out,
                                 float nsigma, dd_candidate *cands, int64_t capacity,
                                 int64_t *count, void *stream) {
  if (!out || !count || capacity < 0 || (capacity > 0 && !cands)) return DD_ERR_ARG;
  if (in_dtype != DD_U8 && in_dtype != DD_F16 && in_dtype != DD_F32) return DD_ERR_DTYPE;
  if (!std::isfinite(nsigma) || ndm < 1) return DD_ERR_ARG;
  if (nsamp_out < 1 || nsamp_out > INT32_MAX) return DD_ERR_SIZE;
  const int64_t nchunks = (nsamp_out + ddk::kDetectChunk - 1) / ddk::kDetectChunk;
  if (ndm > kNoAllocMaxRows || nchunks * ndm > kNoAllocMaxChunks) return DD_ERR_SIZE;
  *count = 0;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return DD_ERR_CUDA;
  unsigned char *base = static_cast<unsigned char *>(noalloc_scratch(device));
  if (!base) return DD_ERR_CUDA;
  dd_row_stats *stats = reinterpret_cast<dd_row_stats *>(base);
  int64_t *counts = reinterpret_cast<int64_t *>(base + kNoAllocStatsBytes);
  int64_t *offsets = reinterpret_cast<int64_t *>(base + kNoAllocStatsBytes + kNoAllocChunkBytes);
  int64_t *total = reinterpret_cast<int64_t *>(base + kNoAllocStatsBytes + 2 * kNoAllocChunkBytes);

  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double thr = static_cast<double>(nsigma);
  const int nch = static_cast<int>(nchunks);
  const dim3 grid(nch, ndm);
  if (in_dtype == DD_U8) {
    const int32_t *D = static_cast<const int32_t *>(out);
    dd_stats_i32<<<ndm, kStatsThreads, 0, s>>>(D, nsamp_out, thr, stats);
    dd_count<int32_t><<<grid, kCountThreads, 0, s>>>(D, nsamp_out, nch, stats, counts);
    dd_scan<<<1, kScanThreads, 0, s>>>(counts, nchunks * ndm, offsets, total);
    if (capacity > 0)
      dd_write<int32_t><<<grid, kCountThreads, 0, s>>>(D, nsamp_out, nch, stats, counts, offsets,
                                                        cands, capacity);
  } else {
    const float *D = static_cast<const float *>(out);
    dd_stats_f32<<<ndm, kStatsThreads, 0, s>>>(D, nsamp_out, thr, stats);
    dd_count<float><<<grid, kCountThreads, 0, s>>>(D, nsamp_out, nch, stats, counts);
    dd_scan<<<1, kScanThreads, 0, s>>>(counts, nchunks * ndm, offsets, total);
    if (capacity > 0)
      dd_write<float><<<grid, kCountThreads, 0, s>>>(D, nsamp_out, nch, stats, counts, offsets,
                                                      cands, capacity);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(count, total, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? DD_ERR_OOM : DD_ERR_CUDA;
  return *count > capacity ? DD_ERR_OVERFLOW : DD_OK;
}
