// dd_detect_dev.cuh -- device pieces of the detection passes (Sec. 3.5
// normalisation, Sec. 3.6 thresholding) shared by dd_detect.cu and the
// one-launch small-beam path (dd_small.cu), so that both compute the same
// statistics, thresholds and candidate lists bit for bit.  Internal to libdd.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "dd_internal.h"

namespace {

// Loads of the detection passes.  PlainLd for data written by earlier
// launches; L2Ld (ld.global.cg, no L1) for data that other CTAs of the same
// launch wrote before a grid barrier.
struct PlainLd {
  template <typename T>
  __device__ __forceinline__ T operator()(const T *p) const { return *p; }
};
struct L2Ld {
  __device__ __forceinline__ float operator()(const float *p) const { return __ldcg(p); }
  __device__ __forceinline__ float4 operator()(const float4 *p) const { return __ldcg(p); }
  __device__ __forceinline__ int32_t operator()(const int32_t *p) const { return __ldcg(p); }
  __device__ __forceinline__ int64_t operator()(const int64_t *p) const {
    return static_cast<int64_t>(__ldcg(reinterpret_cast<const long long *>(p)));
  }
};

__device__ __forceinline__ double snr_of(double v, double mean, double sigma) {
  return __ddiv_rn(__dsub_rn(v, mean), sigma);
}

// Order-preserving map of non-NaN floats onto uint32.
__device__ __forceinline__ uint32_t float_order(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_float(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Smallest float x (-inf .. +inf) with snr_of((double)x) > thr; +inf passes
// for any finite thr, so it bounds the search.
__device__ float float_threshold(double mean, double sigma, double thr) {
  uint32_t lo = float_order(-INFINITY), hi = float_order(INFINITY);
  if (snr_of(-static_cast<double>(INFINITY), mean, sigma) > thr) return -INFINITY;
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (snr_of(static_cast<double>(order_float(mid)), mean, sigma) > thr) hi = mid; else lo = mid;
  }
  return order_float(hi);
}

// The candidate test, equivalent to snr > nsigma in IEEE double.
__device__ __forceinline__ bool is_candidate(int32_t v, const dd_row_stats &st) {
  return st.any && static_cast<int64_t>(v) >= st.ithr;
}
__device__ __forceinline__ bool is_candidate(float v, const dd_row_stats &st) {
  return st.any && v >= st.fthr;
}

constexpr int kTileThreads = 256;
constexpr int kTileList = 1024;  // tiles examined per round

// float_threshold by the whole CTA (kTileThreads threads, uniform call): each
// round probes kTileThreads - 1 evenly spaced points of the open interval
// (lo, hi) of float orders at once and keeps the largest probe that fails
// and the smallest that passes.  The predicate is monotone in the order, so
// this finds the same boundary as the bisection, in 5 rounds instead of 32
// dependent double divisions.
__device__ __forceinline__ float float_threshold_cta(double mean, double sigma, double thr) {
  __shared__ uint32_t s_lo, s_hi;
  if (snr_of(-static_cast<double>(INFINITY), mean, sigma) > thr) return -INFINITY;
  uint32_t lo = float_order(-INFINITY), hi = float_order(INFINITY);
  while (hi - lo > 1) {  // pred(lo) false, pred(hi) true
    const uint32_t k = threadIdx.x;
    const uint32_t x =
        lo + static_cast<uint32_t>(static_cast<uint64_t>(hi - lo) * k / kTileThreads);
    __syncthreads();  // the previous round's reads of s_lo / s_hi are done
    if (k == 0) s_lo = lo, s_hi = hi;
    __syncthreads();
    if (k > 0 && x > lo) {  // x < hi since k < kTileThreads
      if (snr_of(static_cast<double>(order_float(x)), mean, sigma) > thr)
        atomicMin(&s_hi, x);
      else
        atomicMax(&s_lo, x);
    }
    __syncthreads();
    lo = s_lo;
    hi = s_hi;
  }
  return order_float(hi);
}

// Exclusive prefix of v over the CTA (kTileThreads threads); *total gets the sum.
__device__ __forceinline__ int block_exclusive(int v, int *total) {
  __shared__ int s_warp[kTileThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  __syncthreads();  // s_warp free from any previous call
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  int before = 0, all = 0;
#pragma unroll
  for (int k = 0; k < kTileThreads / 32; ++k) {
    const int x = s_warp[k];
    before += k < w ? x : 0;
    all += x;
  }
  *total = all;
  return before + inc - v;
}

// Row d's candidates per tile of TILE samples: the tiles that `reaches(tt)`
// admits (their largest value passes the threshold; no other tile can hold a
// candidate) are read and counted into tcnt[tt], the others get 0; the row
// total goes to *rowcount.  Called by the whole CTA after st is final.
// LIST: tiles examined per round (shared-memory list size).
template <typename T, int TILE, typename Reaches, typename Ld = PlainLd, int LIST = kTileList>
__device__ __forceinline__ void count_row_tiles(const T *row, int64_t n, int ntiles, const dd_row_stats &st,
                                Reaches reaches, int32_t *tcnt, int64_t *rowcount,
                                Ld ld = Ld()) {
  constexpr int kPer = TILE / kTileThreads;  // consecutive samples per thread
  static_assert(TILE % kTileThreads == 0, "whole samples per thread");
  __shared__ int s_list[LIST];
  __shared__ int s_nlist;
  int64_t total = 0;  // thread 0
  for (int base = 0; base < ntiles; base += LIST) {
    if (threadIdx.x == 0) s_nlist = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < LIST && base + k < ntiles; k += kTileThreads) {
      const int tt = base + k;
      if (st.any && reaches(tt)) {
        s_list[atomicAdd(&s_nlist, 1)] = tt;  // order irrelevant: counts go by tile
      } else {
        tcnt[tt] = 0;
      }
    }
    __syncthreads();
    const int nl = s_nlist;
    for (int k = 0; k < nl; ++k) {
      const int tt = s_list[k];
      const int64_t t0 = static_cast<int64_t>(tt) * TILE + threadIdx.x * kPer;
      int mine = 0;
#pragma unroll
      for (int u = 0; u < kPer; ++u)
        mine += (t0 + u < n && is_candidate(ld(row + t0 + u), st)) ? 1 : 0;
      int tile_total = 0;
      block_exclusive(mine, &tile_total);
      if (threadIdx.x == 0) {
        tcnt[tt] = tile_total;
        total += tile_total;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *rowcount = total;
}

// Row d's candidates, tile by tile in time order and each tile's in time
// order, from list position `run` on (the candidates of the earlier rows);
// only tiles with a non-zero count in tcnt are read.  Whole CTA.
// pre_tile >= 0: the caller already computed, for tile pre_tile, the snr of
// this thread's candidates (pre_snr[u] for sample u of the thread's kPer).
template <typename T, int TILE, typename Ld = PlainLd, int LIST = kTileList>
__device__ __forceinline__ void write_row_tiles(const T *row, int64_t n, int ntiles, const dd_row_stats &st,
                                const int32_t *tcnt, int64_t run, int32_t d,
                                dd_candidate *cands, int64_t capacity, Ld ld = Ld(),
                                int pre_tile = -1, const float *pre_snr = nullptr) {
  constexpr int kPer = TILE / kTileThreads;
  __shared__ int s_cnt[LIST];
  for (int base = 0; base < ntiles && run < capacity; base += LIST) {
    __syncthreads();  // s_cnt free from the previous round
    for (int k = threadIdx.x; k < LIST && base + k < ntiles; k += kTileThreads)
      s_cnt[k] = ld(tcnt + base + k);
    __syncthreads();
    const int lim = ntiles - base < LIST ? ntiles - base : LIST;
    // the tiles with candidates, 32 at a time in order (every warp finds the
    // same ones, so the loop below is uniform across the CTA)
    for (int k0 = 0; k0 < lim && run < capacity; k0 += 32) {
     const int kl = k0 + (threadIdx.x & 31);
     unsigned todo = __ballot_sync(0xffffffffu, kl < lim && s_cnt[kl] != 0);
     while (todo && run < capacity) {
      const int k = k0 + __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t t0 = static_cast<int64_t>(base + k) * TILE + threadIdx.x * kPer;
      unsigned mask = 0;
      T v[kPer];
      float snr[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        v[u] = t0 + u < n ? ld(row + t0 + u) : T(0);
        if (t0 + u < n && is_candidate(v[u], st)) {
          mask |= 1u << u;
          // the division (~0.3 us in FP64) overlaps the prefix below
          snr[u] = base + k == pre_tile
                       ? pre_snr[u]
                       : static_cast<float>(snr_of(static_cast<double>(v[u]), st.mean, st.sigma));
        }
      }
      int tile_total = 0;
      int64_t idx = run + block_exclusive(__popc(mask), &tile_total);
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        if (mask & (1u << u)) {
          if (idx < capacity) {
            dd_candidate cd;
            cd.dm_idx = d;
            cd.t = static_cast<int32_t>(t0 + u);
            cd.value = static_cast<float>(v[u]);
            cd.snr = snr[u];
            cands[idx] = cd;
          }
          ++idx;
        }
      }
      run += tile_total;
     }
    }
  }
}

// Sum of the earlier rows' counts, rowcount[0 .. d-1] (whole CTA; every
// thread gets it).
template <typename Ld = PlainLd>
__device__ __forceinline__ int64_t rows_before(const int64_t *rowcount, int d, Ld ld = Ld()) {
  __shared__ long long s_part[kTileThreads / 32];
  long long before = 0;
  for (int r = threadIdx.x; r < d; r += kTileThreads) before += ld(rowcount + r);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
  __syncthreads();  // s_part free from a previous call
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = before;
  __syncthreads();
  before = 0;
#pragma unroll
  for (int w = 0; w < kTileThreads / 32; ++w) before += s_part[w];
  return before;
}

// The float threshold from an estimate (one warp, uniform arguments): the
// 32 floats around float(mean + thr * sigma) are tested at once; if the
// first passes nowhere but a later one does, the first passing one is the
// boundary (the predicate is monotone), i.e. float_threshold's result.
// Returns false when the boundary is not inside the window (the caller then
// runs the full search).
__device__ __forceinline__ bool float_threshold_window(double mean, double sigma, double thr,
                                                       float *fthr) {
  const int lane = threadIdx.x & 31;
  const float f = __double2float_rn(__fma_rn(thr, sigma, mean));
  if (f != f) return false;
  const int64_t base = static_cast<int64_t>(float_order(f)) - 16;
  if (base < static_cast<int64_t>(float_order(-INFINITY)) ||
      base + 31 > static_cast<int64_t>(float_order(INFINITY)))
    return false;
  const uint32_t o = static_cast<uint32_t>(base + lane);
  const bool pass = snr_of(static_cast<double>(order_float(o)), mean, sigma) > thr;
  const unsigned mask = __ballot_sync(0xffffffffu, pass);
  if (mask == 0u || (mask & 1u)) return false;
  *fthr = order_float(static_cast<uint32_t>(base + __ffs(mask) - 1));
  return true;
}

// The same for the integer threshold (int_threshold's result): the 32
// integers around floor(mean + thr * sigma), inside [INT32_MIN, INT32_MAX + 1].
__device__ __forceinline__ bool int_threshold_window(double mean, double sigma, double thr,
                                                     int64_t *ithr) {
  const int lane = threadIdx.x & 31;
  const double e = floor(__fma_rn(thr, sigma, mean));
  if (!(e >= static_cast<double>(INT32_MIN) + 16.0 && e <= static_cast<double>(INT32_MAX) - 15.0))
    return false;
  const int64_t base = static_cast<int64_t>(e) - 16;
  const bool pass = snr_of(static_cast<double>(base + lane), mean, sigma) > thr;
  const unsigned mask = __ballot_sync(0xffffffffu, pass);
  if (mask == 0u || (mask & 1u)) return false;
  *ithr = base + __ffs(mask) - 1;
  return true;
}

// A float row's statistics from its tiles' partials {K, S1 = sum (D - K),
// S2 = sum (D - K)^2, max} (ts[0 .. ntiles-1], TILE samples each, the last
// one n - (ntiles-1)*TILE), as shifted sums about K0, tile 0's K (the
// shifted-data method of dd_stats_f32, in FP64):
//   A1 = sum over tiles of S1 + n_t (K - K0)                = sum (D - K0)
//   A2 = sum over tiles of S2 + (K - K0)(2 S1 + n_t (K - K0)) = sum (D - K0)^2
// each thread adding a contiguous run of tiles in order, the threads' sums
// added by xor butterfly within warps and then the warps in order; then, with
// r = rn = 1/n (correctly rounded, __drcp_rn: computed by the caller ahead of
// time, an FP64 division taking ~0.3 us on this GPU),
//   mean = K0 + A1 r,  rms = sqrt(max(A2 - A1 (A1 r), 0) r),
// and the float threshold for nsigma thr (float_threshold_window, else the
// whole CTA's float_threshold_cta).  Whole CTA; every thread gets the result.
template <int TILE, typename Ld = PlainLd>
__device__ __forceinline__ dd_row_stats row_stats_f32(const float4 *ts, int64_t n, int ntiles, double thr,
                                      double rn, Ld ld = Ld()) {
  __shared__ double s_a[2][kTileThreads / 32];
  __shared__ dd_row_stats s_st;
  __shared__ int s_found;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int per = (ntiles + kTileThreads - 1) / kTileThreads;
  const double K0 = static_cast<double>(ld(ts).x);
  double a1 = 0.0, a2 = 0.0;
  for (int tt = threadIdx.x * per; tt < (threadIdx.x + 1) * per && tt < ntiles; ++tt) {
    const float4 v = ld(ts + tt);
    const int64_t rest = n - static_cast<int64_t>(tt) * TILE;
    const double nt = static_cast<double>(rest < TILE ? rest : TILE);
    const double dk = __dsub_rn(static_cast<double>(v.x), K0);  // exact
    const double s1 = v.y, s2 = v.z;
    a1 = __dadd_rn(a1, __fma_rn(nt, dk, s1));
    a2 = __dadd_rn(a2, __fma_rn(dk, __fma_rn(nt, dk, __dmul_rn(2.0, s1)), s2));
  }
  // warps past the last tile hold zeros: they skip the butterfly
  if (w * 32 * per < ntiles) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a1 = __dadd_rn(a1, __shfl_xor_sync(0xffffffffu, a1, o));
      a2 = __dadd_rn(a2, __shfl_xor_sync(0xffffffffu, a2, o));
    }
  }
  __syncthreads();  // s_a / s_st free from a previous call
  if (lane == 0) s_a[0][w] = a1, s_a[1][w] = a2;
  __syncthreads();
  if (w == 0) {
    double A1 = s_a[0][0], A2 = s_a[1][0];
    const int nw = (ntiles + 32 * per - 1) / (32 * per);  // warps with tiles
    for (int k = 1; k < nw && k < kTileThreads / 32; ++k) {
      A1 = __dadd_rn(A1, s_a[0][k]);
      A2 = __dadd_rn(A2, s_a[1][k]);
    }
    const double m1 = __dmul_rn(A1, rn);
    const double m2 = __fma_rn(-A1, m1, A2);
    dd_row_stats st;
    st.mean = __dadd_rn(K0, m1);
    st.sigma = __dsqrt_rn(__dmul_rn(m2 > 0.0 ? m2 : 0.0, rn));
    st.any = st.sigma > 0.0;
    st.ithr = static_cast<int64_t>(INT32_MAX) + 1;
    st.fthr = INFINITY;
    const bool found = !st.any || float_threshold_window(st.mean, st.sigma, thr, &st.fthr);
    if (lane == 0) {
      s_st = st;
      s_found = found ? 1 : 0;
    }
  }
  __syncthreads();
  dd_row_stats st = s_st;
  if (!s_found) st.fthr = float_threshold_cta(st.mean, st.sigma, thr);  // uniform
  return st;
}

}  // namespace
