// dd_direct_dev.cuh -- device pieces of the plain-load dedispersion kernel
// shared by dd_dedisp_direct.cu and the one-launch small-beam path
// (dd_small.cu): the channel sums of a CTA's (time tile, DM group) and the
// tile's partial statistics, so that both give the same outputs and
// partials bit for bit.  Internal to libdd.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]  (Sec. 2.1.1, brute-force equation).
// A CTA covers kDirectThreads consecutive output samples (one per thread) of
// NDMS consecutive DM trials, with one register accumulator per trial (the
// thesis's Sec. 2.4 layout); delays of a group of channels for the CTA's
// trials are staged in shared memory (channel/DM order keeps that load
// coalesced, Sec. 3.4).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kDirectThreads = 256;
constexpr int kDelayChans = 64;

template <typename T>
struct DirectTraits;
// load: a sample from global memory (read-only path); load_shared: from a
// copy in shared memory; both give the sample's value in acc_t.
template <>
struct DirectTraits<uint8_t> {
  using acc_t = int32_t;
  static __device__ __forceinline__ int32_t load(const uint8_t *p) { return __ldg(p); }
  static __device__ __forceinline__ int32_t load_shared(const uint8_t *p) { return *p; }
};
template <>
struct DirectTraits<uint16_t> {  // IEEE binary16 bits
  using acc_t = float;
  static __device__ __forceinline__ float load(const uint16_t *p) {
    return __half2float(__ushort_as_half(__ldg(p)));
  }
  static __device__ __forceinline__ float load_shared(const uint16_t *p) {
    return __half2float(__ushort_as_half(*p));
  }
};
template <>
struct DirectTraits<float> {
  using acc_t = float;
  static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ float load_shared(const float *p) { return *p; }
};

// Channels loaded ahead of their adds: kInFlight samples per thread in
// flight (U channels x NDMS trials), so that a thread waits for one memory
// round trip per U channels instead of one per channel.
constexpr int kInFlight = 32;

// acc[j] = sum over channels c (in order 0 .. nchan-1) of
// in[c][t + delays[c][d0 + j]] for the calling thread's output sample t
// (when live; trials past ndm read with delay 0 and are never stored).
// Whole CTA (shared delay staging); s_delay holds kDelayChans x NDMS.
template <typename T, int NDMS>
__device__ __forceinline__ void direct_sums(const T *__restrict__ in, int64_t pitch,
                                            const int32_t *__restrict__ delays, int32_t nchan,
                                            int32_t ndm, int d0, int64_t t, bool live,
                                            typename DirectTraits<T>::acc_t (&acc)[NDMS],
                                            int32_t (*s_delay)[NDMS]) {
  using acc_t = typename DirectTraits<T>::acc_t;
  constexpr int U = kInFlight / NDMS > 1 ? kInFlight / NDMS : 1;
  static_assert(kDelayChans % U == 0, "whole channel groups per delay stage");
#pragma unroll
  for (int j = 0; j < NDMS; ++j) acc[j] = acc_t(0);
  for (int c0 = 0; c0 < nchan; c0 += kDelayChans) {
    const int nc = nchan - c0 < kDelayChans ? nchan - c0 : kDelayChans;
    __syncthreads();  // s_delay free from the previous stage
    for (int i = threadIdx.x; i < kDelayChans * NDMS; i += kDirectThreads) {
      const int cc = i / NDMS, j = i % NDMS;
      s_delay[cc][j] = (cc < nc && d0 + j < ndm)
                           ? delays[static_cast<int64_t>(c0 + cc) * ndm + d0 + j]
                           : 0;
    }
    __syncthreads();
    if (!live) continue;
    const T *base = in + static_cast<int64_t>(c0) * pitch + t;
    for (int cc = 0; cc < nc; cc += U) {
      acc_t v[U][NDMS];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (cc + u < nc) {
          const T *row = base + static_cast<int64_t>(cc + u) * pitch;
#pragma unroll
          for (int j = 0; j < NDMS; ++j) v[u][j] = DirectTraits<T>::load(row + s_delay[cc + u][j]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (cc + u < nc) {
#pragma unroll
          for (int j = 0; j < NDMS; ++j) acc[j] += v[u][j];
        }
      }
    }
  }
}

template <int NDMS>
struct PartialScratch {
  float k[NDMS];
  float red[3 * NDMS][kDirectThreads / 32];
};

// The CTA's time tile (its kDirectThreads outputs, one per thread, `live`
// for those before nsamp_out) of trials d0 .. d0+NDMS-1: each trial's
// partials {K, sum (D - K), sum (D - K)^2, max D}, K the tile's first output,
// to tilestats[(d0 + j) * ntiles + tile], each sum in a fixed order (lanes
// by xor butterfly, then the warps in order).  Whole CTA.
template <int NDMS>
__device__ __forceinline__ void tile_partials(const float (&acc)[NDMS], bool live, int d0,
                                              int32_t ndm, int64_t ntiles, int64_t tile,
                                              float4 *tilestats, PartialScratch<NDMS> &sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // sh free from a previous tile
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NDMS; ++j) sh.k[j] = acc[j];  // thread 0 holds the tile's first output
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NDMS; ++j) {
    const float y = live ? __fsub_rn(acc[j], sh.k[j]) : 0.f;
    float s1 = y, s2 = live ? __fmul_rn(y, y) : 0.f, mx = live ? acc[j] : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 = __fadd_rn(s1, __shfl_xor_sync(0xffffffffu, s1, o));
      s2 = __fadd_rn(s2, __shfl_xor_sync(0xffffffffu, s2, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      sh.red[3 * j][w] = s1;
      sh.red[3 * j + 1][w] = s2;
      sh.red[3 * j + 2][w] = mx;
    }
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < NDMS && d0 + j < ndm) {
    float s1 = sh.red[3 * j][0], s2 = sh.red[3 * j + 1][0], mx = sh.red[3 * j + 2][0];
#pragma unroll
    for (int k = 1; k < kDirectThreads / 32; ++k) {
      s1 = __fadd_rn(s1, sh.red[3 * j][k]);
      s2 = __fadd_rn(s2, sh.red[3 * j + 1][k]);
      mx = fmaxf(mx, sh.red[3 * j + 2][k]);
    }
    tilestats[static_cast<int64_t>(d0 + j) * ntiles + tile] = make_float4(sh.k[j], s1, s2, mx);
  }
}

}  // namespace
