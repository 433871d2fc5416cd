// dd_dedisp_direct.cu -- plain-load dedispersion kernel (any alignment, any
// pitch): the layout-agnostic path of dd_execute.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]  (Sec. 2.1.1, brute-force equation).
// The grid maps onto the output (DM tile, time tile) space; each thread owns
// one output sample for 16 (or, for small outputs, 4) consecutive DM trials,
// with one register accumulator per trial (the thesis's Sec. 2.4 layout),
// and reads the input through the L1/L2 caches.  Delays of a group of channels for the CTA's DM
// tile are staged in shared memory (channel/DM order keeps that load
// coalesced, Sec. 3.4).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dd_internal.h"

namespace {

constexpr int kDirectThreads = 256;
constexpr int kDelayChans = 64;
static_assert(kDirectThreads == ddk::kOctetTileSamples,
              "a CTA's time tile is one per-tile statistics tile");

template <typename T>
struct DirectTraits;
template <>
struct DirectTraits<uint8_t> {
  using acc_t = int32_t;
  static __device__ __forceinline__ int32_t load(const uint8_t *p) { return __ldg(p); }
};
template <>
struct DirectTraits<uint16_t> {  // IEEE binary16 bits
  using acc_t = float;
  static __device__ __forceinline__ float load(const uint16_t *p) {
    return __half2float(__ushort_as_half(__ldg(p)));
  }
};
template <>
struct DirectTraits<float> {
  using acc_t = float;
  static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
};

// Sum of v over the CTA in a fixed order (warp shuffles, then the warps in
// order); every thread gets the result.  `red` holds kDirectThreads / 32
// entries.
template <typename F, typename Op>
__device__ __forceinline__ F cta_reduce(F v, F *red, Op op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();  // red free from the previous reduction
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  F r = red[0];
#pragma unroll
  for (int w = 1; w < kDirectThreads / 32; ++w) r = op(r, red[w]);
  return r;
}

// NDMS DM trials per thread (16, or 4 for small outputs, so that the grid
// covers the GPU).  With tilestats (float rows only), the CTA's 256 outputs
// of each of its trials -- one statistics tile -- give that tile's partials
// {K, sum (D - K), sum (D - K)^2, max D}, K the tile's first output, in a
// fixed order.
template <typename T, int NDMS>
__global__ void __launch_bounds__(kDirectThreads)
dd_dedisperse_direct(const T *__restrict__ in, int64_t pitch, const int32_t *__restrict__ delays,
                     int32_t nchan, int32_t ndm, int64_t nsamp_out,
                     typename DirectTraits<T>::acc_t *__restrict__ out, int64_t out_pitch,
                     float4 *__restrict__ tilestats) {
  using acc_t = typename DirectTraits<T>::acc_t;
  __shared__ int32_t s_delay[kDelayChans][NDMS];
  __shared__ float s_red[kDirectThreads / 32];
  __shared__ float s_k;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * kDirectThreads + threadIdx.x;
  const int d0 = blockIdx.y * NDMS;
  const bool live = t < nsamp_out;
  acc_t acc[NDMS];
#pragma unroll
  for (int j = 0; j < NDMS; ++j) acc[j] = acc_t(0);

  for (int c0 = 0; c0 < nchan; c0 += kDelayChans) {
    const int nc = nchan - c0 < kDelayChans ? nchan - c0 : kDelayChans;
    __syncthreads();
    for (int i = threadIdx.x; i < kDelayChans * NDMS; i += kDirectThreads) {
      const int cc = i / NDMS, j = i % NDMS;
      // trials past ndm read with delay 0 (in range) and are never stored
      s_delay[cc][j] = (cc < nc && d0 + j < ndm)
                           ? delays[static_cast<int64_t>(c0 + cc) * ndm + d0 + j]
                           : 0;
    }
    __syncthreads();
    if (live) {
      for (int cc = 0; cc < nc; ++cc) {
        const T *row = in + static_cast<int64_t>(c0 + cc) * pitch + t;
#pragma unroll
        for (int j = 0; j < NDMS; ++j) acc[j] += DirectTraits<T>::load(row + s_delay[cc][j]);
      }
    }
  }
  if (live) {
#pragma unroll
    for (int j = 0; j < NDMS; ++j)
      if (d0 + j < ndm) out[static_cast<int64_t>(d0 + j) * out_pitch + t] = acc[j];
  }
  if constexpr (!std::is_same<acc_t, int32_t>::value) {
    if (tilestats) {
      const int64_t ntiles = (nsamp_out + kDirectThreads - 1) / kDirectThreads;
#pragma unroll 1
      for (int j = 0; j < NDMS; ++j) {
        if (d0 + j >= ndm) break;  // the same in every thread
        if (threadIdx.x == 0) s_k = acc[j];  // thread 0 holds the tile's first output
        __syncthreads();
        const float K = s_k;
        const float y = live ? acc[j] - K : 0.f;
        const float s1 = cta_reduce(y, s_red, [](float a, float b) { return a + b; });
        const float s2 = cta_reduce(live ? y * y : 0.f, s_red,
                                    [](float a, float b) { return a + b; });
        const float mx = cta_reduce(live ? static_cast<float>(acc[j]) : -INFINITY, s_red,
                                    [](float a, float b) { return fmaxf(a, b); });
        if (threadIdx.x == 0)
          tilestats[static_cast<int64_t>(d0 + j) * ntiles + blockIdx.x] = make_float4(K, s1, s2, mx);
      }
    }
  }
}

template <typename T, typename A>
void launch(int ndms, const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
            void *out, int64_t out_pitch, float4 *tilestats, cudaStream_t stream) {
  const unsigned tiles = static_cast<unsigned>((nsamp_out + kDirectThreads - 1) / kDirectThreads);
  if (ndms == 16) {
    const dim3 grid(tiles, static_cast<unsigned>((p->ndm + 15) / 16));
    dd_dedisperse_direct<T, 16><<<grid, kDirectThreads, 0, stream>>>(
        static_cast<const T *>(block), pitch, p->d_delays, p->nchan, p->ndm, nsamp_out,
        static_cast<A *>(out), out_pitch, tilestats);
  } else {
    const dim3 grid(tiles, static_cast<unsigned>((p->ndm + 3) / 4));
    dd_dedisperse_direct<T, 4><<<grid, kDirectThreads, 0, stream>>>(
        static_cast<const T *>(block), pitch, p->d_delays, p->nchan, p->ndm, nsamp_out,
        static_cast<A *>(out), out_pitch, tilestats);
  }
}

}  // namespace

namespace ddk {

int launch_dedisperse_direct(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                             void *out, int64_t out_pitch, float4 *tilestats, cudaStream_t stream,
                             cudaError_t *err) {
  // 16 trials per thread unless that leaves fewer than two CTAs per SM
  const int64_t tiles = (nsamp_out + kDirectThreads - 1) / kDirectThreads;
  const int ndms = tiles * ((p->ndm + 15) / 16) < 2 * static_cast<int64_t>(p->sm_count) ? 4 : 16;
  switch (p->dtype) {
    case DD_U8:
      launch<uint8_t, int32_t>(ndms, p, block, pitch, nsamp_out, out, out_pitch, nullptr, stream);
      break;
    case DD_F16:
      launch<uint16_t, float>(ndms, p, block, pitch, nsamp_out, out, out_pitch, tilestats, stream);
      break;
    default:
      launch<float, float>(ndms, p, block, pitch, nsamp_out, out, out_pitch, tilestats, stream);
      break;
  }
  *err = cudaGetLastError();
  return *err == cudaSuccess ? 1 : -1;
}

}  // namespace ddk
