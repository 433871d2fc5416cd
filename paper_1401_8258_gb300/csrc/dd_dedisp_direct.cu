// dd_dedisp_direct.cu -- plain-load dedispersion kernel (any alignment, any
// pitch): the layout-agnostic path of dd_execute.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]  (Sec. 2.1.1, brute-force equation).
// The grid maps onto the output (DM tile, time tile) space; each thread owns
// one output sample for kDirectDms consecutive DM trials, with one register
// accumulator per trial (the thesis's Sec. 2.4 layout), and reads the input
// through the L1/L2 caches.  Delays of a group of channels for the CTA's DM
// tile are staged in shared memory (channel/DM order keeps that load
// coalesced, Sec. 3.4).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace {

constexpr int kDirectThreads = 256;
constexpr int kDirectDms = 16;
constexpr int kDelayChans = 64;

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

template <typename T>
__global__ void __launch_bounds__(kDirectThreads)
dd_dedisperse_direct(const T *__restrict__ in, int64_t pitch, const int32_t *__restrict__ delays,
                     int32_t nchan, int32_t ndm, int64_t nsamp_out,
                     typename DirectTraits<T>::acc_t *__restrict__ out, int64_t out_pitch) {
  using acc_t = typename DirectTraits<T>::acc_t;
  __shared__ int32_t s_delay[kDelayChans][kDirectDms];
  const int64_t t = static_cast<int64_t>(blockIdx.x) * kDirectThreads + threadIdx.x;
  const int d0 = blockIdx.y * kDirectDms;
  const bool live = t < nsamp_out;
  acc_t acc[kDirectDms];
#pragma unroll
  for (int j = 0; j < kDirectDms; ++j) acc[j] = acc_t(0);

  for (int c0 = 0; c0 < nchan; c0 += kDelayChans) {
    const int nc = nchan - c0 < kDelayChans ? nchan - c0 : kDelayChans;
    __syncthreads();
    for (int i = threadIdx.x; i < kDelayChans * kDirectDms; i += kDirectThreads) {
      const int cc = i / kDirectDms, j = i % kDirectDms;
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
        for (int j = 0; j < kDirectDms; ++j) acc[j] += DirectTraits<T>::load(row + s_delay[cc][j]);
      }
    }
  }
  if (live) {
#pragma unroll
    for (int j = 0; j < kDirectDms; ++j)
      if (d0 + j < ndm) out[static_cast<int64_t>(d0 + j) * out_pitch + t] = acc[j];
  }
}

}  // namespace

namespace ddk {

int launch_dedisperse_direct(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                             void *out, int64_t out_pitch, cudaStream_t stream, cudaError_t *err) {
  const dim3 grid(static_cast<unsigned>((nsamp_out + kDirectThreads - 1) / kDirectThreads),
                  static_cast<unsigned>((p->ndm + kDirectDms - 1) / kDirectDms));
  switch (p->dtype) {
    case DD_U8:
      dd_dedisperse_direct<uint8_t><<<grid, kDirectThreads, 0, stream>>>(
          static_cast<const uint8_t *>(block), pitch, p->d_delays, p->nchan, p->ndm, nsamp_out,
          static_cast<int32_t *>(out), out_pitch);
      break;
    case DD_F16:
      dd_dedisperse_direct<uint16_t><<<grid, kDirectThreads, 0, stream>>>(
          static_cast<const uint16_t *>(block), pitch, p->d_delays, p->nchan, p->ndm, nsamp_out,
          static_cast<float *>(out), out_pitch);
      break;
    default:
      dd_dedisperse_direct<float><<<grid, kDirectThreads, 0, stream>>>(
          static_cast<const float *>(block), pitch, p->d_delays, p->nchan, p->ndm, nsamp_out,
          static_cast<float *>(out), out_pitch);
      break;
  }
  *err = cudaGetLastError();
  return *err == cudaSuccess ? 1 : -1;
}

}  // namespace ddk
