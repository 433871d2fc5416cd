// dd_dedisp_direct.cu -- plain-load dedispersion kernel (any alignment, any
// pitch): the layout-agnostic path of dd_execute.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]  (Sec. 2.1.1, brute-force equation).
// The grid maps onto the output (DM tile, time tile) space; each thread owns
// one output sample for 16 (or, for small outputs, 4) consecutive DM trials,
// with one register accumulator per trial (the thesis's Sec. 2.4 layout),
// and reads the input through the L1/L2 caches, several channels' samples in
// flight at once (direct_sums).  Delays of a group of channels for the CTA's
// DM tile are staged in shared memory (channel/DM order keeps that load
// coalesced, Sec. 3.4).
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dd_direct_dev.cuh"
#include "dd_internal.h"

namespace {

static_assert(kDirectThreads == ddk::kOctetTileSamples,
              "a CTA's time tile is one per-tile statistics tile");

// NDMS DM trials per thread (16, or 4 for small outputs, so that the grid
// covers the GPU).  With tilestats (float rows only), the CTA's 256 outputs
// of each of its trials -- one statistics tile -- give that tile's partials
// (tile_partials).
template <typename T, int NDMS>
__global__ void __launch_bounds__(kDirectThreads)
dd_dedisperse_direct(const T *__restrict__ in, int64_t pitch, const int32_t *__restrict__ delays,
                     int32_t nchan, int32_t ndm, int64_t nsamp_out,
                     typename DirectTraits<T>::acc_t *__restrict__ out, int64_t out_pitch,
                     float4 *__restrict__ tilestats) {
  using acc_t = typename DirectTraits<T>::acc_t;
  __shared__ int32_t s_delay[kDelayChans][NDMS];
  const int64_t t = static_cast<int64_t>(blockIdx.x) * kDirectThreads + threadIdx.x;
  const int d0 = blockIdx.y * NDMS;
  const bool live = t < nsamp_out;
  acc_t acc[NDMS];
  direct_sums<T, NDMS>(in, pitch, delays, nchan, ndm, d0, t, live, acc, s_delay);
  if (live) {
#pragma unroll
    for (int j = 0; j < NDMS; ++j)
      if (d0 + j < ndm) out[static_cast<int64_t>(d0 + j) * out_pitch + t] = acc[j];
  }
  if constexpr (!std::is_same<acc_t, int32_t>::value) {
    __shared__ PartialScratch<NDMS> s_part;
    if (tilestats) {
      const int64_t ntiles = (nsamp_out + kDirectThreads - 1) / kDirectThreads;
      tile_partials<NDMS>(acc, live, d0, ndm, ntiles, blockIdx.x, tilestats, s_part);
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

int direct_trials_per_thread(const dd_plan *p, int64_t nsamp_out) {
  // 16 trials per thread unless that leaves fewer than two CTAs per SM
  const int64_t tiles = (nsamp_out + kDirectThreads - 1) / kDirectThreads;
  return tiles * ((p->ndm + 15) / 16) < 2 * static_cast<int64_t>(p->sm_count) ? 4 : 16;
}

int launch_dedisperse_direct(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                             void *out, int64_t out_pitch, float4 *tilestats, cudaStream_t stream,
                             cudaError_t *err) {
  const int ndms = direct_trials_per_thread(p, nsamp_out);
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
