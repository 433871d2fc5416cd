// dd_dedisp_octet.cu -- staged dedispersion kernel for f16 and f32
// filterbanks.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]   (Sec. 2.1.1, brute-force equation),
// summed in FP32.
//
// Data flow per CTA (one 128-trial DM tile x one 256-sample time tile), per
// chunk of 16 channels:
//   1. one warp queues bulk copies (cp.async.bulk, the TMA engine) of each
//      channel's input window -- the "channel vector" of Sec. 2.4, sized by
//      the largest and smallest delay of the tile -- plus the chunk's plan
//      record into shared memory, signalling an mbarrier; copies run three
//      chunks ahead of the accumulation;
//   2. all threads build pattern rows: word i of a row holds, for one
//      relative-delay pattern of an octet of channels, the eight channels'
//      FP32 sum at output time i (dd_octet_plan.cpp); rows of chunk k+1 are
//      built while chunk k is accumulated (double buffer), with one CTA
//      barrier per chunk;
//   3. every thread adds, for each of its DM trials and output samples, one
//      row word per octet into an FP32 register accumulator: eight
//      channel-samples per add and per shared-memory word.
// The sum is blocked (eight channels, then octets in channel order) rather
// than sequential over channels; its rounding error is bounded by
// (8 + nchan/8) * 2^-24 * sum_c |I|, below the sequential bound.
// Waits on the mbarriers are bounded (globaltimer): on expiry the CTA records
// DD_ERR_DEVICE_TIMEOUT in the plan's status word, waits (bounded) for its
// own copies still in flight, and returns without writing output.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_device.cuh"
#include "dd_internal.h"
#include "dd_octet.h"

namespace {

using namespace ddo;
using namespace dddev;

struct OctetArgs {
  const uint8_t *block;
  int64_t pitch_bytes;  // bytes per channel row (multiple of 16)
  int32_t ndm;
  int64_t nsamp_out;
  float *out;
  int64_t out_pitch;  // elements between output rows (>= nsamp_out)
  const int32_t *recs;
  const int32_t *raw_meta;
  int32_t nchunks;
  int32_t nchan_pad;
  int32_t rec_words;
  int32_t raw_stride;  // elements
  int32_t prow_words;
  int32_t *status;     // plan's sticky device status word
  uint64_t timeout_ns;
  int32_t skip_copies;  // test hook: queue nothing, so the first wait runs out
};

// Input elements in shared memory: `raw` is the stored sample, `add` sums it
// into an FP32 value (f16 samples enter the sum exactly: add.f32.f16 widens
// the half before the single rounding of the add).
template <typename T>
struct Elem;
template <>
struct Elem<float> {
  using raw = float;
  static __device__ __forceinline__ float load(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
  }
  static __device__ __forceinline__ float widen(float x) { return x; }
  static __device__ __forceinline__ float add(float v, float x) { return v + x; }
};
template <>
struct Elem<__half> {
  using raw = unsigned short;
  static __device__ __forceinline__ unsigned short load(uint32_t addr) {
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
  }
  static __device__ __forceinline__ float widen(unsigned short x) {
    return __half2float(__ushort_as_half(x));
  }
  static __device__ __forceinline__ float add(float v, unsigned short x) {
    float r;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(x), "f"(v));
    return r;
  }
};

template <int OFF>
__device__ __forceinline__ float ldsf_off(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
  return v;
}
__device__ __forceinline__ void stsf(uint32_t addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// acc[j] += row word at a + 128 j, j = J..kTimesPerThread-1
template <int J>
struct AccRow {
  static __device__ __forceinline__ void run(float (&acc)[kTimesPerThread], uint32_t a) {
    acc[J] += ldsf_off<128 * J>(a);
    AccRow<J + 1>::run(acc, a);
  }
};
template <>
struct AccRow<kTimesPerThread> {
  static __device__ __forceinline__ void run(float (&)[kTimesPerThread], uint32_t) {}
};

// Queue the bulk copies of chunk `ch` (its record and the raw windows of its
// 8*opc channels) on mbarrier `bar`.  Called by all 32 lanes of one warp:
// lane s < 8*opc owns channel slot s and reads its window from the plan's
// table in global memory; lane 0 posts the byte count.
__device__ void issue_chunk(const OctetArgs &a, int opc, int esize, int tile, int64_t t_cta,
                            int ch, uint32_t bar, uint32_t rec_dst, uint32_t slots_dst,
                            int lane) {
  const int slots = kGroup * opc;
  uint32_t len = 0;
  int64_t off = 0;
  const int c = ch * slots + lane;
  if (lane < slots && c < a.nchan_pad) {
    const int32_t *m = a.raw_meta + (static_cast<int64_t>(tile) * a.nchan_pad + c) * 2;
    const int32_t start = __ldg(m), need = __ldg(m + 1);
    if (need > 0) {
      off = (t_cta + start) * esize;  // multiple of 16 bytes
      int64_t n = (static_cast<int64_t>(need) * esize + 15) & ~static_cast<int64_t>(15);
      if (off + n > a.pitch_bytes) n = a.pitch_bytes - off;  // stay inside the row
      len = n > 0 ? static_cast<uint32_t>(n) : 0u;
    }
  }
  uint32_t total = len;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if (lane == 0) {
    mbar_expect_tx(bar, total + static_cast<uint32_t>(a.rec_words) * 4);
    const int32_t *rec_src = a.recs + (static_cast<int64_t>(tile) * a.nchunks + ch) * a.rec_words;
    bulk_g2s(rec_dst, rec_src, static_cast<uint32_t>(a.rec_words) * 4, bar);
  }
  __syncwarp();
  if (len > 0) {
    const uint8_t *src = a.block + static_cast<int64_t>(c) * a.pitch_bytes + off;
    bulk_g2s(slots_dst + static_cast<uint32_t>(lane * a.raw_stride * esize), src, len, bar);
  }
}

// Build all pattern rows of an octet, one build unit (dd_octet.h) at a
// time: lane l builds row word first+l of every row -- per pattern the sum
// over the eight channels of the sample at that channel's shift.  Channel 0
// has the same sample in every pattern.  When every shift of the unit is 0
// or 1 (the common case), each lane loads both candidate samples of every
// channel once and selects per pattern; otherwise it loads each pattern's
// samples directly.
template <typename T>
__device__ __forceinline__ void build_unit(const int32_t *ud, uint32_t zero, uint32_t prow,
                                           int lane) {
  const int4 h0 = reinterpret_cast<const int4 *>(ud)[0];
  const uint32_t items = (static_cast<uint32_t>(h0.x) >> 20) & 63u;
  if (static_cast<uint32_t>(lane) >= items) return;
  const int4 h1 = reinterpret_cast<const int4 *>(ud)[1];
  const int4 h2 = reinterpret_cast<const int4 *>(ud)[2];
  const int4 h3 = reinterpret_cast<const int4 *>(ud)[3];
  const uint32_t npat = static_cast<uint32_t>(h0.y) & 0xffu;
  const uint32_t row_bytes = 4u * ((static_cast<uint32_t>(h0.y) >> 8) & 0xffffu);
  const uint32_t offw[4] = {static_cast<uint32_t>(h0.z), static_cast<uint32_t>(h0.w),
                            static_cast<uint32_t>(h1.x), static_cast<uint32_t>(h1.y)};
  const uint32_t codes[8] = {static_cast<uint32_t>(h1.z), static_cast<uint32_t>(h1.w),
                             static_cast<uint32_t>(h2.x), static_cast<uint32_t>(h2.y),
                             static_cast<uint32_t>(h2.z), static_cast<uint32_t>(h2.w),
                             static_cast<uint32_t>(h3.x), static_cast<uint32_t>(h3.y)};
  constexpr uint32_t es = sizeof(T);
  uint32_t addr[kGroup];
#pragma unroll
  for (int k = 0; k < kGroup; ++k)
    addr[k] = zero + es * (((offw[k / 2] >> (16 * (k & 1))) & 0xffffu) + lane);
  using E = Elem<T>;
  const float v0 = E::widen(E::load(addr[0]));
  uint32_t dst = prow + 4u * ((static_cast<uint32_t>(h0.x) & 0xfffffu) + lane);
  if ((static_cast<uint32_t>(h0.y) >> 30) & 1u) {
    typename E::raw r0[kGroup], r1[kGroup];
#pragma unroll
    for (int k = 1; k < kGroup; ++k)
      r0[k] = E::load(addr[k]), r1[k] = E::load(addr[k] + es);
#pragma unroll
    for (int p = 0; p < kMaxPatterns; ++p) {
      if (static_cast<uint32_t>(p) >= npat) break;
      const uint32_t code = codes[p >> 1] >> (16 * (p & 1));
      float v = v0;
#pragma unroll
      for (int k = 1; k < kGroup; ++k) v = E::add(v, ((code >> (2 * k)) & 1u) ? r1[k] : r0[k]);
      stsf(dst, v);
      dst += row_bytes;
    }
    return;
  }
#pragma unroll
  for (int p = 0; p < kMaxPatterns; ++p) {
    if (static_cast<uint32_t>(p) >= npat) break;
    const uint32_t code = codes[p >> 1] >> (16 * (p & 1));
    float v = v0;
#pragma unroll
    for (int k = 1; k < kGroup; ++k) v = E::add(v, E::load(addr[k] + es * ((code >> (2 * k)) & 3u)));
    stsf(dst, v);
    dst += row_bytes;
  }
}

template <typename T>
__device__ __forceinline__ void build_rows(const int32_t *rec, uint32_t zero, uint32_t prow,
                                           int units_off, int starts_off, int warp, int lane,
                                           int m0, int m1) {
  const int first = reinterpret_cast<const uint16_t *>(rec + starts_off)[warp];
  const int32_t *units = rec + units_off;
#pragma unroll 1
  for (int m = m0; m < m1; ++m) build_unit<T>(units + (first + m) * kUnitWords, zero, prow, lane);
}

template <typename T, int ND_THR>
__global__ void __launch_bounds__(kThreads, 1) dd_dedisperse_octet(OctetArgs a) {
  constexpr int ND_CTA = kDmGroups * ND_THR;
  constexpr int kUnitsOff = units_offset(ND_CTA);
  constexpr int kStartsOff = warp_start_offset(ND_CTA);
  constexpr int kEs = sizeof(T);
  constexpr int kOpc = kEs == 4 ? kOpcF32 : 2;  // octets per chunk
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x;  // DM tiles fastest: concurrent CTAs share input in L2
  const int64_t t_cta = static_cast<int64_t>(blockIdx.y) * kTimeTile;

  // shared-memory layout (dd_octet.h)
  const uint32_t bar0 = smem_addr(smem);
  auto tma_bar = [&](int m) { return bar0 + 8u * (m % kRawStages); };
  const uint32_t rec_bytes = static_cast<uint32_t>(a.rec_words) * 4;
  const uint32_t rec_off = kBarrierBytes;
  const uint32_t raw_off = rec_off + kRecStages * rec_bytes;
  const uint32_t zero_bytes = kZeroElems * kEs;
  const uint32_t stage_bytes = zero_bytes + kGroup * kOpc * static_cast<uint32_t>(a.raw_stride) * kEs;
  const uint32_t prow_off = raw_off + kRawStages * stage_bytes;
  const uint32_t prow_bytes = static_cast<uint32_t>(a.prow_words) * 4;
  auto rec_ptr = [&](int m) {
    return reinterpret_cast<const int32_t *>(smem + rec_off + (m % kRecStages) * rec_bytes);
  };
  auto rec_addr = [&](int m) { return bar0 + rec_off + (m % kRecStages) * rec_bytes; };
  auto zero_addr = [&](int m) { return bar0 + raw_off + (m % kRawStages) * stage_bytes; };
  auto prow_addr = [&](int m) { return bar0 + prow_off + (m % kRowStages) * prow_bytes; };

  for (int s = 0; s < kRawStages; ++s)
    for (uint32_t i = 4u * tid; i < zero_bytes; i += 4u * kThreads)
      *reinterpret_cast<uint32_t *>(smem + raw_off + s * stage_bytes + i) = 0u;
  if (tid == 0) {
    for (int b = 0; b < kRawStages; ++b) mbar_init(tma_bar(b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Pipeline (chunk m uses raw stage m%3, record stage m%4, row stage m%2):
  // iteration k starts with a CTA barrier (rows of chunk k built, chunk k-1
  // consumed); warp 0 then queues the copies of chunk k+3 into the stages of
  // chunks k (raw) and k-1 (record); every warp waits (bounded) for the copies
  // of chunk k+1 and builds its share of chunk k+1's rows after each octet of
  // chunk k it accumulates.  A copy wait that runs out is folded into the
  // next barrier (barrier-or), so every thread leaves the loop together.
  int issued = 0;
  if (warp == 0 && !a.skip_copies) {
    const int prefill = a.nchunks < kRawStages ? a.nchunks : kRawStages;
    for (int m = 0; m < prefill; ++m)
      issue_chunk(a, kOpc, kEs, tile, t_cta, m, tma_bar(m), rec_addr(m),
                  zero_addr(m) + zero_bytes, lane);
    issued = prefill;
  }
  float acc[ND_THR][kTimesPerThread];
#pragma unroll
  for (int i = 0; i < ND_THR; ++i)
#pragma unroll
    for (int j = 0; j < kTimesPerThread; ++j) acc[i][j] = 0.f;

  bool ok = warp_wait(tma_bar(0), 0, a.timeout_ns, lane);
  if (ok) {
    const int32_t *r0 = rec_ptr(0);
    const uint16_t *st = reinterpret_cast<const uint16_t *>(r0 + kStartsOff);
    build_rows<T>(r0, zero_addr(0), prow_addr(0), kUnitsOff, kStartsOff, warp, lane, 0,
                  st[warp + 1] - st[warp]);
  }

  bool aborted = false;
  for (int k = 0; k < a.nchunks; ++k) {
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    if (warp == 0 && k + kRawStages < a.nchunks && !a.skip_copies) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int m = k + kRawStages;
      issue_chunk(a, kOpc, kEs, tile, t_cta, m, tma_bar(m), rec_addr(m),
                  zero_addr(m) + zero_bytes, lane);
      issued = m + 1;
    }
    const bool next = k + 1 < a.nchunks;
    const int32_t *rec = rec_ptr(k);
    const int no = rec[2];
    const int32_t *A = rec + kRecHeader + warp * ND_THR;
    const uint32_t prow = prow_addr(k) + 4u * static_cast<uint32_t>(lane);
    const int32_t *rec_n = rec_ptr(k + 1);
    int nunits = -1;  // this warp's build units of chunk k+1, once its copies landed
    int m_done = 0;
#pragma unroll
    for (int o = 0; o < kOpc; ++o) {
      if (o < no) {
        int off[ND_THR];
#pragma unroll
        for (int i = 0; i < ND_THR; ++i) off[i] = A[o * ND_CTA + i];
#pragma unroll
        for (int i = 0; i < ND_THR; ++i)
          AccRow<0>::run(acc[i], prow + 4u * static_cast<uint32_t>(off[i]));
      }
      if (next && ok) {
        if (nunits < 0) {
          ok = warp_wait(tma_bar(k + 1), ((k + 1) / kRawStages) & 1, a.timeout_ns, lane);
          if (!ok) continue;  // reported at the next barrier
          const uint16_t *st = reinterpret_cast<const uint16_t *>(rec_n + kStartsOff);
          nunits = st[warp + 1] - st[warp];
        }
        const int m_to = (nunits * (o + 1) + kOpc - 1) / kOpc;
        if (m_to > m_done) {
          build_rows<T>(rec_n, zero_addr(k + 1), prow_addr(k + 1), kUnitsOff, kStartsOff, warp,
                        lane, m_done, m_to);
          m_done = m_to;
        }
      }
    }
  }
  if (!aborted && __syncthreads_or(!ok)) aborted = true;  // last chunk's copy wait

  if (aborted) {
    if (tid == 0) {
      atomicExch(a.status, 1);
      for (int m = issued > kRawStages ? issued - kRawStages : 0; m < issued; ++m)
        mbar_wait_bounded(tma_bar(m), (m / kRawStages) & 1, a.timeout_ns);
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < ND_THR; ++i) {
    const int d = tile * ND_CTA + warp * ND_THR + i;
    if (d >= a.ndm) continue;
    float *orow = a.out + static_cast<int64_t>(d) * a.out_pitch;
#pragma unroll
    for (int j = 0; j < kTimesPerThread; ++j) {
      const int64_t t = t_cta + lane + 32 * j;
      if (t < a.nsamp_out) orow[t] = acc[i][j];
    }
  }
}

template <typename T, int ND_THR>
int launch(const OctetArgs &a, const OctetDevice &q, int64_t nsamp_out, cudaStream_t stream,
           cudaError_t *err) {
  const dim3 grid(static_cast<unsigned>(q.tables.ntiles),
                  static_cast<unsigned>((nsamp_out + kTimeTile - 1) / kTimeTile));
  const int smem = q.tables.smem_bytes;
  *err = cudaFuncSetAttribute(dd_dedisperse_octet<T, ND_THR>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (*err == cudaSuccess) dd_dedisperse_octet<T, ND_THR><<<grid, kThreads, smem, stream>>>(a);
  if (*err == cudaSuccess) *err = cudaGetLastError();
  return *err == cudaSuccess ? 1 : -1;
}

}  // namespace

namespace ddk {

bool octet_supported(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out) {
  if (!p->octet || p->dtype == DD_U8) return false;
  if ((nsamp_out + kTimeTile - 1) / kTimeTile > 65535) return false;  // grid.y limit
  const int64_t pitch_bytes = pitch * elem_size(p->dtype);
  return (reinterpret_cast<uintptr_t>(block) & 15) == 0 && (pitch_bytes & 15) == 0;
}

int launch_dedisperse_octet(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                            void *out, int64_t out_pitch, cudaStream_t stream, cudaError_t *err) {
  const OctetDevice &q = *p->octet;
  OctetArgs a;
  a.block = static_cast<const uint8_t *>(block);
  a.pitch_bytes = pitch * elem_size(p->dtype);
  a.ndm = p->ndm;
  a.nsamp_out = nsamp_out;
  a.out = static_cast<float *>(out);
  a.out_pitch = out_pitch;
  a.recs = q.d_recs;
  a.raw_meta = q.d_raw_meta;
  a.nchunks = q.tables.nchunks;
  a.nchan_pad = q.tables.nchan_pad;
  a.rec_words = q.tables.rec_words;
  a.raw_stride = q.tables.raw_stride;
  a.prow_words = q.tables.prow_words;
  a.status = p->d_error;
  a.timeout_ns = p->wait_timeout_ns;
  a.skip_copies = p->debug_skip_copies;
  const bool wide = q.tables.nd_thr == kNdThr;
  if (p->dtype == DD_F32)
    return wide ? launch<float, kNdThr>(a, q, nsamp_out, stream, err)
                : launch<float, kNdThr / 2>(a, q, nsamp_out, stream, err);
  return wide ? launch<__half, kNdThr>(a, q, nsamp_out, stream, err)
              : launch<__half, kNdThr / 2>(a, q, nsamp_out, stream, err);
}

}  // namespace ddk
