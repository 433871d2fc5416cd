// dd_dedisp_quad.cu -- staged dedispersion kernel for u8 filterbanks.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]   (Sec. 2.1.1, brute-force equation),
// exact in int32.
//
// Data flow per CTA (one DM tile x one 512-sample time tile), per chunk of
// 16 channels:
//   1. one warp queues bulk copies (cp.async.bulk, the TMA engine) of each
//      channel's input window -- the "channel vector" of Sec. 2.4, sized by
//      the largest and smallest delay of the tile -- plus the chunk's plan
//      record into shared memory, signalling an mbarrier; copies run three
//      chunks ahead of the accumulation (triple-buffered windows);
//   2. all threads interleave the four channels of every quad into pattern
//      rows: word i of a row holds the four channels' samples that one
//      relative-delay pattern adds at one output time (dd_quad_plan.cpp);
//      rows of chunk k+1 are built while chunk k is accumulated (double
//      buffer), with one CTA barrier per chunk;
//   3. every thread adds, for each of its DM trials and output samples, one
//      32-bit row word with a 4-way byte dot product (dp4a, weights 1) into
//      an int32 register accumulator: four channel-adds per instruction and
//      one shared-memory word per four adds.
// Waits on the mbarriers are bounded (globaltimer): on expiry the CTA records
// DD_ERR_DEVICE_TIMEOUT in the plan's status word, waits (bounded) for its
// own copies still in flight, and returns without writing output.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"
#include "dd_quad.h"

namespace {

using namespace ddq;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait that may suspend the thread for up to ~kSuspendNs while the phase
// is incomplete (it resumes as soon as the phase completes), so that waiting
// warps do not take issue slots from working ones.
constexpr uint32_t kSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "n"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// Wait on an mbarrier phase for at most timeout_ns.
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  while (!mbar_try_wait_sleep(bar, parity))
    if (global_timer() - t0 > timeout_ns) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// Shared load with a compile-time byte offset folded into the instruction.
template <int OFF>
__device__ __forceinline__ uint32_t lds32_off(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
  return v;
}

__device__ __forceinline__ uint32_t dp4a_ones(uint32_t a, uint32_t acc) {
  uint32_t r;
  asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(0x01010101u), "r"(acc));
  return r;
}

template <int J>
struct Acc8 {
  // acc[j] += dp4a(word at base + 128 j) for j = J..7
  static __device__ __forceinline__ void run(int (&acc)[kTimesPerThread], uint32_t base) {
    acc[J] = static_cast<int>(dp4a_ones(lds32_off<128 * J>(base), static_cast<uint32_t>(acc[J])));
    Acc8<J + 1>::run(acc, base);
  }
};
template <>
struct Acc8<kTimesPerThread> {
  static __device__ __forceinline__ void run(int (&)[kTimesPerThread], uint32_t) {}
};

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                       uint32_t d) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}

struct QuadArgs {
  const uint8_t *block;
  int64_t pitch;  // bytes per channel row (multiple of 16)
  int32_t ndm;
  int64_t nsamp_out;
  int32_t *out;
  const int32_t *recs;
  const int32_t *raw_meta;
  int32_t nchunks;
  int32_t nchan_pad;
  int32_t rec_words;
  int32_t raw_stride;
  int32_t prow_words;
  int32_t *status;  // plan's sticky device status word
  uint64_t timeout_ns;
  int32_t skip_copies;  // test hook: queue nothing, so the first wait runs out
};

// Queue the bulk copies of chunk `ch` (its record and the raw windows of its
// 4*kQuadsPerChunk channels) on mbarrier `bar`.  Called by all 32 lanes of
// one warp: lane s < 16 owns channel slot s; lane 0 posts the byte count.
__device__ void issue_chunk(const QuadArgs &a, const int32_t *meta_s, int tile, int64_t t_cta,
                            int ch, uint32_t bar, uint32_t rec_dst, uint32_t raw_dst, int lane) {
  constexpr int kSlots = 4 * kQuadsPerChunk;
  uint32_t len = 0;
  const int c = ch * kSlots + lane;
  if (lane < kSlots && c < a.nchan_pad) {
    const int32_t start = meta_s[2 * c], need = meta_s[2 * c + 1];
    if (need > 0) {
      const int64_t off = t_cta + start;                     // multiple of 16
      int64_t n = (static_cast<int64_t>(need) + 15) & ~static_cast<int64_t>(15);
      if (off + n > a.pitch) n = a.pitch - off;              // stay inside the row
      len = static_cast<uint32_t>(n);
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
    const uint8_t *src = a.block + static_cast<int64_t>(c) * a.pitch + t_cta + meta_s[2 * c];
    bulk_g2s(raw_dst + lane * a.raw_stride, src, len, bar);
  }
}

// Interleave the four channels of a quad into all of its pattern rows, one
// build unit (dd_quad.h) at a time: lane l builds item first+l (4 output
// samples) of every row.  Per channel it loads the three aligned words that
// hold the earliest needed sample and the next 8 bytes -- enough for every
// pattern, whose first samples differ by at most 4 -- then for each pattern
// funnels out the 4 samples at that pattern's byte shift; a 4x4 byte transpose
// turns the four channels' words into four row words.
__device__ __forceinline__ void build_unit(const int32_t *ud, uint32_t raw, uint32_t prow,
                                           int lane) {
  const int4 d0 = reinterpret_cast<const int4 *>(ud)[0];
  const int4 d1 = reinterpret_cast<const int4 *>(ud)[1];
  const uint32_t items = (static_cast<uint32_t>(d0.z) >> 20) & 63u;
  if (static_cast<uint32_t>(lane) >= items) return;
  const uint32_t npat = static_cast<uint32_t>(d0.z) >> 26;
  const uint32_t off[4] = {static_cast<uint32_t>(d0.x) & 0xffffu, static_cast<uint32_t>(d0.x) >> 16,
                           static_cast<uint32_t>(d0.y) & 0xffffu, static_cast<uint32_t>(d0.y) >> 16};
  uint32_t w0[4], w1[4], w2[4];
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    const bool pad = off[ch] == 0xffffu;                         // padding channel: zeros
    const uint32_t w = raw + (pad ? 0u : off[ch]) + 4u * lane;  // always in bounds
    w0[ch] = pad ? 0u : lds32(w);
    w1[ch] = pad ? 0u : lds32_off<4>(w);
    w2[ch] = pad ? 0u : lds32_off<8>(w);
  }
  const uint32_t codes[4] = {static_cast<uint32_t>(d1.x), static_cast<uint32_t>(d1.y),
                             static_cast<uint32_t>(d1.z), static_cast<uint32_t>(d1.w)};
  uint32_t dst = prow + 4u * (static_cast<uint32_t>(d0.z) & 0xfffffu) + 16u * lane;
  const uint32_t row_bytes = 4u * static_cast<uint32_t>(d0.w);
#pragma unroll
  for (int p = 0; p < kMaxPatterns; ++p) {
    if (static_cast<uint32_t>(p) >= npat) break;
    const uint32_t code = (codes[p >> 1] >> (12 * (p & 1))) & 0xfffu;
    uint32_t v[4];
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      const uint32_t sh = (code >> (3 * ch)) & 7u;  // 0..7 bytes into w0:w1:w2
      const uint32_t lo = sh >= 4u ? w1[ch] : w0[ch];
      const uint32_t hi = sh >= 4u ? w2[ch] : w1[ch];
      v[ch] = prmt(lo, hi, 0x3210u + 0x1111u * (sh & 3u));
    }
    const uint32_t lo01 = prmt(v[0], v[1], 0x5140u), hi01 = prmt(v[0], v[1], 0x7362u);
    const uint32_t lo23 = prmt(v[2], v[3], 0x5140u), hi23 = prmt(v[2], v[3], 0x7362u);
    sts128(dst, prmt(lo01, lo23, 0x5410u), prmt(lo01, lo23, 0x7632u), prmt(hi01, hi23, 0x5410u),
           prmt(hi01, hi23, 0x7632u));
    dst += row_bytes;
  }
}

// This warp's build units m0 .. m1-1 (counted within its own list).
__device__ __forceinline__ void build_rows(const int32_t *rec, uint32_t raw, uint32_t prow,
                                           int units_off, int warp, int lane, int m0, int m1,
                                           int starts_off) {
  const int first = reinterpret_cast<const uint16_t *>(rec + starts_off)[warp];
  const int32_t *units = rec + units_off;
#pragma unroll 1
  for (int m = m0; m < m1; ++m) build_unit(units + (first + m) * kUnitWords, raw, prow, lane);
}

// Build units this warp takes in a chunk.
__device__ __forceinline__ int warp_segments(const int32_t *rec, int warp, int starts_off) {
  const uint16_t *starts = reinterpret_cast<const uint16_t *>(rec + starts_off);
  return starts[warp + 1] - starts[warp];
}

// Warp-wide bounded wait on an mbarrier phase: lane 0 waits (sleeping in
// try_wait) until the phase completes or timeout_ns passes; then every lane
// acquires the completed phase.  Returns false if the wait gave up.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, uint64_t timeout_ns,
                                          int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait_bounded(bar, parity, timeout_ns) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) mbar_try_wait(bar, parity);
  return ok != 0;
}

template <int ND_THR>
__global__ void __launch_bounds__(kThreads, 1) dd_dedisperse_quad_u8(QuadArgs a) {
  constexpr int ND_CTA = kDmGroups * ND_THR;
  constexpr int kSegsOff = units_offset(ND_CTA);
  constexpr int kStartsOff = warp_start_offset(ND_CTA);
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tg = warp & (kTimeGroups - 1);
  const int dg = warp / kTimeGroups;
  // DM tiles vary fastest across the grid, so the CTAs resident at any time
  // cover a narrow span of input samples for all DM tiles and share the
  // input windows through L2 instead of re-reading them from HBM.
  const int tile = blockIdx.x;
  const int64_t t_cta = static_cast<int64_t>(blockIdx.y) * kTimeTile;

  // shared-memory layout (dd_quad.h): copy mbarriers, raw window table,
  // records, raw window buffers, pattern-row buffers
  const uint32_t bar0 = smem_addr(smem);
  auto tma_bar = [&](int m) { return bar0 + 8u * (m % kRawStages); };
  int32_t *meta_s = reinterpret_cast<int32_t *>(smem + kBarrierBytes);
  const uint32_t meta_bytes = static_cast<uint32_t>((a.nchan_pad * 8 + 15) / 16 * 16);
  const uint32_t rec_bytes = static_cast<uint32_t>(a.rec_words) * 4;
  const uint32_t rec_off = kBarrierBytes + meta_bytes;
  const uint32_t raw_off = rec_off + kRecStages * rec_bytes;
  const uint32_t raw_bytes = 4u * kQuadsPerChunk * static_cast<uint32_t>(a.raw_stride);
  const uint32_t prow_off = raw_off + kRawStages * raw_bytes;
  const uint32_t prow_bytes = static_cast<uint32_t>(a.prow_words) * 4;
  auto rec_ptr = [&](int m) {
    return reinterpret_cast<const int32_t *>(smem + rec_off + (m % kRecStages) * rec_bytes);
  };
  auto rec_addr = [&](int m) { return bar0 + rec_off + (m % kRecStages) * rec_bytes; };
  auto raw_addr = [&](int m) { return bar0 + raw_off + (m % kRawStages) * raw_bytes; };
  auto prow_addr = [&](int m) { return bar0 + prow_off + (m % kRowStages) * prow_bytes; };

  const int32_t *meta_g = a.raw_meta + static_cast<int64_t>(tile) * a.nchan_pad * 2;
  for (int i = tid; i < 2 * a.nchan_pad; i += kThreads) meta_s[i] = meta_g[i];
  if (tid == 0) {
    for (int b = 0; b < kRawStages; ++b) mbar_init(tma_bar(b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Pipeline (chunk m uses raw stage m%3, record stage m%4, row stage m%2):
  // iteration k starts with a CTA barrier (rows of chunk k built, chunk k-1
  // consumed); warp 0 then queues the copies of chunk k+3 into the stages of
  // chunks k (raw) and k-1 (record); every warp waits (bounded) for the copies
  // of chunk k+1 and builds its share of chunk k+1's rows, spread over the
  // accumulation of chunk k.  A copy wait that runs out is folded into the
  // next barrier (barrier-or), so every thread leaves the loop together.
  int issued = 0;  // chunks queued (warp 0)
  if (warp == 0 && !a.skip_copies) {
    const int prefill = a.nchunks < kRawStages ? a.nchunks : kRawStages;
    for (int m = 0; m < prefill; ++m)
      issue_chunk(a, meta_s, tile, t_cta, m, tma_bar(m), rec_addr(m), raw_addr(m), lane);
    issued = prefill;
  }

  int acc[ND_THR][kTimesPerThread];
#pragma unroll
  for (int i = 0; i < ND_THR; ++i)
#pragma unroll
    for (int j = 0; j < kTimesPerThread; ++j) acc[i][j] = 0;
  const uint32_t my_word = static_cast<uint32_t>(tg * 32 * kTimesPerThread + lane);

  bool ok = warp_wait(tma_bar(0), 0, a.timeout_ns, lane);
  if (ok)
    build_rows(rec_ptr(0), raw_addr(0), prow_addr(0), kSegsOff, warp, lane, 0,
               warp_segments(rec_ptr(0), warp, kStartsOff), kStartsOff);

  bool aborted = false;
  for (int k = 0; k < a.nchunks; ++k) {
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    if (warp == 0 && k + kRawStages < a.nchunks && !a.skip_copies) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int m = k + kRawStages;
      issue_chunk(a, meta_s, tile, t_cta, m, tma_bar(m), rec_addr(m), raw_addr(m), lane);
      issued = m + 1;
    }
    // accumulate chunk k (four channels per dp4a) and build this warp's share
    // of chunk k+1's rows after each quad; the copies of chunk k+1 are waited
    // for (bounded) just before the first build step, and each quad's offset
    // table is fetched one quad ahead
    const bool next = k + 1 < a.nchunks;
    const int32_t *rec = rec_ptr(k);
    const int nq = rec[2];
    const int32_t *A = rec + kRecHeader + dg * ND_THR;  // 16-byte aligned
    const uint32_t prow = prow_addr(k);
    const int32_t *rec_n = rec_ptr(k + 1);
    int nseg_w = -1;  // build units of chunk k+1 for this warp, once its copies landed
    int m_done = 0;
    int4 a_next[ND_THR / 4];
#pragma unroll
    for (int i4 = 0; i4 < ND_THR / 4; ++i4) a_next[i4] = reinterpret_cast<const int4 *>(A)[i4];
#pragma unroll 1
    for (int q = 0; q < kQuadsPerChunk; ++q) {
      if (q < nq) {
        int4 a_cur[ND_THR / 4];
#pragma unroll
        for (int i4 = 0; i4 < ND_THR / 4; ++i4) a_cur[i4] = a_next[i4];
        if (q + 1 < nq) {
#pragma unroll
          for (int i4 = 0; i4 < ND_THR / 4; ++i4)
            a_next[i4] = reinterpret_cast<const int4 *>(A + (q + 1) * ND_CTA)[i4];
        }
#pragma unroll
        for (int i4 = 0; i4 < ND_THR / 4; ++i4) {
          const int off[4] = {a_cur[i4].x, a_cur[i4].y, a_cur[i4].z, a_cur[i4].w};
#pragma unroll
          for (int ii = 0; ii < 4; ++ii)
            Acc8<0>::run(acc[4 * i4 + ii], prow + 4u * (static_cast<uint32_t>(off[ii]) + my_word));
        }
      }
      if (next && ok) {
        if (nseg_w < 0) {
          ok = warp_wait(tma_bar(k + 1), ((k + 1) / kRawStages) & 1, a.timeout_ns, lane);
          if (!ok) continue;  // reported at the next barrier
          nseg_w = warp_segments(rec_n, warp, kStartsOff);
        }
        const int m_to = (nseg_w * (q + 1) + kQuadsPerChunk - 1) / kQuadsPerChunk;
        if (m_to > m_done) {
          build_rows(rec_n, raw_addr(k + 1), prow_addr(k + 1), kSegsOff, warp, lane, m_done, m_to,
                     kStartsOff);
          m_done = m_to;
        }
      }
    }
  }
  if (!aborted && __syncthreads_or(!ok)) aborted = true;  // last chunk's copy wait

  if (aborted) {
    // a bounded wait ran out: record it; warp 0 waits, bounded, for the
    // copies it queued that may still be in flight (the last kRawStages
    // queued, each on its own barrier) before the CTA leaves
    if (tid == 0) {
      atomicExch(a.status, 1);
      for (int m = issued > kRawStages ? issued - kRawStages : 0; m < issued; ++m)
        mbar_wait_bounded(tma_bar(m), (m / kRawStages) & 1, a.timeout_ns);
    }
    return;
  }

#pragma unroll
  for (int i = 0; i < ND_THR; ++i) {
    const int d = tile * ND_CTA + dg * ND_THR + i;
    if (d >= a.ndm) continue;
    int32_t *orow = a.out + static_cast<int64_t>(d) * a.nsamp_out;
#pragma unroll
    for (int j = 0; j < kTimesPerThread; ++j) {
      const int64_t t = t_cta + my_word + 32 * j;
      if (t < a.nsamp_out) orow[t] = acc[i][j];
    }
  }
}

}  // namespace

namespace ddk {

bool quad_supported(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out) {
  if (!p->quad || p->dtype != DD_U8) return false;
  if ((nsamp_out + kTimeTile - 1) / kTimeTile > 65535) return false;  // grid.y limit
  return (reinterpret_cast<uintptr_t>(block) & 15) == 0 && (pitch & 15) == 0;
}

int launch_dedisperse_quad(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                           void *out, cudaStream_t stream, cudaError_t *err) {
  const QuadDevice &q = *p->quad;
  QuadArgs a;
  a.block = static_cast<const uint8_t *>(block);
  a.pitch = pitch;
  a.ndm = p->ndm;
  a.nsamp_out = nsamp_out;
  a.out = static_cast<int32_t *>(out);
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
  const dim3 grid(static_cast<unsigned>(q.tables.ntiles),
                  static_cast<unsigned>((nsamp_out + kTimeTile - 1) / kTimeTile));
  const int smem = q.tables.smem_bytes;
  if (q.tables.nd_thr == kNdThr) {
    *err = cudaFuncSetAttribute(dd_dedisperse_quad_u8<kNdThr>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (*err == cudaSuccess) dd_dedisperse_quad_u8<kNdThr><<<grid, kThreads, smem, stream>>>(a);
  } else {
    *err = cudaFuncSetAttribute(dd_dedisperse_quad_u8<kNdThr / 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (*err == cudaSuccess) dd_dedisperse_quad_u8<kNdThr / 2><<<grid, kThreads, smem, stream>>>(a);
  }
  if (*err == cudaSuccess) *err = cudaGetLastError();
  return *err == cudaSuccess ? 1 : -1;
}

}  // namespace ddk
