// dd_dedisp_quad.cu -- staged dedispersion kernel for u8 filterbanks.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]   (Sec. 2.1.1, brute-force equation),
// exact in int32.
//
// Data flow per CTA (one DM tile x one 512-sample time tile), per chunk of
// 16 channels:
//   1. one thread queues bulk copies (cp.async.bulk, the TMA engine) of each
//      channel's input window -- the "channel vector" of Sec. 2.2, sized by
//      the largest and smallest delay of the tile -- plus the chunk's plan
//      record into shared memory, signalling an mbarrier; the copies for the
//      next chunk are in flight while this one is used (double buffer);
//   2. all threads interleave the four channels of every quad into pattern
//      rows: word i of a row holds the four channels' samples that one
//      relative-delay pattern adds at one output time (dd_quad_plan.cpp);
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

// Spin on an mbarrier phase for at most timeout_ns.
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
  const uint64_t t0 = global_timer();
  while (!mbar_try_wait(bar, parity))
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
  int32_t *status;  // plan's sticky device status word
  uint64_t timeout_ns;
  int32_t skip_copies;  // test hook: queue nothing, so the first wait runs out
};

// Queue the bulk copies of chunk `ch` into buffer `buf` (one thread).
__device__ void issue_chunk(const QuadArgs &a, int tile, int64_t t_cta, int ch, uint32_t bar,
                            uint32_t rec_dst, uint32_t raw_dst) {
  const int32_t *rec_src = a.recs + (static_cast<int64_t>(tile) * a.nchunks + ch) * a.rec_words;
  const int32_t *meta = a.raw_meta + (static_cast<int64_t>(tile) * a.nchan_pad + ch * 4 * kQuadsPerChunk) * 2;
  uint32_t len[4 * kQuadsPerChunk];
  uint32_t total = static_cast<uint32_t>(a.rec_words) * 4;
  for (int s = 0; s < 4 * kQuadsPerChunk; ++s) {
    len[s] = 0;
    if (ch * 4 * kQuadsPerChunk + s >= a.nchan_pad) continue;
    const int32_t start = meta[2 * s], need = meta[2 * s + 1];
    if (need <= 0) continue;
    const int64_t off = t_cta + start;                       // multiple of 16
    int64_t n = (static_cast<int64_t>(need) + 15) & ~static_cast<int64_t>(15);
    if (off + n > a.pitch) n = a.pitch - off;                // stay inside the row
    len[s] = static_cast<uint32_t>(n);
    total += len[s];
  }
  mbar_expect_tx(bar, total);
  bulk_g2s(rec_dst, rec_src, static_cast<uint32_t>(a.rec_words) * 4, bar);
  for (int s = 0; s < 4 * kQuadsPerChunk; ++s) {
    if (len[s] == 0) continue;
    const int c = ch * 4 * kQuadsPerChunk + s;
    const uint8_t *src = a.block + static_cast<int64_t>(c) * a.pitch + t_cta + meta[2 * s];
    bulk_g2s(raw_dst + s * a.raw_stride, src, len[s], bar);
  }
}

template <int ND_THR>
__global__ void __launch_bounds__(kThreads, 1) dd_dedisperse_quad_u8(QuadArgs a) {
  constexpr int ND_CTA = kDmGroups * ND_THR;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tg = warp & (kTimeGroups - 1);
  const int dg = warp / kTimeGroups;
  const int tile = blockIdx.y;
  const int64_t t_cta = static_cast<int64_t>(blockIdx.x) * kTimeTile;

  const uint32_t bar0 = smem_addr(smem);
  const uint32_t rec0 = bar0 + 16;
  const uint32_t rec_bytes = static_cast<uint32_t>(a.rec_words) * 4;
  const uint32_t raw0 = rec0 + 2 * rec_bytes;
  const uint32_t raw_bytes = 4u * kQuadsPerChunk * static_cast<uint32_t>(a.raw_stride);
  const uint32_t prow = raw0 + 2 * raw_bytes;

  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = -1;
    if (!a.skip_copies) {
      issue_chunk(a, tile, t_cta, 0, bar0, rec0, raw0);
      if (a.nchunks > 1) issue_chunk(a, tile, t_cta, 1, bar0 + 8, rec0 + rec_bytes, raw0 + raw_bytes);
    }
  }
  __syncthreads();

  int acc[ND_THR][kTimesPerThread];
#pragma unroll
  for (int i = 0; i < ND_THR; ++i)
#pragma unroll
    for (int j = 0; j < kTimesPerThread; ++j) acc[i][j] = 0;

  const uint32_t my_word = static_cast<uint32_t>(tg * 32 * kTimesPerThread + lane);

  for (int k = 0; k < a.nchunks; ++k) {
    const int buf = k & 1;
    const uint32_t bar = bar0 + 8 * buf;
    const uint32_t parity = (k >> 1) & 1;
    // thread 0 alone spins (bounded); the outcome is made CTA-uniform
    if (tid == 0 && !mbar_wait_bounded(bar, parity, a.timeout_ns)) {
      s_abort = k;
      atomicExch(a.status, 1);
    }
    __syncthreads();
    if (s_abort >= 0) break;
    mbar_try_wait(bar, parity);  // phase complete: acquire the copied bytes

    // ---- build pattern rows from the raw channel windows
    const int32_t *rec = reinterpret_cast<const int32_t *>(smem + 16 + buf * rec_bytes);
    const int nrows = rec[0];
    const int items = rec[1];
    const int nq = rec[2];
    const int32_t *rows = rec + kRecHeader + kQuadsPerChunk * ND_CTA;
    const uint32_t raw = raw0 + buf * raw_bytes;
    int r = 0;
    for (int it = tid; it < items; it += kThreads) {
      while (r + 1 < nrows && it >= rows[(r + 1) * kRowWords + 2]) ++r;
      const int32_t *row = rows + r * kRowWords;
      const int i4 = it - row[2];
      const uint32_t slot = raw + static_cast<uint32_t>(row[3] * 4) * a.raw_stride;
      uint32_t v[4];
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        const int32_t o = row[4 + ch];
        if (o < 0) {
          v[ch] = 0;
        } else {
          const uint32_t pos = static_cast<uint32_t>(o + 4 * i4);
          const uint32_t w = slot + ch * a.raw_stride + (pos & ~3u);
          v[ch] = prmt(lds32(w), lds32(w + 4), 0x3210u + 0x1111u * (pos & 3u));
        }
      }
      // 4x4 byte transpose: word j = {ch0[j], ch1[j], ch2[j], ch3[j]}
      const uint32_t lo01 = prmt(v[0], v[1], 0x5140u), hi01 = prmt(v[0], v[1], 0x7362u);
      const uint32_t lo23 = prmt(v[2], v[3], 0x5140u), hi23 = prmt(v[2], v[3], 0x7362u);
      sts128(prow + 4u * static_cast<uint32_t>(row[0] + 4 * i4), prmt(lo01, lo23, 0x5410u),
             prmt(lo01, lo23, 0x7632u), prmt(hi01, hi23, 0x5410u), prmt(hi01, hi23, 0x7632u));
    }
    __syncthreads();  // pattern rows ready

    // ---- accumulate: four channels per dp4a
    const int32_t *A = rec + kRecHeader + dg * ND_THR;  // 16-byte aligned
#pragma unroll 1
    for (int q = 0; q < nq; ++q) {
      const int4 *A4 = reinterpret_cast<const int4 *>(A + q * ND_CTA);
#pragma unroll
      for (int i4 = 0; i4 < ND_THR / 4; ++i4) {
        const int4 a4 = A4[i4];
        const int off[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
          const int i = 4 * i4 + ii;
          const uint32_t base = prow + 4u * (static_cast<uint32_t>(off[ii]) + my_word);
#pragma unroll
          for (int j = 0; j < kTimesPerThread; ++j)
            acc[i][j] = static_cast<int>(
                __dp4a(lds32(base + 128u * j), 0x01010101u, static_cast<uint32_t>(acc[i][j])));
        }
      }
    }
    __syncthreads();  // record, raw window and pattern rows of buffer `buf` consumed

    if (tid == 0 && k + 2 < a.nchunks && !a.skip_copies) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_chunk(a, tile, t_cta, k + 2, bar, rec0 + buf * rec_bytes, raw);
    }
  }

  if (s_abort >= 0) {
    // wait (bounded) for this CTA's own copies still in flight: chunks k and
    // k+1 were queued when chunk k's wait ran out; then leave
    if (tid == 0 && !a.skip_copies) {
      for (int m = s_abort; m < a.nchunks && m <= s_abort + 1; ++m)
        mbar_wait_bounded(bar0 + 8 * (m & 1), (m >> 1) & 1, a.timeout_ns);
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

bool quad_supported(const dd_plan *p, const void *block, int64_t pitch) {
  if (!p->quad || p->dtype != DD_U8) return false;
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
  a.status = p->d_error;
  a.timeout_ns = p->wait_timeout_ns;
  a.skip_copies = p->debug_skip_copies;
  const dim3 grid(static_cast<unsigned>((nsamp_out + kTimeTile - 1) / kTimeTile),
                  static_cast<unsigned>(q.tables.ntiles));
  const int smem = q.tables.smem_bytes;
  if (q.tables.nd_thr == 16) {
    *err = cudaFuncSetAttribute(dd_dedisperse_quad_u8<16>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (*err == cudaSuccess) dd_dedisperse_quad_u8<16><<<grid, kThreads, smem, stream>>>(a);
  } else {
    *err = cudaFuncSetAttribute(dd_dedisperse_quad_u8<8>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (*err == cudaSuccess) dd_dedisperse_quad_u8<8><<<grid, kThreads, smem, stream>>>(a);
  }
  if (*err == cudaSuccess) *err = cudaGetLastError();
  return *err == cudaSuccess ? 1 : -1;
}

}  // namespace ddk
