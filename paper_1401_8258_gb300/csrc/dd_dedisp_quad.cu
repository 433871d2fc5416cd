// dd_dedisp_quad.cu -- staged dedispersion kernel for u8 filterbanks.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]   (Sec. 2.1.1, brute-force equation),
// exact in integers.
//
// Data flow per CTA (one DM tile x one 512-sample time tile, taken as 256
// sample pairs (t, t + 256)), per chunk of 16 channels, in two warp roles
// that hand chunks to each other through named barriers:
//   1. a building warp queues bulk copies (cp.async.bulk, the TMA engine) of
//      each channel's input window -- the "channel vector" of Sec. 2.4,
//      sized by the largest and smallest delay of the tile -- plus the
//      chunk's plan record into shared memory, signalling an mbarrier,
//      1 to 3 chunks ahead of the chunk being built (the staging depth, a
//      template parameter picked per plan by the autotuner);
//   2. 12 building warps build pattern rows: word i of a row holds, for one
//      relative-delay pattern of a quad of channels, the four channels' sum
//      at pair i as two 16-bit halves (dd_quad_plan.cpp); they build chunk
//      k+1 while the accumulating warps add chunk k (double-buffered rows);
//   3. 16 accumulating warps add, for each of their DM trials and sample
//      pairs, the row words of two quads to a packed accumulator with one
//      three-input integer add: 16 channel-samples per instruction and 8 per
//      32-bit shared-memory word.  Every 64 quads the 16-bit halves are
//      drained into 32-bit sums kept in tensor memory (tcgen05.st /
//      tcgen05.ld), which spares the 64 registers per thread they would take.
// Waits on the mbarriers are bounded (globaltimer): on expiry the CTA records
// DD_ERR_DEVICE_TIMEOUT in the plan's status word, waits (bounded) for its
// own copies still in flight, frees its tensor memory and returns without
// writing output.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "dd_device.cuh"
#include "dd_internal.h"
#include "dd_quad.h"

namespace {

using namespace ddq;
using namespace dddev;

// N consecutive row offsets of one quad from the (16-byte aligned) record.
template <int N>
__device__ __forceinline__ void load_offsets(const int32_t *p, int (&o)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 4) {
      const int4 v = reinterpret_cast<const int4 *>(p)[i / 4];
      o[i] = v.x, o[i + 1] = v.y, o[i + 2] = v.z, o[i + 3] = v.w;
    }
  } else if constexpr (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const int2 v = reinterpret_cast<const int2 *>(p)[i / 2];
      o[i] = v.x, o[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] = p[i];
  }
}

// acc[j] += word at a + 128 j (+ word at b + 128 j) for j = J..kPairsPerThread-1
template <int J>
struct AccPairs {
  static __device__ __forceinline__ void two(uint32_t (&acc)[kPairsPerThread], uint32_t a,
                                             uint32_t b) {
    acc[J] += lds32_off<128 * J>(a) + lds32_off<128 * J>(b);
    AccPairs<J + 1>::two(acc, a, b);
  }
  static __device__ __forceinline__ void one(uint32_t (&acc)[kPairsPerThread], uint32_t a) {
    acc[J] += lds32_off<128 * J>(a);
    AccPairs<J + 1>::one(acc, a);
  }
};
template <>
struct AccPairs<kPairsPerThread> {
  static __device__ __forceinline__ void two(uint32_t (&)[kPairsPerThread], uint32_t, uint32_t) {}
  static __device__ __forceinline__ void one(uint32_t (&)[kPairsPerThread], uint32_t) {}
};

// ---- tensor memory (per-CTA scratch for the 32-bit sums) ----
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 16 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// Kernel parameters of one launch: the beams' descriptors (dd_quad.h) and
// the shared work queue.
struct QuadLaunch {
  Beam beams[kMaxBeams];
  int32_t nbeams;
  int64_t total_items;
  unsigned long long *next_item;  // work-queue head (zero at launch)
  int32_t *status;                // sticky device status word
  uint64_t timeout_ns;
  int32_t skip_copies;            // test hook: queue nothing, so the first wait runs out
};

// Queue the bulk copies of chunk `ch` (its record and the raw windows of its
// 4*kQuadsPerChunk channels) on mbarrier `bar`.  Called by all 32 lanes of
// one warp: lane s < 16 owns channel slot s; lane 0 posts the byte count.
__device__ void issue_chunk(const Beam &a, const int32_t *meta_s, int tile, int64_t t_cta,
                            int ch, uint32_t bar, uint32_t rec_dst, uint32_t raw_dst, int lane) {
  constexpr int kSlots = 4 * kQuadsPerChunk;
  uint32_t len = 0, skip = 0;
  int64_t lo = 0;
  const int c = ch * kSlots + lane;
  if (lane < kSlots && c < a.nchan_pad) {
    const int32_t start = meta_s[2 * c], need = meta_s[2 * c + 1];
    if (need > 0) {
      // window [off, off + need) rounded to 16 bytes and clipped to the row;
      // its part before the row start (off = -16 in the first time tile)
      // feeds only row words no trial reads
      const int64_t off = t_cta + start;  // multiple of 16
      int64_t hi = off + ((static_cast<int64_t>(need) + 15) & ~static_cast<int64_t>(15));
      if (hi > a.pitch) hi = a.pitch;
      lo = off < 0 ? 0 : off;
      if (hi > lo) {
        len = static_cast<uint32_t>(hi - lo);
        skip = static_cast<uint32_t>(lo - off);
      }
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
    const uint8_t *src = a.block + static_cast<int64_t>(c) * a.pitch + lo;
    bulk_g2s(raw_dst + lane * a.raw_stride + skip, src, len, bar);
  }
}

// Build all pattern rows of a quad, one build unit (dd_quad.h) at a time:
// lane l builds item first+l (4 row words) of every row.  Per channel it
// loads the two aligned words that hold the earliest needed sample and the
// next 4 bytes, for the first and the second half of the pair (kHalf bytes
// on) -- enough for every pattern, whose byte shifts stay within 0..4.  For
// each pattern it funnels out the 4 samples at that pattern's shift (prmt
// with the unit's selector) and sums the four channels in 16-bit lanes: the
// odd bytes (prmt) and the whole words are summed, and the even-byte sum is
// their difference (exact modulo 2^32).  Channel 0 has the same shift in
// every pattern, so its part is formed once per unit.
__device__ __forceinline__ void build_unit(const int32_t *ud, uint32_t raw, uint32_t prow,
                                           int lane) {
  const int4 h = reinterpret_cast<const int4 *>(ud)[0];
  const uint32_t items = (static_cast<uint32_t>(h.z) >> 20) & 63u;
  if (static_cast<uint32_t>(lane) >= items) return;
  const uint32_t npat = static_cast<uint32_t>(h.z) >> 26;
  const uint32_t off[4] = {static_cast<uint32_t>(h.x) & 0xffffu, static_cast<uint32_t>(h.x) >> 16,
                           static_cast<uint32_t>(h.y) & 0xffffu, static_cast<uint32_t>(h.y) >> 16};
  uint32_t a0[4], a1[4], b0[4], b1[4];
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    const bool pad = off[ch] == 0xffffu;                         // padding channel: zeros
    const uint32_t w = raw + (pad ? 0u : off[ch]) + 4u * lane;  // always in bounds
    a0[ch] = pad ? 0u : lds32(w);
    a1[ch] = pad ? 0u : lds32_off<4>(w);
    b0[ch] = pad ? 0u : lds32_off<kHalf>(w);
    b1[ch] = pad ? 0u : lds32_off<kHalf + 4>(w);
  }
  const uint32_t sel0 = static_cast<uint32_t>(h.w) >> 16;
  const uint32_t va0 = prmt(a0[0], a1[0], sel0), vb0 = prmt(b0[0], b1[0], sel0);
  const uint32_t oa0 = prmt(va0, 0u, 0x4341u), ob0 = prmt(vb0, 0u, 0x4341u);
  uint32_t dst = prow + 4u * (static_cast<uint32_t>(h.z) & 0xfffffu) + 16u * lane;
  const uint32_t row_bytes = 4u * (static_cast<uint32_t>(h.w) & 0xffffu);
  // the 4 row words of one pattern from its selectors of channels 1..3
  auto pattern = [&](uint32_t s12, uint32_t s3, uint32_t dst_p) {
    const uint32_t sel[4] = {0u, s12, s12 >> 16, s3};  // prmt reads bits 0..15
    uint32_t sa = va0, sb = vb0, oa = oa0, ob = ob0;   // word sums and odd-byte sums
#pragma unroll
    for (int ch = 1; ch < 4; ++ch) {
      const uint32_t va = prmt(a0[ch], a1[ch], sel[ch]), vb = prmt(b0[ch], b1[ch], sel[ch]);
      sa += va;
      sb += vb;
      oa += prmt(va, 0u, 0x4341u);  // bytes 1, 3 -> 16-bit lanes
      ob += prmt(vb, 0u, 0x4341u);
    }
    const uint32_t ea = sa - (oa << 8), eb = sb - (ob << 8);  // bytes 0, 2 sums
    // word w + j: low half = first-half sum at sample j, high half = second
    sts128(dst_p, prmt(ea, eb, 0x5410u), prmt(oa, ob, 0x5410u), prmt(ea, eb, 0x7632u),
           prmt(oa, ob, 0x7632u));
  };
  // two patterns per step (independent chains for the scheduler)
  const int4 *sels = reinterpret_cast<const int4 *>(ud + 4);
#pragma unroll
  for (int p = 0; p < kMaxPatterns; p += 2) {
    if (static_cast<uint32_t>(p) >= npat) break;
    const int4 sp = sels[p / 2];
    if (static_cast<uint32_t>(p) + 1 < npat) {
      pattern(static_cast<uint32_t>(sp.x), static_cast<uint32_t>(sp.y), dst);
      pattern(static_cast<uint32_t>(sp.z), static_cast<uint32_t>(sp.w), dst + row_bytes);
    } else {
      pattern(static_cast<uint32_t>(sp.x), static_cast<uint32_t>(sp.y), dst);
    }
    dst += 2 * row_bytes;
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

constexpr int kBarFull = 1;                           // + row stage: its chunk's rows built
constexpr int kBarEmpty = kBarFull + kRowStages;       // + row stage: rows, record consumed
constexpr int kBarBuild = kBarEmpty + kRowStages;      // building warps among themselves
static_assert(kBarBuild < 16, "named barrier ids");
constexpr int kBuildThreads = 32 * kBuildWarps;

// Drain the packed accumulators into the 32-bit sums in tensor memory:
// entry m = i * kPairsPerThread + j (trial i, pair j) sits in columns 2m
// (first half) and 2m + 1 (second half) of this thread's lane, moved 8
// entries (16 columns) at a time.  `load`: add to the sums stored so far.
template <int ND_THR>
__device__ __forceinline__ void drain(uint32_t (&acc)[ND_THR][kPairsPerThread], uint32_t taddr,
                                      bool load) {
#pragma unroll
  for (int blk = 0; blk < ND_THR * kPairsPerThread / 8; ++blk) {
    uint32_t v[16];
    if (load) {
      tmem_ld16(taddr + 16u * blk, v);
    } else {
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = 0;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int m = 8 * blk + e;
      uint32_t &w = acc[m / kPairsPerThread][m % kPairsPerThread];
      v[2 * e] += w & 0xffffu;
      v[2 * e + 1] += w >> 16;
      w = 0;
    }
    tmem_st16(taddr + 16u * blk, v);
  }
}

// Arguments of the accumulating role for one work item (the kernel's
// per-item state the role reads).
struct AccArgs {
  const Beam &a;
  uint8_t *smem;
  uint32_t bar0, rec_off, rec_bytes;
  int rec_stages;
  uint32_t prow_off, prow_bytes, tmem_base;
  int warp, lane, dg;
  uint32_t my_pair;
  int tile, ttile;
  int64_t t_cta;
};

// The accumulating role of one work item for a beam of ND_THR trials per
// thread: per chunk, wait for its rows, add them, signal the stage
// consumed; drain the 16-bit halves into tensor memory every kFlushQuads
// quads; write the outputs (and, with rowsums, the row sums and tile
// maxima).  Returns true if the building warps stopped at a copy wait that
// ran out.
template <int ND_THR>
__device__ __forceinline__ bool acc_item(const AccArgs &g) {
  constexpr int ND_CTA = kDmGroups * ND_THR;
  constexpr uint32_t kColsPerThread = 2 * ND_THR * kPairsPerThread;
  constexpr int kFlushChunks = kFlushQuads / kQuadsPerChunk;
  const Beam &a = g.a;
  const int warp = g.warp, lane = g.lane, dg = g.dg, tile = g.tile, ttile = g.ttile;
  const uint32_t my_pair = g.my_pair;
  const int64_t t_cta = g.t_cta;
  volatile int32_t *abort_at = reinterpret_cast<volatile int32_t *>(g.smem + kAbortSlot);
  auto rec_ptr = [&](int m) {
    return reinterpret_cast<const int32_t *>(g.smem + g.rec_off + (m % g.rec_stages) * g.rec_bytes);
  };
  auto prow_addr = [&](int m) { return g.bar0 + g.prow_off + (m % kRowStages) * g.prow_bytes; };
  bool aborted = false;
  const uint32_t taddr = g.tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                         static_cast<uint32_t>(warp >> 2) * kColsPerThread;
  uint32_t acc[ND_THR][kPairsPerThread];
#pragma unroll
  for (int i = 0; i < ND_THR; ++i)
#pragma unroll
    for (int j = 0; j < kPairsPerThread; ++j) acc[i][j] = 0;
  bool drained = false;  // tensor memory holds sums of this item
  for (int k = 0; k < a.nchunks; ++k) {
    bar_sync(kBarFull + k % kRowStages, kThreads);
    if (*abort_at == k) {  // rows of chunk k were not built
      aborted = true;
      break;
    }
    const int32_t *rec = rec_ptr(k);
    const int nq = rec[2];
    const int32_t *A = rec + kRecHeader + dg * ND_THR;  // 16-byte aligned
    const uint32_t prow = prow_addr(k);
    int a_next[2][ND_THR];
    load_offsets<ND_THR>(A, a_next[0]);
    load_offsets<ND_THR>(A + ND_CTA, a_next[1]);
#pragma unroll
    for (int q = 0; q < kQuadsPerChunk; q += 2) {
      if (q < nq) {
        int a_cur[2][ND_THR];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int i = 0; i < ND_THR; ++i) a_cur[h][i] = a_next[h][i];
        if (q + 2 < nq) {
          load_offsets<ND_THR>(A + (q + 2) * ND_CTA, a_next[0]);
          load_offsets<ND_THR>(A + (q + 3) * ND_CTA, a_next[1]);
        }
        if (q + 1 < nq) {
#pragma unroll
          for (int i = 0; i < ND_THR; ++i)
            AccPairs<0>::two(acc[i],
                             prow + 4u * (static_cast<uint32_t>(a_cur[0][i]) + my_pair),
                             prow + 4u * (static_cast<uint32_t>(a_cur[1][i]) + my_pair));
        } else {
#pragma unroll
          for (int i = 0; i < ND_THR; ++i)
            AccPairs<0>::one(acc[i],
                             prow + 4u * (static_cast<uint32_t>(a_cur[0][i]) + my_pair));
        }
      }
    }
    bar_arrive(kBarEmpty + k % kRowStages, kThreads);
    // at most kFlushQuads quads in the 16-bit halves
    if ((k + 1) % kFlushChunks == 0 && k + 1 < a.nchunks) {
      drain<ND_THR>(acc, taddr, drained);
      drained = true;
    }
  }
  if (!aborted) {
    // final sums: stored part (if any) + the packed halves; pair j of
    // trial i covers samples my_pair + 32 j and my_pair + 32 j + kHalf.
    // Per trial, this thread's exact sum, sum of squares and largest
    // value of the samples it stores (for the detection statistics).
    long long s1[ND_THR], s2[ND_THR];
    int32_t mx[ND_THR];
#pragma unroll
    for (int i = 0; i < ND_THR; ++i) s1[i] = 0, s2[i] = 0, mx[i] = INT32_MIN;
#pragma unroll
    for (int blk = 0; blk < ND_THR * kPairsPerThread / 8; ++blk) {
      uint32_t v[16];
      if (drained) {
        tmem_ld16(taddr + 16u * blk, v);
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = 0;
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int m = 8 * blk + e;
        const int i = m / kPairsPerThread, j = m % kPairsPerThread;
        const int d = tile * ND_CTA + dg * ND_THR + i;
        if (d >= a.ndm) continue;
        int32_t *orow = a.out + static_cast<int64_t>(d) * a.out_pitch;
        const uint32_t w = acc[i][j];
        const int64_t t = t_cta + my_pair + 32 * j;
        const int32_t lo = static_cast<int32_t>(v[2 * e] + (w & 0xffffu));
        const int32_t hi = static_cast<int32_t>(v[2 * e + 1] + (w >> 16));
        if (t < a.nsamp_out) {
          orow[t] = lo;
          s1[i] += lo, s2[i] += static_cast<long long>(lo) * lo, mx[i] = max(mx[i], lo);
        }
        if (t + kHalf < a.nsamp_out) {
          orow[t + kHalf] = hi;
          s1[i] += hi, s2[i] += static_cast<long long>(hi) * hi, mx[i] = max(mx[i], hi);
        }
      }
    }
    if (a.rowsums) {
      // one warp holds all kTimeTile samples of its trials: reduce over
      // lanes; integer sums make the row totals independent of order
#pragma unroll
      for (int i = 0; i < ND_THR; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          s1[i] += __shfl_xor_sync(0xffffffffu, s1[i], o);
          s2[i] += __shfl_xor_sync(0xffffffffu, s2[i], o);
          mx[i] = max(mx[i], __shfl_xor_sync(0xffffffffu, mx[i], o));
        }
        const int d = tile * ND_CTA + dg * ND_THR + i;
        if (lane == 0 && d < a.ndm) {
          atomicAdd(reinterpret_cast<unsigned long long *>(a.rowsums + 2 * d),
                    static_cast<unsigned long long>(s1[i]));
          atomicAdd(reinterpret_cast<unsigned long long *>(a.rowsums + 2 * d + 1),
                    static_cast<unsigned long long>(s2[i]));
          a.tilemax[static_cast<int64_t>(d) * a.ntiles_t + ttile] = mx[i];
        }
      }
    }
  }

  return aborted;
}

// Persistent kernel: each CTA takes work items (one DM tile x one time tile
// of one beam) from the launch's queue until it is empty.  Per item every
// warp role runs the chunk pipeline below from a clean state (mbarriers
// re-initialised, every named-barrier phase of the previous item complete);
// tensor memory is allocated once per CTA.
// W: the tile width (trials per accumulating thread) of every beam of the
// launch, or 0 for launches of mixed widths, which pick each item's width at
// run time (a kernel that holds all three accumulating loops needs more
// registers than one that holds one).
template <int CA, int W>
__global__ void __launch_bounds__(kThreads, 1)
dd_dedisperse_quad_u8(const __grid_constant__ QuadLaunch L) {
  // staging depth: copies queued CA chunks ahead, kRaw raw window buffers,
  // kRec records
  constexpr int kRaw = raw_stages(CA), kRec = rec_stages(CA);
  // tensor-memory columns, for the widest tile: accumulating warp w uses
  // lane quarter w % 4 and column block w / 4 of 2 * ND_THR *
  // kPairsPerThread columns (one per sum; narrower tiles use fewer)
  constexpr uint32_t kTmemCols = kAccThreads / 32 / 4 * (2 * kNdThr * kPairsPerThread);
  static_assert(kAccThreads % 128 == 0, "whole warp quartets");
  static_assert((kNdThr / 4) * kPairsPerThread % 8 == 0 && kTmemCols >= 32 && kTmemCols <= 512 &&
                    (kTmemCols & (kTmemCols - 1)) == 0,
                "tensor-memory allocation must be a power of two in 32..512 columns");
  static_assert(kFlushQuads % kQuadsPerChunk == 0, "drain at chunk boundaries");
  static_assert(kTimeGroups == 1, "a warp holds whole time tiles of its trials (tile maxima)");
  static_assert(CA >= kMinCopyAhead && CA <= kMaxCopyAhead && 8 * kRaw <= kTmemSlot &&
                    kItemSlot + 8 <= kBarrierBytes,
                "pipeline depths");
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const uint32_t bar0 = smem_addr(smem);
  auto tma_bar = [&](int m) { return bar0 + 8u * (m % kRaw); };
  // chunk at which the building warps stopped after a copy wait ran out
  volatile int32_t *abort_at = reinterpret_cast<volatile int32_t *>(smem + kAbortSlot);
  volatile long long *item_s = reinterpret_cast<volatile long long *>(smem + kItemSlot);
  int32_t *meta_s = reinterpret_cast<int32_t *>(smem + kBarrierBytes);

  if (warp == 0) tmem_alloc(bar0 + kTmemSlot, kTmemCols);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t *>(smem + kTmemSlot);
  const bool builder = warp >= kAccThreads / 32;
  const int dg = warp / kTimeGroups;
  const int tg = warp & (kTimeGroups - 1);
  const uint32_t my_pair = static_cast<uint32_t>(tg * 32 * kPairsPerThread + lane);

  for (;;) {
    if (tid == 0) *item_s = static_cast<long long>(atomicAdd(L.next_item, 1ull));
    __syncthreads();
    const long long item = *item_s;
    if (item >= L.total_items) break;
    int b = 0;
    while (b + 1 < L.nbeams && item >= L.beams[b + 1].item_begin) ++b;
    const Beam &a = L.beams[b];
    // DM tiles vary fastest along the queue, so the items in flight at any
    // time cover a narrow span of input samples for all DM tiles and share
    // the input windows through L2 instead of re-reading them from HBM.
    const long long local = item - a.item_begin;
    const int tile = static_cast<int>(local % a.ntiles_dm);
    const int ttile = static_cast<int>(local / a.ntiles_dm);
    const int64_t t_cta = static_cast<int64_t>(ttile) * kTimeTile;

    // shared-memory layout (dd_quad.h): copy mbarriers, tensor-memory
    // address and flags, raw window table, records, raw window buffers,
    // pattern rows
    const uint32_t meta_bytes = static_cast<uint32_t>((a.nchan_pad * 8 + 15) / 16 * 16);
    const uint32_t rec_bytes = static_cast<uint32_t>(a.rec_words) * 4;
    const uint32_t rec_off = kBarrierBytes + meta_bytes;
    const uint32_t raw_off = rec_off + kRec * rec_bytes;
    const uint32_t raw_bytes = 4u * kQuadsPerChunk * static_cast<uint32_t>(a.raw_stride);
    const uint32_t prow_off = raw_off + kRaw * raw_bytes;
    const uint32_t prow_bytes = static_cast<uint32_t>(a.prow_words) * 4;
    auto rec_ptr = [&](int m) {
      return reinterpret_cast<const int32_t *>(smem + rec_off + (m % kRec) * rec_bytes);
    };
    auto rec_addr = [&](int m) { return bar0 + rec_off + (m % kRec) * rec_bytes; };
    auto raw_addr = [&](int m) { return bar0 + raw_off + (m % kRaw) * raw_bytes; };
    auto prow_addr = [&](int m) { return bar0 + prow_off + (m % kRowStages) * prow_bytes; };

    const int32_t *meta_g = a.raw_meta + static_cast<int64_t>(tile) * a.nchan_pad * 2;
    for (int i = tid; i < 2 * a.nchan_pad; i += kThreads) meta_s[i] = meta_g[i];
    if (tid == 0) {
      for (int s = 0; s < kRaw; ++s) mbar_init(tma_bar(s), 1);
      *abort_at = INT32_MAX;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // Pipeline (chunk m: raw stage m % kRaw, record stage m %
    // kRec, row stage m % kRowStages).  Building warps, chunk j: wait
    // until the accumulating warps are done with chunk j - kRowStages (its
    // row stage is reused, and so are older record stages); wait (bounded)
    // for the copies of chunk j and agree among themselves that they landed;
    // the first building warp queues the copies of chunk j + CA (into
    // the raw stage of chunk j-1 and the record stage of chunk j-kRowStages);
    // build this warp's units of chunk j's rows; signal the rows built.
    // Accumulating warps, chunk k: wait for its rows, add them, signal the
    // stage consumed.  A copy wait that runs out records its chunk in
    // abort_at before that chunk's rows signal; both roles leave at that
    // chunk, and the building warps then wait for the consumed signals still
    // outstanding, so every barrier phase completes.
    bool aborted = false;
    int issued = 0;  // chunks queued (first building warp)
    if (builder) {
      // this beam's record layout (its tile width)
      const int nd_cta = kDmGroups * a.nd_thr;
      const int segs_off = units_offset(nd_cta), starts_off = warp_start_offset(nd_cta);
      const int bw = warp - kAccThreads / 32;
      const bool issuer = bw == 0 && !L.skip_copies;
      if (issuer) {
        const int prefill = a.nchunks < CA ? a.nchunks : CA;
        for (int m = 0; m < prefill; ++m)
          issue_chunk(a, meta_s, tile, t_cta, m, tma_bar(m), rec_addr(m), raw_addr(m), lane);
        issued = prefill;
      }
      for (int j = 0; j < a.nchunks; ++j) {
        if (j >= kRowStages) bar_sync(kBarEmpty + j % kRowStages, kThreads);
        const bool ok = warp_wait(tma_bar(j), (j / kRaw) & 1, L.timeout_ns, lane);
        if (bar_or(kBarBuild, kBuildThreads, !ok)) {
          if (bw == 0 && lane == 0) *abort_at = j;
          aborted = true;
          bar_arrive(kBarFull + j % kRowStages, kThreads);
          // consumed signals still outstanding: chunks j-kRowStages+1 .. j-1
          for (int m = j - kRowStages + 1; m < j; ++m)
            if (m >= 0) bar_sync(kBarEmpty + m % kRowStages, kThreads);
          break;
        }
        if (issuer && j + CA < a.nchunks) {
          // every building warp is past chunk j-1 (bar_or above) and the
          // accumulating warps past chunk j-kRowStages (bar_sync): the raw
          // stage of chunk j-1 and the record stage of chunk j-kRowStages are
          // free
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          const int m = j + CA;
          issue_chunk(a, meta_s, tile, t_cta, m, tma_bar(m), rec_addr(m), raw_addr(m), lane);
          issued = m + 1;
        }
        const int32_t *rec = rec_ptr(j);
        build_rows(rec, raw_addr(j), prow_addr(j), segs_off, bw, lane, 0,
                   warp_segments(rec, bw, starts_off), starts_off);
        bar_arrive(kBarFull + j % kRowStages, kThreads);
      }
      if (!aborted) {
        // consumed signals of the last kRowStages chunks
        for (int m = a.nchunks - kRowStages; m < a.nchunks; ++m)
          if (m >= 0) bar_sync(kBarEmpty + m % kRowStages, kThreads);
      }
    } else {
      // the accumulating role for this beam's tile width
      const AccArgs args{a,    smem, bar0,    rec_off, rec_bytes, kRec, prow_off, prow_bytes,
                         tmem_base, warp, lane, dg, my_pair, tile, ttile, t_cta};
      if constexpr (W != 0)
        aborted = acc_item<W>(args);
      else if (a.nd_thr == kNdThr)
        aborted = acc_item<kNdThr>(args);
      else if (a.nd_thr == kNdThr / 2)
        aborted = acc_item<kNdThr / 2>(args);
      else
        aborted = acc_item<kNdThr / 4>(args);
    }

    // the item is complete in every warp (tensor-memory accesses waited)
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (*abort_at != INT32_MAX) {
      if (builder && warp - kAccThreads / 32 == 0 && lane == 0) {
        // a bounded wait ran out: record it, and wait (bounded) for the
        // copies this warp queued that may still be in flight (the last
        // kRaw queued, each on its own barrier) before leaving
        atomicExch(L.status, 1);
        for (int m = issued > kRaw ? issued - kRaw : 0; m < issued; ++m)
          mbar_wait_bounded(tma_bar(m), (m / kRaw) & 1, L.timeout_ns);
      }
      __syncthreads();
      break;
    }
  }
  // every thread's tensor-memory accesses are complete before the
  // allocating warp frees the columns
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, kTmemCols);
}

// The kernel at staging depth copy_ahead for tile width w (0: mixed).
template <int W>
auto pick_depth(int copy_ahead) {
  return copy_ahead == 1   ? dd_dedisperse_quad_u8<1, W>
         : copy_ahead == 3 ? dd_dedisperse_quad_u8<3, W>
                           : dd_dedisperse_quad_u8<2, W>;
}
auto pick_kernel(int copy_ahead, int w) {
  return w == kNdThr       ? pick_depth<kNdThr>(copy_ahead)
         : w == kNdThr / 2 ? pick_depth<kNdThr / 2>(copy_ahead)
         : w == kNdThr / 4 ? pick_depth<kNdThr / 4>(copy_ahead)
                           : pick_depth<0>(copy_ahead);
}

}  // namespace

namespace ddk {

bool quad_supported(const dd_plan *p, const void *block, int64_t pitch, int64_t /*nsamp_out*/) {
  if (!p->quad || p->dtype != DD_U8) return false;  // the work queue has no tile-count limit
  return (reinterpret_cast<uintptr_t>(block) & 15) == 0 && (pitch & 15) == 0;
}

int launch_quad_beams(const Beam *beams, int nbeams, int nd_thr, int copy_ahead, int smem,
                      int device_sms,
                      unsigned long long *next_item, int32_t *status, uint64_t timeout_ns,
                      int32_t skip_copies, cudaStream_t stream, cudaError_t *err) {
  if (nbeams < 1 || nbeams > kMaxBeams) {
    *err = cudaErrorInvalidValue;
    return -1;
  }
  QuadLaunch L;
  std::memset(&L, 0, sizeof(L));
  int64_t items = 0;
  for (int i = 0; i < nbeams; ++i) {
    L.beams[i] = beams[i];
    L.beams[i].item_begin = items;
    items += static_cast<int64_t>(beams[i].ntiles_dm) * beams[i].ntiles_t;
  }
  L.nbeams = nbeams;
  L.total_items = items;
  L.next_item = next_item;
  L.status = status;
  L.timeout_ns = timeout_ns;
  L.skip_copies = skip_copies;
  if (copy_ahead < kMinCopyAhead || copy_ahead > kMaxCopyAhead) {
    *err = cudaErrorInvalidValue;
    return -1;
  }
  int width = beams[0].nd_thr;  // one width for every beam, else 0
  for (int i = 0; i < nbeams; ++i) {
    const int w = beams[i].nd_thr;
    if (w != kNdThr && w != kNdThr / 2 && w != kNdThr / 4) {
      *err = cudaErrorInvalidValue;
      return -1;
    }
    if (w != width) width = 0;
  }
  auto kern = pick_kernel(copy_ahead, width);
  *err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int per_sm = 0;
  if (*err == cudaSuccess)
    *err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (*err == cudaSuccess) *err = cudaMemsetAsync(next_item, 0, sizeof(unsigned long long), stream);
  if (*err == cudaSuccess) {
    int64_t grid = static_cast<int64_t>(device_sms) * (per_sm > 0 ? per_sm : 1);
    if (grid > items) grid = items;
    if (grid > 0) kern<<<static_cast<unsigned>(grid), kThreads, smem, stream>>>(L);
    *err = cudaGetLastError();
  }
  return *err == cudaSuccess ? 1 : -1;
}

Beam quad_beam(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out, void *out,
               int64_t out_pitch, int64_t *rowsums, int32_t *tilemax) {
  const QuadDevice &q = *p->quad;
  Beam b;
  std::memset(&b, 0, sizeof(b));
  b.block = static_cast<const uint8_t *>(block);
  b.out = static_cast<int32_t *>(out);
  b.recs = q.d_recs;
  b.raw_meta = q.d_raw_meta;
  b.rowsums = rowsums;
  b.tilemax = tilemax;
  b.pitch = pitch;
  b.nsamp_out = nsamp_out;
  b.out_pitch = out_pitch;
  b.ndm = p->ndm;
  b.nchunks = q.tables.nchunks;
  b.nchan_pad = q.tables.nchan_pad;
  b.rec_words = q.tables.rec_words;
  b.raw_stride = q.tables.raw_stride;
  b.prow_words = q.tables.prow_words;
  b.ntiles_dm = q.tables.ntiles;
  b.nd_thr = q.tables.nd_thr;
  b.ntiles_t = static_cast<int32_t>((nsamp_out + kTimeTile - 1) / kTimeTile);
  return b;
}

int launch_dedisperse_quad(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                           void *out, int64_t out_pitch, int64_t *rowsums, int32_t *tilemax,
                           cudaStream_t stream, cudaError_t *err) {
  const Beam b = quad_beam(p, block, pitch, nsamp_out, out, out_pitch, rowsums, tilemax);
  return launch_quad_beams(&b, 1, p->quad->tables.nd_thr, p->quad->tables.copy_ahead,
                           p->quad->tables.smem_bytes, p->sm_count,
                           p->d_next_item, p->d_error, p->wait_timeout_ns,
                           p->debug_skip_copies, stream, err);
}

}  // namespace ddk
