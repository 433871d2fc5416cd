// dd_dedisp_octet.cu -- staged dedispersion kernel for f16 and f32
// filterbanks.
//
// D[d][t] = sum_c I[c][t + delay(c,d)]   (Sec. 2.1.1, brute-force equation),
// summed in FP32.
//
// Data flow per work item (one 128-trial DM tile x one 256-sample time tile),
// per chunk of 16 channels, in two warp roles that hand chunks to each other
// through named barriers:
//   1. a building warp queues bulk copies (cp.async.bulk, the TMA engine) of
//      each channel's input window -- the "channel vector" of Sec. 2.4, sized
//      by the largest and smallest delay of the tile -- plus the chunk's plan
//      record into shared memory, signalling an mbarrier, two chunks ahead of
//      the chunk being built;
//   2. 11 building warps build pattern rows: word i of a row holds, for one
//      relative-delay pattern of an octet of channels, the eight channels'
//      FP32 sum at output time i (dd_octet_plan.cpp); they build chunk k+1
//      while the accumulating warps add chunk k (double-buffered rows);
//   3. 16 accumulating warps add, for each of their DM trials and output
//      samples, one row word per octet into FP32 register accumulators:
//      eight channel-samples per add and per shared-memory word.
// The two roles split the launch's registers (setmaxnreg): the accumulating
// warps hold 64 accumulators per thread, the building warps need few.
// The kernel is persistent: each CTA takes work items (beam, DM tile, time
// tile) from a device counter, DM tiles fastest, so that the items in flight
// share their input windows in L2.
// The sum is blocked (eight channels, then octets in channel order) rather
// than sequential over channels; its rounding error is bounded by
// (8 + nchan/8) * 2^-24 * sum_c |I|, below the sequential bound, and the
// order per output does not depend on the tile.
// Waits on the mbarriers are bounded (globaltimer): on expiry the CTA records
// DD_ERR_DEVICE_TIMEOUT in the status word, waits (bounded) for its own
// copies still in flight, and returns without writing the item's output.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "dd_device.cuh"
#include "dd_internal.h"
#include "dd_octet.h"

namespace {

using namespace ddo;
using namespace dddev;

// Kernel parameters of one launch: the beams' descriptors (dd_octet.h) and
// the shared work queue.
struct OctetLaunch {
  Beam beams[kMaxBeams];
  int32_t nbeams;
  int64_t total_items;
  unsigned long long *next_item;  // work-queue head (zero at launch)
  int32_t *status;                // sticky device status word
  uint64_t timeout_ns;
  int32_t skip_copies;            // test hook: queue nothing, so the first wait runs out
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

__device__ __forceinline__ void stsf(uint32_t addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// acc[j] += row word at a + 128 j (output sample lane + 32 j of one trial),
// j = J .. kTimesPerThread-1, each load at a compile-time offset
template <int OFF>
__device__ __forceinline__ float ldsf_off(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
  return v;
}
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

__device__ __forceinline__ void setmaxnreg_inc_acc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kAccRegs));
}
__device__ __forceinline__ void setmaxnreg_dec_build() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kBuildRegs));
}

// Window of channel slot `lane` of chunk `ch` (its start and length in
// elements, from the plan's table in global memory): loaded one chunk before
// the copies are queued, so that the load's latency overlaps other work.
struct Window {
  int32_t start = 0, need = 0;
};
__device__ __forceinline__ Window load_window(const Beam &a, int opc, int tile, int ch,
                                              int lane) {
  Window w;
  const int c = ch * kGroup * opc + lane;
  if (lane < kGroup * opc && c < a.nchan_pad && ch < a.nchunks) {
    const int2 m = __ldg(reinterpret_cast<const int2 *>(a.raw_meta) +
                         static_cast<int64_t>(tile) * a.nchan_pad + c);
    w.start = m.x, w.need = m.y;
  }
  return w;
}

// Queue the bulk copies of chunk `ch` (its record and the raw windows of its
// 8*opc channels) on mbarrier `bar`.  Called by all 32 lanes of one warp:
// lane s < 8*opc owns channel slot s with window `w`; lane 0 posts the byte
// count.
__device__ void issue_chunk(const Beam &a, int opc, int esize, int tile, int64_t t_cta, int ch,
                            Window w, uint32_t bar, uint32_t rec_dst, uint32_t slots_dst,
                            int lane) {
  uint32_t len = 0, skip = 0;
  int64_t lo = 0;
  const int c = ch * kGroup * opc + lane;
  if (w.need > 0) {
    // window [off, off + need) rounded to 16 bytes and clipped to the row;
    // its part before the row start (a window of a channel below the
    // reference in the first time tile) feeds only row words no output reads
    const int64_t off = (t_cta + w.start) * esize;  // multiple of 16 bytes
    int64_t hi = off + ((static_cast<int64_t>(w.need) * esize + 15) & ~static_cast<int64_t>(15));
    if (hi > a.pitch_bytes) hi = a.pitch_bytes;
    lo = off < 0 ? 0 : off;
    if (hi > lo) {
      len = static_cast<uint32_t>(hi - lo);
      skip = static_cast<uint32_t>(lo - off);
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
    const uint8_t *src = a.block + static_cast<int64_t>(c) * a.pitch_bytes + lo;
    bulk_g2s(slots_dst + static_cast<uint32_t>(lane * a.raw_stride * esize) + skip, src, len, bar);
  }
}

// The rows of one build unit whose shifts are all at most MAXB (1 or 2):
// every channel's candidate samples are loaded once (as many as that
// channel's largest shift needs; the others repeat the last loaded one, so
// the selects below stay exact without a branch), then each pattern sums, in
// channel order, each channel's candidate at the pattern's shift -- shift
// bit 0 picks r1 over r0, bit 1 (MAXB 2) picks r2 -- two patterns at a time.
// The reference channel's shift is 0 in every pattern: it adds r0.  f16
// candidates are widened to FP32 once, as they are loaded (exact); each
// FP32 add of a widened sample rounds as the mixed f32 + f16 add does.
template <typename T, int MAXB>
__device__ __forceinline__ void build_selects(const uint32_t (&addr)[kGroup],
                                              const uint32_t *codes, uint32_t cb, uint32_t npat,
                                              uint32_t dst, uint32_t row_bytes) {
  using E = Elem<T>;
  constexpr uint32_t es = sizeof(T);
  float r0[kGroup], r1[kGroup], r2[kGroup];
#pragma unroll
  for (int k = 0; k < kGroup; ++k) {
    const uint32_t bk = (cb >> (2 * k)) & 3u;
    r0[k] = E::widen(E::load(addr[k]));
    if (k == kRefChan) continue;
    r1[k] = bk >= 1 ? E::widen(E::load(addr[k] + es)) : r0[k];
    r2[k] = MAXB >= 2 && bk >= 2 ? E::widen(E::load(addr[k] + 2 * es)) : r1[k];
  }
  auto pick = [&](uint32_t code, int k) -> float {
    const float lo = ((code >> (2 * k)) & 1u) ? r1[k] : r0[k];
    return MAXB == 1 ? lo : (((code >> (2 * k)) & 2u) ? r2[k] : lo);
  };
  // every code word read up front and the pattern loop unrolled, so that
  // the code loads and the two patterns' selects need not wait in turn
  const int4 c03 = reinterpret_cast<const int4 *>(codes)[0];
  const int4 c47 = reinterpret_cast<const int4 *>(codes)[1];
  const uint32_t cw[8] = {static_cast<uint32_t>(c03.x), static_cast<uint32_t>(c03.y),
                          static_cast<uint32_t>(c03.z), static_cast<uint32_t>(c03.w),
                          static_cast<uint32_t>(c47.x), static_cast<uint32_t>(c47.y),
                          static_cast<uint32_t>(c47.z), static_cast<uint32_t>(c47.w)};
  auto pattern = [&](uint32_t code, uint32_t a) {
    float v = pick(code, 0);
#pragma unroll
    for (int k = 1; k < kGroup; ++k) v = __fadd_rn(v, k == kRefChan ? r0[k] : pick(code, k));
    stsf(a, v);
  };
#pragma unroll
  for (uint32_t p = 0; p < kMaxPatterns; p += 2) {
    if (p >= npat) break;
    pattern(cw[p >> 1], dst + p * row_bytes);
    if (p + 1 < npat) pattern(cw[p >> 1] >> 16, dst + (p + 1) * row_bytes);
  }
}

// Build the pattern rows of one build unit (dd_octet.h): lane l builds row
// word first+l of each of the unit's rows -- per pattern the sum,
// in channel order, of each channel's sample at its shift.  When every shift
// of the unit is at most 2 (the common case) the candidate samples are loaded
// once and selected per pattern; otherwise each pattern's samples are loaded
// directly.
template <typename T>
__device__ __forceinline__ void build_unit(const int32_t *ud, uint32_t zero, uint32_t prow,
                                           int lane) {
  const int4 h0 = reinterpret_cast<const int4 *>(ud)[0];
  const uint32_t items = (static_cast<uint32_t>(h0.x) >> 20) & 63u;
  if (static_cast<uint32_t>(lane) >= items) return;
  const int4 h1 = reinterpret_cast<const int4 *>(ud)[1];
  const uint32_t npat = static_cast<uint32_t>(h0.y) & 0xffu;
  const uint32_t row_bytes = 4u * ((static_cast<uint32_t>(h0.y) >> 8) & 0x1fffffu);
  const uint32_t bound = (static_cast<uint32_t>(h0.y) >> 29) & 3u;
  const uint32_t offw[4] = {static_cast<uint32_t>(h0.z), static_cast<uint32_t>(h0.w),
                            static_cast<uint32_t>(h1.x), static_cast<uint32_t>(h1.y)};
  const uint32_t cb = static_cast<uint32_t>(h1.z);  // word kBoundsWord: per channel, largest shift
  static_assert(kBoundsWord == 6, "bounds word read from the second header vector");
  const uint32_t *codes = reinterpret_cast<const uint32_t *>(ud + kCodesWord);
  constexpr uint32_t es = sizeof(T);
  uint32_t addr[kGroup];
#pragma unroll
  for (int k = 0; k < kGroup; ++k)
    addr[k] = zero + es * (((offw[k / 2] >> (16 * (k & 1))) & 0xffffu) + lane);
  const uint32_t dst = prow + 4u * ((static_cast<uint32_t>(h0.x) & 0xfffffu) + lane);
  if (bound == 1) {
    build_selects<T, 1>(addr, codes, cb, npat, dst, row_bytes);
  } else if (bound == 2) {
    build_selects<T, 2>(addr, codes, cb, npat, dst, row_bytes);
  } else {
    using E = Elem<T>;
#pragma unroll 1
    for (uint32_t p = 0; p < npat; ++p) {
      const uint32_t code = codes[p >> 1] >> (16 * (p & 1));
      auto shift = [&](int k) { return (code >> (2 * k)) & 3u; };
      float v = E::widen(E::load(addr[0] + es * shift(0)));
#pragma unroll
      for (int k = 1; k < kGroup; ++k) v = E::add(v, E::load(addr[k] + es * shift(k)));
      stsf(dst + p * row_bytes, v);
    }
  }
}

constexpr int kBarFull = 1;                       // + row stage: its chunk's rows built
constexpr int kBarEmpty = kBarFull + kRowStages;  // + row stage: rows, record consumed
constexpr int kBarBuild = kBarEmpty + kRowStages;  // building warps among themselves
constexpr int kBarItem = kBarBuild + 1;           // all warps: next work item published
constexpr int kBarItemEnd = kBarItem + 1;         // all warps: item done, shared memory free
static_assert(kBarItemEnd < 16, "named barrier ids");

// Shared-memory layout of one item (dd_octet.h): copy mbarriers and flags,
// records, raw stages (zero area + window slots), pattern-row stages.
template <typename T>
struct Layout {
  static constexpr int kEs = sizeof(T);
  static constexpr int kOpc = kEs == 4 ? kOpcF32 : 2;  // octets per chunk
  uint32_t base, rec_bytes, raw_off, stage_bytes, prow_off, prow_bytes;
  __device__ Layout(uint32_t bar0, const Beam &a) {
    base = bar0;
    rec_bytes = static_cast<uint32_t>(a.rec_words) * 4;
    raw_off = kBarrierBytes + kRecStages * rec_bytes;
    stage_bytes = zero_bytes() + kGroup * kOpc * static_cast<uint32_t>(a.raw_stride) * kEs;
    prow_off = raw_off + kRawStages * stage_bytes;
    prow_bytes = static_cast<uint32_t>(a.prow_words) * 4;
  }
  static __device__ constexpr uint32_t zero_bytes() { return kZeroElems * kEs; }
  __device__ uint32_t rec(int m) const { return kBarrierBytes + (m % kRecStages) * rec_bytes; }
  __device__ uint32_t zero(int m) const { return raw_off + (m % kRawStages) * stage_bytes; }
  __device__ uint32_t prow(int m) const { return prow_off + (m % kRowStages) * prow_bytes; }
};

// The work item published in shared memory: its beam, DM tile and first
// output sample.  DM tiles vary fastest along the queue, so the items in
// flight at any time cover a narrow span of input samples for all DM tiles
// and share the input windows through L2 instead of re-reading them.
struct Item {
  int beam, tile;
  int64_t t_cta;
};
// Queue slot `item` as (beam, DM tile, time tile); false for an empty slot
// (the DM tile's time tile, after its skew, outside the beam's block).
__device__ __forceinline__ bool decode_item(const OctetLaunch &L, long long item, Item *it) {
  int b = 0;
  while (b + 1 < L.nbeams && item >= L.beams[b + 1].item_begin) ++b;
  const Beam &a = L.beams[b];
  const long long local = item - a.item_begin;
  const int tile = static_cast<int>(local % a.ntiles_dm);
  const long long ttile = local / a.ntiles_dm - __ldg(a.skew + tile);
  it->beam = b;
  it->tile = tile;
  it->t_cta = ttile * kTimeTile;
  return ttile >= 0 && ttile < a.ntiles_t;
}

// Next non-empty queue slot (one thread per CTA): the slot number, or
// total_items when the queue is drained.
__device__ __forceinline__ long long fetch_item(const OctetLaunch &L) {
  for (;;) {
    const long long item = static_cast<long long>(atomicAdd(L.next_item, 1ull));
    Item it;
    if (item >= L.total_items || decode_item(L, item, &it)) return item;
  }
}

__device__ __forceinline__ bool next_item(const OctetLaunch &L, const uint8_t *smem, Item *it) {
  const long long item = *reinterpret_cast<const volatile long long *>(smem + kItemSlot);
  if (item >= L.total_items) return false;
  decode_item(L, item, it);
  return true;
}

// Per item, the building warps run chunk j: wait until the accumulating
// warps are done with chunk j - kRowStages (its row stage is reused, and so
// are older record stages); wait (bounded) for the copies of chunk j and
// agree among themselves that they landed; the first building warp queues
// the copies of chunk j + kCopyAhead (into the raw stage of chunk j-1 and
// the record stage of chunk j-kRowStages); build this warp's units of chunk
// j's rows; signal the rows built.  The accumulating warps run chunk k: wait
// for its rows, add them, signal the stage consumed.  A copy wait that runs
// out records its chunk in the abort slot before that chunk's rows signal;
// both roles leave at that chunk, and the building warps then wait for the
// consumed signals still outstanding, so every barrier phase completes.
// Each role keeps its own persistent loop, so that each runs under its own
// register budget (setmaxnreg); they meet at the item barriers.
template <typename T, int ND_THR>
__device__ __forceinline__ void build_role(const OctetLaunch &L, uint8_t *smem, int warp,
                                           int lane) {
  constexpr int ND_CTA = kDmGroups * ND_THR;
  constexpr int kUnitsOff = units_offset(ND_CTA);
  constexpr int kStartsOff = warp_start_offset(ND_CTA);
  using Lay = Layout<T>;
  const int bw = warp - kAccThreads / 32;
  const int btid = bw * 32 + lane;
  const bool issuer = bw == 0 && !L.skip_copies;
  const uint32_t bar0 = smem_addr(smem);
  auto tma_bar = [&](int m) { return bar0 + 8u * (m % kRawStages); };
  volatile int32_t *abort_at = reinterpret_cast<volatile int32_t *>(smem + kAbortSlot);
  for (;;) {
    if (btid == 0) {
      *reinterpret_cast<volatile long long *>(smem + kItemSlot) = fetch_item(L);
      *abort_at = INT32_MAX;
    }
    bar_sync(kBarItem, kThreads);
    Item it;
    if (!next_item(L, smem, &it)) return;
    const Beam &a = L.beams[it.beam];
    const Lay lay(bar0, a);
    // the zero areas (padding channels read them) sit where this beam's
    // layout puts them; the mbarriers start a fresh phase count
    for (int s = 0; s < kRawStages; ++s)
      for (uint32_t i = 4u * btid; i < Lay::zero_bytes(); i += 4u * kBuildThreads)
        *reinterpret_cast<uint32_t *>(smem + lay.zero(s) + i) = 0u;
    if (btid == 0) {
      for (int s = 0; s < kRawStages; ++s) mbar_init(tma_bar(s), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    bar_sync(kBarBuild, kBuildThreads);
    int issued = 0;  // chunks queued (first building warp)
    Window next_w;   // window of the next chunk to queue (first building warp)
    if (issuer) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int prefill = a.nchunks < kCopyAhead ? a.nchunks : kCopyAhead;
      for (int m = 0; m < prefill; ++m)
        issue_chunk(a, Lay::kOpc, Lay::kEs, it.tile, it.t_cta, m,
                    load_window(a, Lay::kOpc, it.tile, m, lane), tma_bar(m), bar0 + lay.rec(m),
                    bar0 + lay.zero(m) + Lay::zero_bytes(), lane);
      issued = prefill;
      next_w = load_window(a, Lay::kOpc, it.tile, prefill, lane);
    }
    bool aborted = false;
    for (int j = 0; j < a.nchunks; ++j) {
      if (j >= kRowStages) bar_sync(kBarEmpty + j % kRowStages, kThreads);
      const bool ok = warp_wait(tma_bar(j), (j / kRawStages) & 1, L.timeout_ns, lane);
      if (bar_or(kBarBuild, kBuildThreads, !ok)) {
        if (btid == 0) *abort_at = j;
        aborted = true;
        bar_arrive(kBarFull + j % kRowStages, kThreads);
        // consumed signals still outstanding: chunks j-kRowStages+1 .. j-1
        for (int m = j - kRowStages + 1; m < j; ++m)
          if (m >= 0) bar_sync(kBarEmpty + m % kRowStages, kThreads);
        break;
      }
      if (issuer && j + kCopyAhead < a.nchunks) {
        // every building warp is past chunk j-1 (bar_or above) and the
        // accumulating warps past chunk j-kRowStages (bar_sync): the raw
        // stage of chunk j-1 and the record stage of chunk j-kRowStages are
        // free
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int m = j + kCopyAhead;
        issue_chunk(a, Lay::kOpc, Lay::kEs, it.tile, it.t_cta, m, next_w, tma_bar(m),
                    bar0 + lay.rec(m), bar0 + lay.zero(m) + Lay::zero_bytes(), lane);
        issued = m + 1;
        next_w = load_window(a, Lay::kOpc, it.tile, m + 1, lane);
      }
      const int32_t *rec = reinterpret_cast<const int32_t *>(smem + lay.rec(j));
      const uint16_t *starts = reinterpret_cast<const uint16_t *>(rec + kStartsOff);
      const int first = starts[bw], last = starts[bw + 1];
      const uint32_t zero = bar0 + lay.zero(j), prow = bar0 + lay.prow(j);
#pragma unroll 1
      for (int m = first; m < last; ++m)
        build_unit<T>(rec + kUnitsOff + m * kUnitWords, zero, prow, lane);
      bar_arrive(kBarFull + j % kRowStages, kThreads);
    }
    if (!aborted) {
      // consumed signals of the last kRowStages chunks
      for (int m = a.nchunks - kRowStages; m < a.nchunks; ++m)
        if (m >= 0) bar_sync(kBarEmpty + m % kRowStages, kThreads);
    }
    bar_sync(kBarItemEnd, kThreads);
    if (*abort_at != INT32_MAX) {
      if (btid == 0) {
        // a bounded wait ran out: record it, and wait (bounded) for the
        // copies this warp queued that may still be in flight (the last
        // kRawStages queued, each on its own barrier) before leaving
        atomicExch(L.status, 1);
        for (int m = issued > kRawStages ? issued - kRawStages : 0; m < issued; ++m)
          mbar_wait_bounded(tma_bar(m), (m / kRawStages) & 1, L.timeout_ns);
      }
      return;
    }
  }
}

template <typename T, int ND_THR>
__device__ __forceinline__ void acc_role(const OctetLaunch &L, uint8_t *smem, int warp, int lane) {
  constexpr int ND_CTA = kDmGroups * ND_THR;
  static_assert(ND_THR % 4 == 0, "offsets are read four at a time");
  using Lay = Layout<T>;
  const uint32_t bar0 = smem_addr(smem);
  volatile int32_t *abort_at = reinterpret_cast<volatile int32_t *>(smem + kAbortSlot);
  for (;;) {
    bar_sync(kBarItem, kThreads);
    Item it;
    if (!next_item(L, smem, &it)) return;
    const Beam &a = L.beams[it.beam];
    const Lay lay(bar0, a);
    float acc[ND_THR][kTimesPerThread];
#pragma unroll
    for (int i = 0; i < ND_THR; ++i)
#pragma unroll
      for (int j = 0; j < kTimesPerThread; ++j) acc[i][j] = 0.f;
    bool aborted = false;
    for (int k = 0; k < a.nchunks; ++k) {
      bar_sync(kBarFull + k % kRowStages, kThreads);
      if (*abort_at == k) {  // rows of chunk k were not built
        aborted = true;
        break;
      }
      const int32_t *rec = reinterpret_cast<const int32_t *>(smem + lay.rec(k));
      const int no = rec[2];
      const int4 *A = reinterpret_cast<const int4 *>(rec + kRecHeader + warp * ND_THR);
      const uint32_t prow = bar0 + lay.prow(k) + 4u * static_cast<uint32_t>(lane);
#pragma unroll
      for (int o = 0; o < Lay::kOpc; ++o) {
        if (o < no) {
          int off[ND_THR];
#pragma unroll
          for (int i = 0; i < ND_THR; i += 4) {
            const int4 v = A[(o * ND_CTA + i) / 4];
            off[i] = v.x, off[i + 1] = v.y, off[i + 2] = v.z, off[i + 3] = v.w;
          }
#pragma unroll
          for (int i = 0; i < ND_THR; ++i)
            AccRow<0>::run(acc[i], prow + 4u * static_cast<uint32_t>(off[i]));
        }
      }
      bar_arrive(kBarEmpty + k % kRowStages, kThreads);
    }
    if (!aborted) {
#pragma unroll
      for (int i = 0; i < ND_THR; ++i) {
        const int d = it.tile * ND_CTA + warp * ND_THR + i;
        if (d >= a.ndm) continue;  // the same for the whole warp
        float *orow = a.out + static_cast<int64_t>(d) * a.out_pitch;
#pragma unroll
        for (int j = 0; j < kTimesPerThread; ++j) {
          const int64_t t = it.t_cta + lane + 32 * j;
          if (t < a.nsamp_out) orow[t] = acc[i][j];
        }
        if (a.tilestats) {
          // this trial's partial statistics over the tile (one warp holds
          // all its samples): sums of y = x - K about the tile's first
          // output K, of y^2, and the largest output, in a fixed order
          const float K = __shfl_sync(0xffffffffu, acc[i][0], 0);
          float s1 = 0.f, s2 = 0.f, mx = -INFINITY;
#pragma unroll
          for (int j = 0; j < kTimesPerThread; ++j) {
            if (it.t_cta + lane + 32 * j < a.nsamp_out) {
              const float y = acc[i][j] - K;
              s1 += y;
              s2 = fmaf(y, y, s2);
              mx = fmaxf(mx, acc[i][j]);
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          }
          if (lane == 0)
            a.tilestats[static_cast<int64_t>(d) * a.ntiles_t + it.t_cta / kTimeTile] =
                make_float4(K, s1, s2, mx);
        }
      }
    }
    bar_sync(kBarItemEnd, kThreads);
    if (*abort_at != INT32_MAX) return;
  }
}

// Persistent kernel: each CTA takes work items (one DM tile x one time tile
// of one beam) from the launch's queue until it is empty.
template <typename T, int ND_THR>
__global__ void __launch_bounds__(kThreads, 1)
dd_dedisperse_octet(const __grid_constant__ OctetLaunch L) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp >= kAccThreads / 32) {
    setmaxnreg_dec_build();
    build_role<T, ND_THR>(L, smem, warp, lane);
  } else {
    setmaxnreg_inc_acc();
    acc_role<T, ND_THR>(L, smem, warp, lane);
  }
}

template <typename T, int ND_THR>
int launch(const OctetLaunch &L, int smem, int device_sms, cudaStream_t stream,
           cudaError_t *err) {
  auto kern = dd_dedisperse_octet<T, ND_THR>;
  *err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  // the register split assumes the launch's kLaunchRegs registers per
  // thread; a kernel compiled to fewer would leave the accumulating warps
  // waiting for registers that are not there, so it is never launched
  cudaFuncAttributes fa;
  if (*err == cudaSuccess) *err = cudaFuncGetAttributes(&fa, kern);
  if (*err == cudaSuccess && fa.numRegs != kLaunchRegs) *err = cudaErrorInvalidConfiguration;
  if (*err == cudaSuccess)
    *err = cudaMemsetAsync(L.next_item, 0, sizeof(unsigned long long), stream);
  if (*err == cudaSuccess) {
    int64_t grid = device_sms;  // one CTA per SM (its shared memory allows no more)
    if (grid > L.total_items) grid = L.total_items;
    if (grid > 0) kern<<<static_cast<unsigned>(grid), kThreads, smem, stream>>>(L);
    *err = cudaGetLastError();
  }
  return *err == cudaSuccess ? 1 : -1;
}

}  // namespace

namespace ddk {

bool octet_supported(const dd_plan *p, const void *block, int64_t pitch, int64_t /*nsamp_out*/) {
  if (!p->octet || p->dtype == DD_U8 || !p->d_next_item) return false;
  const int64_t pitch_bytes = pitch * elem_size(p->dtype);  // the work queue has no tile limit
  return (reinterpret_cast<uintptr_t>(block) & 15) == 0 && (pitch_bytes & 15) == 0;
}

ddo::Beam octet_beam(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                     void *out, int64_t out_pitch, float4 *tilestats) {
  const OctetDevice &q = *p->octet;
  Beam b;
  std::memset(&b, 0, sizeof(b));
  b.block = static_cast<const uint8_t *>(block);
  b.out = static_cast<float *>(out);
  b.recs = q.d_recs;
  b.raw_meta = q.d_raw_meta;
  b.skew = q.d_skew;
  b.tilestats = tilestats;
  b.max_skew = q.tables.max_skew;
  b.pitch_bytes = pitch * elem_size(p->dtype);
  b.nsamp_out = nsamp_out;
  b.out_pitch = out_pitch;
  b.ndm = p->ndm;
  b.nchunks = q.tables.nchunks;
  b.nchan_pad = q.tables.nchan_pad;
  b.rec_words = q.tables.rec_words;
  b.raw_stride = q.tables.raw_stride;
  b.prow_words = q.tables.prow_words;
  b.ntiles_dm = q.tables.ntiles;
  b.ntiles_t = static_cast<int32_t>((nsamp_out + kTimeTile - 1) / kTimeTile);
  return b;
}

int launch_octet_beams(const ddo::Beam *beams, int nbeams, int32_t dtype, int nd_thr, int smem,
                       int device_sms, unsigned long long *next_item, int32_t *status,
                       uint64_t timeout_ns, int32_t skip_copies, cudaStream_t stream,
                       cudaError_t *err) {
  if (nbeams < 1 || nbeams > kMaxBeams || (dtype != DD_F16 && dtype != DD_F32) ||
      (nd_thr != kNdThr && nd_thr != kNdThr / 2)) {
    *err = cudaErrorInvalidValue;
    return -1;
  }
  OctetLaunch L;
  std::memset(&L, 0, sizeof(L));
  int64_t items = 0;
  for (int i = 0; i < nbeams; ++i) {
    L.beams[i] = beams[i];
    L.beams[i].item_begin = items;
    items += static_cast<int64_t>(beams[i].ntiles_dm) * (beams[i].ntiles_t + beams[i].max_skew);
  }
  L.nbeams = nbeams;
  L.total_items = items;
  L.next_item = next_item;
  L.status = status;
  L.timeout_ns = timeout_ns;
  L.skip_copies = skip_copies;
  const bool wide = nd_thr == kNdThr;
  if (dtype == DD_F32)
    return wide ? launch<float, kNdThr>(L, smem, device_sms, stream, err)
                : launch<float, kNdThr / 2>(L, smem, device_sms, stream, err);
  return wide ? launch<__half, kNdThr>(L, smem, device_sms, stream, err)
              : launch<__half, kNdThr / 2>(L, smem, device_sms, stream, err);
}

int launch_dedisperse_octet(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                            void *out, int64_t out_pitch, float4 *tilestats, cudaStream_t stream,
                            cudaError_t *err) {
  const Beam b = octet_beam(p, block, pitch, nsamp_out, out, out_pitch, tilestats);
  return launch_octet_beams(&b, 1, p->dtype, p->octet->tables.nd_thr, p->octet->tables.smem_bytes,
                            p->sm_count, p->d_next_item, p->d_error, p->wait_timeout_ns,
                            p->debug_skip_copies, stream, err);
}

}  // namespace ddk
