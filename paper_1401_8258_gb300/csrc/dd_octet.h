// dd_octet.h -- shape constants and plan-time tables of the staged octet
// kernel for f16 and f32 input (internal to libdd).
//
// CTA tile: kDmGroups x nd_thr DM trials (16 x 8 = 128, or 16 x 4 = 64) by
// kTimeTile (256) output samples.  Two warp roles: 16 accumulating warps =
// 16 DM groups, a thread owning nd_thr trials x kTimesPerThread samples
// (sample = lane + 32*j); and kBuildWarps (8) building warps that queue the
// copies and build the pattern rows one chunk ahead.  Channels are taken in
// groups of kGroup = 8 adjacent channels ("octets"), `opc` (2) octets per
// chunk.
//
// Pattern rows.  For octet o of a DM tile, the delays of its channels are
// taken relative to its reference channel r (channel kRefChan of the octet,
// or its last real channel if it has fewer): e_k(d) = delay(c_k, d) -
// delay(c_r, d).  Let b be the smallest reference delay over the tile's
// trials.  Each distinct relative-delay pattern p of the octet has a row of
// L float words (L = kTimeTile + largest reference delay - b, rounded up to
// 4); word i of row p holds the sum over the octet's channels k, in channel
// order, of I[c_k][t_cta + b + e_k(p) + i].  The rows of an octet are
// contiguous.
//
// Per (DM tile, chunk) record, int32 words:
//   [0] unused                 [1] unused
//   [2] octets in this chunk   [3] number of build units
//   A[kMaxOctetsPerChunk][nd_cta]  word offset, within the chunk's row area,
//                              of the row word that holds output sample 0 of
//                              the tile for that octet and trial
//   units[kMaxUnits][16]: one warp-wide build step each -- items first ..
//     first+31 (item = one row word) of the consecutive pattern rows p0 ..
//     p0+patterns-1 of one octet (those that some trial of the tile reads
//     there, or a half of them); lane l builds item first+l:
//     [0] row-area word offset of item `first` of row p0 | items << 20
//     [1] patterns | L << 8 | shift bound << 29 (every shift of the unit is
//         at most 1: 1; at most 2: 2; otherwise 0)
//     [2..5] element offsets, from the raw stage's zero area, of channels
//         0..7 (16 bits each, two per word): the earliest sample any pattern
//         needs for item `first`; padding channels point into the zero area
//     [6] per channel k, its largest shift over the patterns (bits 2k ..
//         2k+1)
//     [8..15] shift codes of rows p0 .., two patterns per word (16 bits
//         each): for channel k the 2-bit element shift 0..3 of the pattern's sample
//         past that offset, at bits 2k .. 2k+1 (0 for the reference channel)
//   warp_start[kBuildWarps + 1] (int16 pairs, after the units): building
//     warp w builds units warp_start[w] .. warp_start[w+1]-1 (balanced on the
//     host; the first kFirstBuilder warps queue the copies and build none).
// raw_meta[tile][nchan_pad][2]: {window start in elements relative to the
// tile's first output sample (16-byte aligned; may be negative below the
// reference channel), elements needed (0 = padding channel)}.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#ifdef __CUDACC__
#define DDO_HD __host__ __device__
#else
#define DDO_HD
#endif

namespace ddo {

// Tile shape; the DDO_* macros exist only to build shape variants for tuning.
#ifndef DDO_TIMES_PER_THREAD
#define DDO_TIMES_PER_THREAD 8
#endif
#ifndef DDO_ND_THR
#define DDO_ND_THR 8
#endif
#ifndef DDO_OPC_F32
#define DDO_OPC_F32 2
#endif
constexpr int kGroup = 8;
constexpr int kRefChan = 3;  // reference channel of an octet (the patterns' delay origin)
constexpr int kDmGroups = 16;
constexpr int kAccThreads = 32 * kDmGroups;              // 512 accumulating threads
#ifndef DDO_BUILD_WARPS
#define DDO_BUILD_WARPS 12
#endif
#ifndef DDO_ACC_REGS
#define DDO_ACC_REGS 80
#endif
#ifndef DDO_DEDICATED_ISSUER
#define DDO_DEDICATED_ISSUER 1
#endif
constexpr int kBuildWarps = DDO_BUILD_WARPS;
// Building warp 0 queues the copies; with kFirstBuilder = 1 it builds no
// rows (its share of the build units goes to the other building warps).
constexpr int kFirstBuilder = DDO_DEDICATED_ISSUER ? 1 : 0;
constexpr int kBuildThreads = 32 * kBuildWarps;          // 384 building threads
constexpr int kThreads = kAccThreads + kBuildThreads;    // 896
// Register split of the two roles (setmaxnreg): the launch gives every
// thread kLaunchRegs (the register file shared out, in whole units of 8);
// accumulating warps take kAccRegs, building warps keep kBuildRegs, within
// the launch's kThreads * kLaunchRegs registers.
constexpr int kLaunchRegs = 65536 / kThreads / 8 * 8;
constexpr int kAccRegs = DDO_ACC_REGS;
constexpr int kBuildRegs =
    (kThreads * kLaunchRegs - kAccThreads * kAccRegs) / kBuildThreads / 8 * 8;
static_assert(kBuildRegs >= 24 && kBuildRegs <= 256 && kAccRegs % 8 == 0 && kAccRegs <= 256,
              "setmaxnreg counts are multiples of 8 in 24..256");
static_assert(kAccThreads * kAccRegs + kBuildThreads * kBuildRegs <= kThreads * kLaunchRegs,
              "register split exceeds the launch's registers");
static_assert(kAccThreads % 128 == 0 && kBuildThreads % 128 == 0,
              "setmaxnreg applies to whole warpgroups");
constexpr int kTimesPerThread = DDO_TIMES_PER_THREAD;
constexpr int kTimeTile = 32 * kTimesPerThread;          // 256
constexpr int kNdThr = DDO_ND_THR;                       // trials per thread (128 per CTA)
constexpr int kOpcF32 = DDO_OPC_F32;                     // octets per chunk for f32 input
constexpr int kMaxOctetsPerChunk = 2;
constexpr int kMaxPatterns = 16;
constexpr int kMaxShift = 3;                             // element shifts 0..3 within a unit
constexpr int kRecHeader = 4;
constexpr int kUnitWords = 16;
constexpr int kBoundsWord = 6;
constexpr int kCodesWord = 8;  // kMaxPatterns / 2 words of shift codes
static_assert(kCodesWord + kMaxPatterns / 2 <= kUnitWords && kUnitWords % 4 == 0,
              "unit layout");
constexpr int kMaxUnits = 64;
constexpr int kZeroElems = 64;                           // zero area for padding channels
constexpr int kMaxSmem = 227 * 1024;

DDO_HD constexpr int units_offset(int nd_cta) {
  return kRecHeader + kMaxOctetsPerChunk * nd_cta;       // multiple of 4 words
}
DDO_HD constexpr int warp_start_offset(int nd_cta) {
  return units_offset(nd_cta) + kMaxUnits * kUnitWords;
}
DDO_HD constexpr int rec_words(int nd_cta) {
  return (warp_start_offset(nd_cta) + (kBuildWarps + 2) / 2 + 3) / 4 * 4;
}

// Pipeline: the building warps queue the copies of a chunk kCopyAhead chunks
// ahead of the one they build, and build chunk k+1's rows while the
// accumulating warps add chunk k (kRowStages row areas).  A raw stage is
// free once its chunk is built; a record once its chunk is accumulated.
constexpr int kCopyAhead = 2;
constexpr int kRawStages = kCopyAhead + 1;
constexpr int kRowStages = 2;
constexpr int kRecStages = kRowStages + kCopyAhead;
constexpr int kBarrierBytes = 64;  // copy mbarriers (8 bytes each) and flags
constexpr int kAbortSlot = 36;     // chunk at which a copy wait ran out
constexpr int kItemSlot = 40;      // current work item (int64)
static_assert(8 * kRawStages <= kAbortSlot && kItemSlot + 8 <= kBarrierBytes, "flag slots");

struct Tables {
  int nd_thr = 0, nd_cta = 0;
  int esize = 4;            // bytes per input element (2: f16, 4: f32)
  int opc = 1;              // octets per chunk
  int ntiles = 0, noctets = 0, nchan_pad = 0, nchunks = 0;
  int rec_words = 0;
  int32_t raw_stride = 0;   // elements per channel window slot (16-byte multiple)
  int32_t prow_words = 0;   // largest pattern-row area of any chunk, in words
  int32_t smem_bytes = 0;
  std::vector<int32_t> recs;      // [ntiles][nchunks][rec_words]
  std::vector<int32_t> raw_meta;  // [ntiles][nchan_pad][2]
  // Work-queue order: DM tile T runs its time tiles skew[T] places later in
  // the queue, skew[T] = the tile's smallest delay of the channel whose
  // largest delay is nearest half the plan's largest, in time tiles; so the
  // items in flight together read nearby input samples at every DM.
  std::vector<int32_t> skew;      // [ntiles]
  int32_t max_skew = 0;
};

// Shared-memory layout: mbarriers (kBarrierBytes), kRecStages records,
// kRawStages raw stages -- each a zero area of kZeroElems elements followed by
// 8*opc window slots of raw_stride elements, so that a unit's element offsets
// count from the stage's zero area --, kRowStages pattern-row areas.
inline int32_t zero_bytes(const Tables &t) { return kZeroElems * t.esize; }  // 16-byte multiple
inline int32_t rec_bytes(const Tables &t) { return t.rec_words * 4; }
inline int32_t raw_stage_bytes(const Tables &t) {
  return zero_bytes(t) + kGroup * t.opc * t.raw_stride * t.esize;
}
inline int32_t smem_bytes(const Tables &t) {
  return kBarrierBytes + kRecStages * rec_bytes(t) + kRawStages * raw_stage_bytes(t) +
         kRowStages * t.prow_words * 4;
}

// One beam of a launch of the (persistent) staged kernel: its block, output,
// tables and work items.  Work item i of the launch belongs to the last beam
// with item_begin <= i; within the beam, slot j = i - item_begin is DM tile
// T = j % ntiles_dm of time tile j / ntiles_dm - skew[T], an empty slot when
// that is outside 0 .. ntiles_t-1 (ntiles_dm * (ntiles_t + max_skew) slots).
struct Beam {
  const uint8_t *block;
  float *out;
  const int32_t *recs;
  const int32_t *raw_meta;
  const int32_t *skew;  // [ntiles_dm] time-tile offset of each DM tile in the queue
  // [ndm][ntiles_t] per (trial, time tile): {K, sum (D - K), sum (D - K)^2,
  // max D} over the tile's outputs, K its first output (null: none kept)
  float4 *tilestats;
  int64_t pitch_bytes;  // bytes per channel row (multiple of 16)
  int64_t nsamp_out;
  int64_t out_pitch;    // elements between output rows (>= nsamp_out)
  int64_t item_begin;
  int32_t ndm, nchunks, nchan_pad, rec_words, raw_stride, prow_words, ntiles_dm, ntiles_t;
  int32_t max_skew;
};
constexpr int kMaxBeams = 64;  // beams per launch (the descriptors travel as kernel parameters)

// Returns 0 and fills *tb, or 1 if this geometry needs more than
// kMaxPatterns patterns per octet and tile, shifts beyond kMaxShift, or more
// shared memory than a CTA has.  esize: 2 (f16) or 4 (f32).
int build_tables(const int32_t *delays, int32_t nchan, int32_t ndm, int nd_thr, int esize,
                 Tables *tb);

}  // namespace ddo
