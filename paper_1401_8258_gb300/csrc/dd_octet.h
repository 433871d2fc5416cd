// dd_octet.h -- shape constants and plan-time tables of the staged octet
// kernel for f16 and f32 input (internal to libdd).
//
// CTA tile: kDmGroups x nd_thr DM trials (16 x 8 = 128, or 16 x 4 = 64) by
// kTimeTile (256) output samples.  16 warps = 16 DM groups; a thread owns
// nd_thr trials x kTimesPerThread samples (sample = lane + 32*j).  Channels
// are taken in groups of kGroup = 8 adjacent channels ("octets"), `opc` (2)
// octets per chunk.
//
// Pattern rows.  For octet o of a DM tile, let b be the smallest channel-0
// delay over the tile's trials.  Each distinct relative-delay pattern p of
// the octet has a row of L float words (L = kTimeTile + largest channel-0
// delay - b, rounded up to 4); word i of row p holds the sum over the octet's
// channels k of I[c_k][t_cta + b + e_k(p) + i], e_k(p) being channel k's
// delay minus channel 0's in that pattern.  The rows of an octet are
// contiguous.
//
// Per (DM tile, chunk) record, int32 words:
//   [0] unused                 [1] unused
//   [2] octets in this chunk   [3] number of build units
//   A[kMaxOctetsPerChunk][nd_cta]  word offset, within the chunk's row area,
//                              of the row word that holds output sample 0 of
//                              the tile for that octet and trial
//   units[kMaxUnits][16]: one warp-wide build step each -- items first ..
//     first+31 (item = one row word) of every pattern row of one octet; lane
//     l builds item first+l:
//     [0] row-area word offset of item `first` of row 0 | items << 20
//     [1] patterns | L << 8 | fast << 30 (fast: every shift is 0 or 1)
//     [2..5] element offsets, from the raw stage's zero area, of channels
//         0..7 (16 bits each, two per word): the earliest sample any pattern
//         needs for item `first`; padding channels point into the zero area
//     [6..13] per pattern p (two per word, 16 bits each): for channel k a
//         2-bit element shift 0..3 of the pattern's sample past that offset
//   warp_start[kThreads/32 + 1] (int16 pairs, after the units): warp w builds
//     units warp_start[w] .. warp_start[w+1]-1 (balanced on the host).
// raw_meta[tile][nchan_pad][2]: {window start in elements relative to the
// tile's first output sample (16-byte aligned), elements needed (0 = padding
// channel)}.
#pragma once

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
constexpr int kDmGroups = 16;
constexpr int kThreads = 32 * kDmGroups;                 // 512
constexpr int kTimesPerThread = DDO_TIMES_PER_THREAD;
constexpr int kTimeTile = 32 * kTimesPerThread;          // 256
constexpr int kNdThr = DDO_ND_THR;                       // trials per thread (128 per CTA)
constexpr int kOpcF32 = DDO_OPC_F32;                     // octets per chunk for f32 input
constexpr int kMaxOctetsPerChunk = 2;
constexpr int kMaxPatterns = 16;
constexpr int kMaxShift = 3;                             // element shifts 0..3 within a unit
constexpr int kRecHeader = 4;
constexpr int kUnitWords = 16;
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
  return (warp_start_offset(nd_cta) + (kThreads / 32 + 2) / 2 + 3) / 4 * 4;
}

constexpr int kRawStages = 3;
constexpr int kRecStages = 4;
constexpr int kRowStages = 2;
constexpr int kBarrierBytes = 64;  // copy mbarriers (8 bytes each)

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

// Returns 0 and fills *tb, or 1 if this geometry needs more than
// kMaxPatterns patterns per octet and tile, shifts beyond kMaxShift, or more
// shared memory than a CTA has.  esize: 2 (f16) or 4 (f32).
int build_tables(const int32_t *delays, int32_t nchan, int32_t ndm, int nd_thr, int esize,
                 Tables *tb);

}  // namespace ddo
