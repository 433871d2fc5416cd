// dd_quad.h -- shape constants and plan-time tables of the staged quad
// kernel for u8 input (internal to libdd).
//
// CTA tile: kDmGroups x nd_thr DM trials by kTimeTile output samples, taken
// as kHalf sample pairs (t, t + kHalf).  Two warp roles: 16 accumulating
// warps = kDmGroups DM groups x kTimeGroups time groups (16 x 1), a thread
// owning nd_thr trials (4) x kPairsPerThread pairs (8; pair = base + lane +
// 32*j); and kBuildWarps (12) building warps that queue the copies and build
// the pattern rows one chunk ahead.  Channels are processed in chunks of
// kQuadsPerChunk quads (4 channels each).
//
// Pattern rows.  For quad q of a DM tile, let b be the smallest channel-0
// delay over the tile's trials, less a per-quad slack x in 0..3 (chosen so
// that every channel's byte shifts fit two loaded words, below).  Each
// distinct relative-delay pattern p of the quad has a row of L words
// (L = kHalf + largest channel-0 delay - b, rounded up to 4); word i of row p
// holds two 16-bit sums over the quad's channels k = 0..3:
//   low half   sum_k I[c_k][t_cta + b + e_k(p) + i]
//   high half  sum_k I[c_k][t_cta + b + e_k(p) + i + kHalf]
// e_k(p) being channel k's delay minus channel 0's in that pattern.  The rows
// of a quad are contiguous.
//
// Per (DM tile, chunk) record, int32 words:
//   [0] unused                   [1] unused
//   [2] quads in this chunk      [3] number of build units
//   A[kQuadsPerChunk][nd_cta]    word offset, within the chunk's pattern-row
//                                area, of the row word that holds output
//                                pair 0 of the tile for that quad and trial
//   units[kMaxUnits][20]: one warp-wide build step each -- items first ..
//     first+31 (item = 4 row words) of the consecutive pattern rows p0 .. of
//     one quad (those that some trial of the tile reads there, or a half of
//     them); lane l builds item first+l of each row:
//     [0] raw-buffer byte offsets of channels 0 | 1 << 16, [1] of 2 | 3 << 16:
//         the aligned word holding the earliest sample any pattern of the
//         quad needs for this item block (0xffff = padding channel, zeros);
//     [2] row-area word offset of item `first` of row p0 | items << 20 |
//         patterns << 26;
//     [3] row length L in words | channel 0's byte selector << 16;
//     [4 + 2p], [5 + 2p] for the unit's p-th pattern: byte selectors (prmt) of channels
//         1 | 2 << 16, and 3: for a byte shift s (0..4) of the pattern's
//         first sample within the two loaded words, 0x3210 + 0x1111 s (the
//         same shift serves the second half, kHalf bytes on).  Channel 0's
//         shift is the same for every pattern (its relative delay is 0).
//   warp_start[kBuildWarps + 1] (int16 pairs, after the units): the units
//     are ordered by the building warp that builds them (balanced on the
//     host, largest first onto the least loaded warp); building warp w builds
//     units warp_start[w] .. warp_start[w+1]-1.
// raw_meta[tile][nchan_pad][2]: {window start relative to the tile's first
// output sample (a multiple of 16; -16 where the slack reaches before the
// first sample), bytes needed (0 = padding channel)}.
#pragma once

#include <cstdint>
#include <vector>

#ifdef __CUDACC__
#define DDQ_HD __host__ __device__
#else
#define DDQ_HD
#endif

namespace ddq {

// Tile shape; the DDQ_* macros exist only to build shape variants for tuning.
#ifndef DDQ_DM_GROUPS
#define DDQ_DM_GROUPS 16
#endif
#ifndef DDQ_TIME_GROUPS
#define DDQ_TIME_GROUPS 1
#endif
#ifndef DDQ_TIMES_PER_THREAD
#define DDQ_TIMES_PER_THREAD 16
#endif
#ifndef DDQ_QUADS_PER_CHUNK
#define DDQ_QUADS_PER_CHUNK 4
#endif
#ifndef DDQ_ND_THR
#define DDQ_ND_THR 4
#endif
constexpr int kDmGroups = DDQ_DM_GROUPS;
constexpr int kTimeGroups = DDQ_TIME_GROUPS;
#ifndef DDQ_BUILD_WARPS
#define DDQ_BUILD_WARPS 12
#endif
constexpr int kAccThreads = 32 * kDmGroups * kTimeGroups;             // 512
constexpr int kBuildWarps = DDQ_BUILD_WARPS;
constexpr int kThreads = kAccThreads + 32 * kBuildWarps;              // 896
constexpr int kTimesPerThread = DDQ_TIMES_PER_THREAD;
constexpr int kTimeTile = kTimeGroups * 32 * kTimesPerThread;         // 512
constexpr int kHalf = kTimeTile / 2;                                  // pair (t, t + kHalf)
constexpr int kPairsPerThread = kTimesPerThread / 2;
// A row word half holds at most 4*255; an accumulator half takes 64 quads
// (64*1020 = 65280 < 65536) before it is drained into 32-bit sums.
constexpr int kFlushQuads = 64;
constexpr int kQuadsPerChunk = DDQ_QUADS_PER_CHUNK;
constexpr int kNdThr = DDQ_ND_THR;  // DM trials per thread of the wide variant
constexpr int kMaxPatterns = 8;
constexpr int kRecHeader = 4;
constexpr int kUnitWords = 4 + 2 * kMaxPatterns;  // 20 (80 bytes)
constexpr int kMaxUnits = 32;
constexpr int kMaxSmem = 227 * 1024;

DDQ_HD constexpr int units_offset(int nd_cta) { return kRecHeader + kQuadsPerChunk * nd_cta; }
DDQ_HD constexpr int warp_start_offset(int nd_cta) { return units_offset(nd_cta) + kMaxUnits * kUnitWords; }
DDQ_HD constexpr int rec_words(int nd_cta) {
  return (warp_start_offset(nd_cta) + (kBuildWarps + 2) / 2 + 3) / 4 * 4;
}

#ifndef DDQ_COPY_AHEAD
#define DDQ_COPY_AHEAD 2
#endif
constexpr int kCopyAhead = DDQ_COPY_AHEAD;  // default staging depth (chunks queued ahead)

struct Tables {
  int nd_thr = 0, nd_cta = 0;
  int copy_ahead = kCopyAhead;  // staging depth that smem_bytes is computed for
  int ntiles = 0, nquads = 0, nchan_pad = 0, nchunks = 0;
  int rec_words = 0;
  int32_t raw_stride = 0;   // bytes per channel window slot (multiple of 16)
  int32_t prow_words = 0;   // largest pattern-row area of any chunk, in words
  int32_t smem_bytes = 0;
  std::vector<int32_t> recs;      // [ntiles][nchunks][rec_words]
  std::vector<int32_t> raw_meta;  // [ntiles][nchan_pad][2]
};

// Pipeline depth: the building warps queue the copies of a chunk copy_ahead
// chunks ahead of the one they build (the staging depth, kMinCopyAhead ..
// kMaxCopyAhead, compiled for each and picked by the autotuner; kCopyAhead by
// default), and the rows of chunk k+1 are built while chunk k is
// accumulated (kRowStages row areas).
#ifndef DDQ_ROW_STAGES
#define DDQ_ROW_STAGES 2
#endif
constexpr int kRowStages = DDQ_ROW_STAGES;
constexpr int kMinCopyAhead = 1, kMaxCopyAhead = 3;
// raw window buffers: the chunk being built and the copy_ahead queued after it
DDQ_HD constexpr int raw_stages(int copy_ahead) { return copy_ahead + 1; }
// a record stays in use until the accumulating warps are done with its
// chunk, up to kRowStages chunks behind the building warps, which queue
// copies copy_ahead chunks ahead
DDQ_HD constexpr int rec_stages(int copy_ahead) { return kRowStages + copy_ahead; }
constexpr int kBarrierBytes = 64;  // copy mbarriers (8 bytes each), tensor-memory address, flags
constexpr int kTmemSlot = 32;      // byte offset of the tensor-memory address
constexpr int kAbortSlot = 36;     // chunk at which a copy wait ran out
constexpr int kItemSlot = 40;      // current work item (int64)

// Shared-memory layout: the mbarriers and tensor-memory address (kBarrierBytes), the tile's raw
// window table (nchan_pad x 2 int32), rec_stages records, raw_stages raw
// window buffers (4*kQuadsPerChunk slots of raw_stride bytes), kRowStages
// pattern-row areas.
inline int32_t rec_bytes(const Tables &t) { return t.rec_words * 4; }
inline int32_t raw_buf_bytes(const Tables &t) { return 4 * kQuadsPerChunk * t.raw_stride; }
inline int32_t meta_bytes(const Tables &t) { return (t.nchan_pad * 8 + 15) / 16 * 16; }
inline int32_t smem_bytes(const Tables &t) {
  return kBarrierBytes + meta_bytes(t) + rec_stages(t.copy_ahead) * rec_bytes(t) +
         raw_stages(t.copy_ahead) * raw_buf_bytes(t) + kRowStages * t.prow_words * 4;
}
// Staging depth of the tables (the records and windows do not depend on it,
// only the shared-memory size); false if that depth does not fit a CTA.
inline bool set_copy_ahead(Tables &t, int copy_ahead) {
  t.copy_ahead = copy_ahead;
  t.smem_bytes = smem_bytes(t);
  return copy_ahead >= kMinCopyAhead && copy_ahead <= kMaxCopyAhead && t.smem_bytes <= kMaxSmem;
}

// Returns 0 and fills *tb, or 1 if this geometry needs more than
// kMaxPatterns patterns per quad and tile or more shared memory than a CTA has.
int build_tables(const int32_t *delays, int32_t nchan, int32_t ndm, int nd_thr, Tables *tb);

// One beam of a launch of the (persistent) staged kernel: its block, output,
// tables and work items.  Work item i of the launch belongs to the last beam
// with item_begin <= i; within the beam, item (i - item_begin) is DM tile
// (i - item_begin) % ntiles_dm of time tile (i - item_begin) / ntiles_dm.
struct Beam {
  const uint8_t *block;
  int32_t *out;
  const int32_t *recs;
  const int32_t *raw_meta;
  int64_t *rowsums;  // [ndm][2] += exact sum D, sum D^2 (null: no statistics)
  int32_t *tilemax;  // [ndm][ntiles_t] largest output of each time tile
  int64_t pitch;     // bytes per channel row (multiple of 16)
  int64_t nsamp_out;
  int64_t out_pitch;  // elements between output rows (>= nsamp_out)
  int64_t item_begin;
  int32_t ndm, nchunks, nchan_pad, rec_words, raw_stride, prow_words, ntiles_dm, ntiles_t;
  int32_t nd_thr;  // trials per accumulating thread of this beam's tables (tile width / 16)
};
constexpr int kMaxBeams = 64;  // beams per launch (the descriptors travel as kernel parameters)

}  // namespace ddq
