// dd_quad_plan.cpp -- plan-time tables of the staged quad kernel
// (dd_dedisp_quad.cu) for u8 input.
//
// The kernel sums four channels per instruction (a byte dot product with
// weights 1,1,1,1).  For that it needs, for each group of four adjacent
// channels ("quad") and each DM trial of the CTA's tile, a shared-memory row
// whose 32-bit word i holds the four channels' samples that the trial adds
// at one output time.  Within a quad the delays of channels 1..3 relative to
// channel 0 take only a few distinct values over a tile of trials (they are
// differences of two rounded delays, Sec. 2.1.1), so one interleaved row per
// distinct relative pattern serves every trial of the tile that has it.
//
// Everything here is integer bookkeeping on the plan's delay table; no part
// of the dedispersion sum happens on the host.
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdint>
#include <vector>

#include "dd_quad.h"

namespace {

inline int32_t round_up(int32_t v, int32_t m) { return (v + m - 1) / m * m; }

}  // namespace

namespace ddq {

int build_tables(const int32_t *delays, int32_t nchan, int32_t ndm, int nd_thr, Tables *tb) {
  const int nd_cta = kDmGroups * nd_thr;
  Tables t;
  t.nd_thr = nd_thr;
  t.nd_cta = nd_cta;
  t.ntiles = (ndm + nd_cta - 1) / nd_cta;
  t.nquads = (nchan + 3) / 4;
  t.nchan_pad = t.nquads * 4;
  t.nchunks = (t.nquads + kQuadsPerChunk - 1) / kQuadsPerChunk;
  t.rec_words = rec_words(nd_cta);
  t.recs.assign(static_cast<size_t>(t.ntiles) * t.nchunks * t.rec_words, 0);
  t.raw_meta.assign(static_cast<size_t>(t.ntiles) * t.nchan_pad * 2, 0);

  // delay of (channel c, i-th trial of tile); padded channels reuse their
  // quad's channel 0 (their data is forced to zero), padded trials reuse the
  // last trial.
  auto delay = [&](int tile, int c, int i) -> int32_t {
    const int d = std::min(tile * nd_cta + i, ndm - 1);
    const int cc = c < nchan ? c : (c & ~3);
    return delays[static_cast<int64_t>(cc) * ndm + d];
  };

  int32_t raw_stride = 16;
  int32_t prow_words = 4;
  // rows of one chunk, kept until raw_stride is known: {row word offset,
  // items, quad, raw byte offset of channel k (-1 = padding)}
  struct Row {
    int32_t off, items, quad, o[4];
  };
  std::vector<std::vector<Row>> chunk_rows(static_cast<size_t>(t.ntiles) * t.nchunks);
  for (int tile = 0; tile < t.ntiles; ++tile) {
    // raw windows: channel c needs samples [t_cta + min delay, t_cta + T + max delay)
    std::vector<int32_t> start(t.nchan_pad), need(t.nchan_pad);
    for (int c = 0; c < t.nchan_pad; ++c) {
      int32_t mn = delay(tile, c, 0), mx = mn;
      for (int i = 1; i < nd_cta; ++i) {
        mn = std::min(mn, delay(tile, c, i));
        mx = std::max(mx, delay(tile, c, i));
      }
      start[c] = mn & ~15;
      need[c] = c < nchan ? mx + kTimeTile - start[c] : 0;
      int32_t *m = &t.raw_meta[(static_cast<size_t>(tile) * t.nchan_pad + c) * 2];
      m[0] = start[c];
      m[1] = need[c];
      raw_stride = std::max(raw_stride, round_up(need[c], 16));
    }
    for (int ch = 0; ch < t.nchunks; ++ch) {
      int32_t *rec = &t.recs[(static_cast<size_t>(tile) * t.nchunks + ch) * t.rec_words];
      int32_t *A = rec + kRecHeader;
      std::vector<Row> &rows = chunk_rows[static_cast<size_t>(tile) * t.nchunks + ch];
      int row_words = 0;
      const int q_lo = ch * kQuadsPerChunk;
      const int nq = std::min(kQuadsPerChunk, t.nquads - q_lo);
      for (int q = 0; q < nq; ++q) {
        const int c0 = 4 * (q_lo + q);
        // distinct relative patterns (delay of channel k minus channel 0)
        std::vector<std::array<int32_t, 3>> pats;
        std::vector<int> pid(nd_cta);
        for (int i = 0; i < nd_cta; ++i) {
          const int32_t d0 = delay(tile, c0, i);
          std::array<int32_t, 3> rel{delay(tile, c0 + 1, i) - d0, delay(tile, c0 + 2, i) - d0,
                                     delay(tile, c0 + 3, i) - d0};
          auto it = std::find(pats.begin(), pats.end(), rel);
          pid[i] = static_cast<int>(it - pats.begin());
          if (it == pats.end()) pats.push_back(rel);
        }
        if (static_cast<int>(pats.size()) > kMaxPatterns) return 1;
        for (size_t p = 0; p < pats.size(); ++p) {
          int32_t bmin = INT32_MAX, bmax = INT32_MIN;
          for (int i = 0; i < nd_cta; ++i)
            if (pid[i] == static_cast<int>(p)) {
              bmin = std::min(bmin, delay(tile, c0, i));
              bmax = std::max(bmax, delay(tile, c0, i));
            }
          Row r;
          r.off = row_words;
          r.items = round_up(kTimeTile + bmax - bmin, 4) / 4;
          r.quad = q;
          for (int k = 0; k < 4; ++k) {
            const int c = c0 + k;
            const int32_t e = k == 0 ? 0 : pats[p][k - 1];
            // bmin + e is a delay of channel c, so the offset is >= 0
            r.o[k] = c >= nchan ? -1 : bmin + e - start[c];
            if (r.o[k] >= 0) raw_stride = std::max(raw_stride, round_up(r.o[k] + 4 * r.items + 4, 16));
          }
          for (int i = 0; i < nd_cta; ++i)
            if (pid[i] == static_cast<int>(p)) A[q * nd_cta + i] = row_words + delay(tile, c0, i) - bmin;
          row_words += 4 * r.items;
          rows.push_back(r);
        }
      }
      rec[2] = nq;
      prow_words = std::max(prow_words, row_words);
    }
  }
  // segment descriptors (need the final raw_stride for the byte offsets)
  if (4 * kQuadsPerChunk * static_cast<int64_t>(raw_stride) >= 0xffff) return 1;
  for (size_t rc = 0; rc < chunk_rows.size(); ++rc) {
    int32_t *rec = &t.recs[rc * t.rec_words];
    int32_t *segs = rec + segs_offset(nd_cta);
    int nsegs = 0;
    for (const Row &r : chunk_rows[rc]) {
      for (int first = 0; first < r.items; first += 32) {
        if (nsegs == kMaxSegments) return 1;
        uint32_t addr[4], shift = 0;
        for (int k = 0; k < 4; ++k) {
          if (r.o[k] < 0) {
            addr[k] = 0xffff;
          } else {
            addr[k] = static_cast<uint32_t>((4 * r.quad + k) * raw_stride + (r.o[k] & ~3) + 4 * first);
            shift |= static_cast<uint32_t>(r.o[k] & 3) << (2 * k);
          }
        }
        const int32_t items = std::min(32, r.items - first);
        int32_t *sd = segs + nsegs * kSegWords;
        sd[0] = static_cast<int32_t>(addr[0] | (addr[1] << 16));
        sd[1] = static_cast<int32_t>(addr[2] | (addr[3] << 16));
        sd[2] = (r.off + 4 * first) | (items << 20);
        sd[3] = static_cast<int32_t>(shift);
        ++nsegs;
      }
    }
    rec[3] = nsegs;
  }
  t.raw_stride = raw_stride;
  t.prow_words = prow_words;
  t.smem_bytes = smem_bytes(t);
  if (t.smem_bytes > kMaxSmem) return 1;
  *tb = std::move(t);
  return 0;
}

}  // namespace ddq

// Host-side access to the tables for the CPU tests (not part of dd.h).
// info[0..9) = {ok, nd_cta, ntiles, nchunks, nchan_pad, rec_words, raw_stride,
// prow_words, smem_bytes}; recs / raw_meta may be NULL (sizes come from info).
extern "C" int ddi_quad_tables(const int32_t *delays, int32_t nchan, int32_t ndm, int32_t nd_thr,
                               int32_t *info, int32_t *recs, int32_t *raw_meta) {
  ddq::Tables t;
  const int rc = ddq::build_tables(delays, nchan, ndm, nd_thr, &t);
  info[0] = rc == 0;
  if (rc != 0) return 0;
  info[1] = t.nd_cta;
  info[2] = t.ntiles;
  info[3] = t.nchunks;
  info[4] = t.nchan_pad;
  info[5] = t.rec_words;
  info[6] = t.raw_stride;
  info[7] = t.prow_words;
  info[8] = t.smem_bytes;
  if (recs) std::copy(t.recs.begin(), t.recs.end(), recs);
  if (raw_meta) std::copy(t.raw_meta.begin(), t.raw_meta.end(), raw_meta);
  return 0;
}
