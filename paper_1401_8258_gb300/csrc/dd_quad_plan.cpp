// dd_quad_plan.cpp -- plan-time tables of the staged quad kernel
// (dd_dedisp_quad.cu) for u8 input.
//
// The kernel adds eight channel samples per 32-bit shared-memory word: for
// each group of four adjacent channels ("quad") and each DM trial of the
// CTA's tile it reads a row whose word i holds the sum of the four channels'
// samples that the trial adds at output time i (low 16 bits) and at time
// i + kHalf (high 16 bits).  Within a quad the delays of channels 1..3
// relative to channel 0 take only a few distinct values over a tile of
// trials (they are differences of two rounded delays, Sec. 2.1.1), so one
// row per distinct relative pattern serves every trial of the tile that has
// it.
//
// Everything here is integer bookkeeping on the plan's delay table; no part
// of the dedispersion sum happens on the host.
#include <algorithm>
#include <array>
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
  // quads of one chunk, kept until raw_stride is known
  struct Quad {
    int32_t row_off, L, npat;
    int32_t emin[4];               // smallest relative delay of channel k over the patterns
    int32_t shift[kMaxPatterns][4];  // e_k(p) - emin[k]
    bool pad[4];
    int32_t raw_off[4];            // byte offset of time b + emin[k] in channel k's window
    // row words of pattern p that some trial reads: lo[p] .. hi[p]-1 (the
    // channel-0 delays of its trials, less b, plus the tile's pairs)
    int32_t lo[kMaxPatterns], hi[kMaxPatterns];
  };
  // slack x (row origin b - x) for which every real channel's byte shifts
  // (b - x + emin) & 3 .. + spread stay within 0..4, i.e. inside two words
  auto slack_for = [&](int32_t b, const int32_t *emin, const int32_t *emax, const bool *pad) {
    for (int x = 0; x < 4; ++x) {
      bool fits = true;
      for (int k = 0; k < 4; ++k)
        if (!pad[k] && ((b - x + emin[k]) & 3) + emax[k] - emin[k] > 4) fits = false;
      if (fits) return x;
    }
    return -1;
  };
  std::vector<std::vector<Quad>> chunk_quads(static_cast<size_t>(t.ntiles) * t.nchunks);
  for (int tile = 0; tile < t.ntiles; ++tile) {
    std::vector<int32_t> start(t.nchan_pad, 0), need(t.nchan_pad, 0);
    for (int ch = 0; ch < t.nchunks; ++ch) {
      int32_t *rec = &t.recs[(static_cast<size_t>(tile) * t.nchunks + ch) * t.rec_words];
      int32_t *A = rec + kRecHeader;
      std::vector<Quad> &quads = chunk_quads[static_cast<size_t>(tile) * t.nchunks + ch];
      int row_words = 0;
      const int q_lo = ch * kQuadsPerChunk;
      const int nq = std::min(kQuadsPerChunk, t.nquads - q_lo);
      for (int q = 0; q < nq; ++q) {
        const int c0 = 4 * (q_lo + q);
        // distinct relative patterns (delay of channel k minus channel 0)
        std::vector<std::array<int32_t, 3>> pats;
        std::vector<int> pid(nd_cta);
        int32_t b = INT32_MAX, bmax = INT32_MIN;
        for (int i = 0; i < nd_cta; ++i) {
          const int32_t d0 = delay(tile, c0, i);
          b = std::min(b, d0);
          bmax = std::max(bmax, d0);
          std::array<int32_t, 3> rel{delay(tile, c0 + 1, i) - d0, delay(tile, c0 + 2, i) - d0,
                                     delay(tile, c0 + 3, i) - d0};
          auto it = std::find(pats.begin(), pats.end(), rel);
          pid[i] = static_cast<int>(it - pats.begin());
          if (it == pats.end()) pats.push_back(rel);
        }
        if (static_cast<int>(pats.size()) > kMaxPatterns) return 1;
        Quad Q;
        Q.row_off = row_words;
        Q.npat = static_cast<int32_t>(pats.size());
        int32_t emax[4];
        for (int k = 0; k < 4; ++k) {
          Q.pad[k] = c0 + k >= nchan;
          Q.emin[k] = INT32_MAX;
          emax[k] = INT32_MIN;
          for (int p = 0; p < Q.npat; ++p) {
            const int32_t e = k == 0 ? 0 : pats[p][k - 1];
            Q.emin[k] = std::min(Q.emin[k], e);
            emax[k] = std::max(emax[k], e);
          }
          for (int p = 0; p < Q.npat; ++p)
            Q.shift[p][k] = (k == 0 ? 0 : pats[p][k - 1]) - Q.emin[k];
        }
        const int x = slack_for(b, Q.emin, emax, Q.pad);
        if (x < 0) return 1;
        b -= x;  // may reach -3 for the first tile; those row words are never read
        Q.L = round_up(kHalf + bmax - b, 4);
        for (int k = 0; k < 4; ++k) {
          const int c = c0 + k;
          if (!Q.pad[k]) {
            // two words per item and half: the last item's words end at
            // (raw_off & ~3) + L + kHalf + 4 bytes into the window
            start[c] = (b + Q.emin[k]) & ~15;
            Q.raw_off[k] = b + Q.emin[k] - start[c];
            need[c] = (Q.raw_off[k] & ~3) + Q.L + kHalf + 4;
            raw_stride = std::max(raw_stride, round_up(need[c], 16));
          } else {
            Q.raw_off[k] = 0;
          }
        }
        for (int p = 0; p < Q.npat; ++p) Q.lo[p] = INT32_MAX, Q.hi[p] = INT32_MIN;
        for (int i = 0; i < nd_cta; ++i) {
          const int32_t w0 = delay(tile, c0, i) - b;
          A[q * nd_cta + i] = row_words + pid[i] * Q.L + w0;
          Q.lo[pid[i]] = std::min(Q.lo[pid[i]], w0);
          Q.hi[pid[i]] = std::max(Q.hi[pid[i]], w0 + kHalf);
        }
        row_words += Q.npat * Q.L;
        quads.push_back(Q);
      }
      rec[2] = nq;
      prow_words = std::max(prow_words, row_words);
    }
    for (int c = 0; c < t.nchan_pad; ++c) {
      int32_t *m = &t.raw_meta[(static_cast<size_t>(tile) * t.nchan_pad + c) * 2];
      m[0] = start[c];
      m[1] = c < nchan ? need[c] : 0;
    }
  }
  // build units (need the final raw_stride for the byte offsets)
  if (4 * kQuadsPerChunk * static_cast<int64_t>(raw_stride) >= 0xffff) return 1;
  constexpr int kWarps = kBuildWarps;
  for (size_t rc = 0; rc < chunk_quads.size(); ++rc) {
    int32_t *rec = &t.recs[rc * t.rec_words];
    // A build unit covers items first .. first+31 (4 row words each) of the
    // consecutive patterns p0 .. p1-1 of one quad: those whose trials read
    // any of its words (the patterns in between included).
    auto make_unit = [&](const Quad &Q, int q, int first, int p0, int p1) {
      const int items = Q.L / 4;
      uint32_t addr[4];
      for (int k = 0; k < 4; ++k)
        addr[k] = Q.pad[k] ? 0xffffu
                           : static_cast<uint32_t>((4 * q + k) * raw_stride +
                                                   (Q.raw_off[k] & ~3) + 4 * first);
      std::array<int32_t, kUnitWords> u{};
      u[0] = static_cast<int32_t>(addr[0] | (addr[1] << 16));
      u[1] = static_cast<int32_t>(addr[2] | (addr[3] << 16));
      u[2] = (Q.row_off + p0 * Q.L + 4 * first) | (std::min(32, items - first) << 20) |
             ((p1 - p0) << 26);
      // prmt selector of the 4 bytes starting s bytes into two words
      auto sel = [&](int p, int k) {
        return 0x3210u + 0x1111u * static_cast<uint32_t>((Q.raw_off[k] & 3) + Q.shift[p][k]);
      };
      u[3] = static_cast<int32_t>(static_cast<uint32_t>(Q.L) | (sel(0, 0) << 16));
      for (int p = p0; p < p1; ++p) {
        u[4 + 2 * (p - p0)] = static_cast<int32_t>(sel(p, 1) | (sel(p, 2) << 16));
        u[5 + 2 * (p - p0)] = static_cast<int32_t>(sel(p, 3));
      }
      return u;
    };
    // cost of a unit ~ its loads + one row store per pattern
    auto cost = [](const std::array<int32_t, kUnitWords> &u) {
      return 2 + static_cast<int>(static_cast<uint32_t>(u[2]) >> 26);
    };
    struct Cand {
      std::array<int32_t, kUnitWords> whole, half[2];
      int cost;
      bool split;  // has two pattern halves (two or more patterns)
    };
    std::vector<Cand> cands;
    for (size_t q = 0; q < chunk_quads[rc].size(); ++q) {
      const Quad &Q = chunk_quads[rc][q];
      const int items = Q.L / 4;
      for (int first = 0; first < items; first += 32) {
        int p0 = Q.npat, p1 = 0;
        for (int p = 0; p < Q.npat; ++p)
          if (Q.lo[p] < 4 * (first + 32) && Q.hi[p] > 4 * first) p0 = std::min(p0, p), p1 = p + 1;
        if (p0 >= p1) continue;  // words past every trial's reach
        Cand c;
        c.whole = make_unit(Q, static_cast<int>(q), first, p0, p1);
        c.cost = cost(c.whole);
        c.split = p1 - p0 >= 2;
        if (c.split) {
          const int pm = p0 + (p1 - p0) / 2;
          c.half[0] = make_unit(Q, static_cast<int>(q), first, p0, pm);
          c.half[1] = make_unit(Q, static_cast<int>(q), first, pm, p1);
        }
        cands.push_back(c);
      }
    }
    // The building warps meet once per chunk, so the chunk takes as long as
    // its busiest warp: largest unit first onto the least loaded warp, with
    // the 0 .. kMaxSplits largest units split in two pattern halves (each
    // half reloads its words), whichever count leaves the busiest warp least
    // loaded; then the units are ordered by warp.
    std::stable_sort(cands.begin(), cands.end(),
                     [](const Cand &x, const Cand &y) { return x.cost > y.cost; });
    constexpr int kMaxSplits = 6;
    std::vector<std::array<int32_t, kUnitWords>> list;
    std::vector<int> order;
    int best_span = INT32_MAX;
    for (int nsplit = 0; nsplit <= kMaxSplits; ++nsplit) {
      std::vector<std::array<int32_t, kUnitWords>> l;
      for (size_t i = 0; i < cands.size(); ++i) {
        if (static_cast<int>(i) < nsplit && cands[i].split) {
          l.push_back(cands[i].half[0]);
          l.push_back(cands[i].half[1]);
        } else {
          l.push_back(cands[i].whole);
        }
      }
      if (static_cast<int>(l.size()) > kMaxUnits) break;
      std::vector<int> ord(l.size());
      for (size_t i = 0; i < ord.size(); ++i) ord[i] = static_cast<int>(i);
      std::stable_sort(ord.begin(), ord.end(),
                       [&](int x, int y) { return cost(l[x]) > cost(l[y]); });
      std::vector<int> ld(kWarps, 0);
      for (int i : ord) {
        const int w = static_cast<int>(std::min_element(ld.begin(), ld.end()) - ld.begin());
        ld[w] += cost(l[i]);
      }
      const int span = *std::max_element(ld.begin(), ld.end());
      if (span < best_span) {
        best_span = span;
        list.swap(l);
        order.swap(ord);
      }
    }
    if (best_span == INT32_MAX) return 1;  // more units than a record holds
    std::vector<int> load(kWarps, 0);
    std::vector<std::vector<int>> per_warp(kWarps);
    for (int i : order) {
      const int w = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
      load[w] += cost(list[i]);
      per_warp[w].push_back(i);
    }
    int32_t *units = rec + units_offset(nd_cta);
    uint16_t *starts = reinterpret_cast<uint16_t *>(rec + warp_start_offset(nd_cta));
    int n = 0;
    for (int w = 0; w < kWarps; ++w) {
      starts[w] = static_cast<uint16_t>(n);
      for (int i : per_warp[w]) {
        for (int j = 0; j < kUnitWords; ++j) units[n * kUnitWords + j] = list[i][j];
        ++n;
      }
    }
    starts[kWarps] = static_cast<uint16_t>(n);
    rec[3] = n;
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
