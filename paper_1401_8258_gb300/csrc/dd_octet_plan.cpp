// dd_octet_plan.cpp -- plan-time tables of the staged octet kernel
// (dd_dedisp_octet.cu) for f16 and f32 input.
//
// The kernel adds eight channels per shared-memory word: for each group of
// eight adjacent channels ("octet") and each DM trial of the CTA's tile it
// reads a row whose word i holds the sum of the eight channels' samples that
// the trial adds at output time i.  Within an octet the delays of the
// channels relative to its reference channel (the middle one, kRefChan) take
// only a few distinct values over a tile of trials (differences of two
// rounded delays, Sec. 2.1.1), so one row per distinct relative pattern
// serves every trial of the tile that has it.  The rows are built by build
// units of 32 row words (dd_octet.h), planned here: which patterns each unit
// builds, the shifts it counts from, and which building warp takes it.
//
// Everything here is integer bookkeeping on the plan's delay table; no part
// of the dedispersion sum happens on the host.
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "dd_octet.h"

namespace {

inline int32_t round_up(int32_t v, int32_t m) { return (v + m - 1) / m * m; }
// largest multiple of m not above v (v may be negative)
inline int32_t floor_to(int32_t v, int32_t m) { return (v >= 0 ? v / m : -((-v + m - 1) / m)) * m; }

}  // namespace

namespace ddo {

int build_tables(const int32_t *delays, int32_t nchan, int32_t ndm, int nd_thr, int esize,
                 Tables *tb) {
  if (esize != 2 && esize != 4) return 1;
  const int nd_cta = kDmGroups * nd_thr;
  const int align = 16 / esize;  // elements per 16 bytes
  Tables t;
  t.nd_thr = nd_thr;
  t.nd_cta = nd_cta;
  t.esize = esize;
  t.opc = esize == 4 ? kOpcF32 : 2;
  t.ntiles = (ndm + nd_cta - 1) / nd_cta;
  t.noctets = (nchan + kGroup - 1) / kGroup;
  t.nchan_pad = t.noctets * kGroup;
  t.nchunks = (t.noctets + t.opc - 1) / t.opc;
  t.rec_words = rec_words(nd_cta);
  t.recs.assign(static_cast<size_t>(t.ntiles) * t.nchunks * t.rec_words, 0);
  t.raw_meta.assign(static_cast<size_t>(t.ntiles) * t.nchan_pad * 2, 0);

  // delay of (channel c, i-th trial of tile); padded trials reuse the last
  auto delay = [&](int tile, int c, int i) -> int32_t {
    const int d = std::min(tile * nd_cta + i, ndm - 1);
    return delays[static_cast<int64_t>(c) * ndm + d];
  };

  struct Octet {
    int32_t row_off, L, npat;
    int32_t shift[kMaxPatterns][kGroup];  // e_k(p) - emin[k]
    // row words of pattern p that some trial reads: lo[p] .. hi[p]-1 (the
    // reference delays of its trials, less b, plus the tile's samples)
    int32_t lo[kMaxPatterns], hi[kMaxPatterns];
    bool pad[kGroup];
    int32_t raw_off[kGroup];               // element offset of time b + emin[k] in its window
  };
  std::vector<std::vector<Octet>> chunk_octets(static_cast<size_t>(t.ntiles) * t.nchunks);
  int32_t raw_stride = align;
  int32_t prow_words = 4;
  for (int tile = 0; tile < t.ntiles; ++tile) {
    std::vector<int32_t> start(t.nchan_pad, 0), need(t.nchan_pad, 0);
    for (int ch = 0; ch < t.nchunks; ++ch) {
      int32_t *rec = &t.recs[(static_cast<size_t>(tile) * t.nchunks + ch) * t.rec_words];
      int32_t *A = rec + kRecHeader;
      std::vector<Octet> &octs = chunk_octets[static_cast<size_t>(tile) * t.nchunks + ch];
      int row_words = 0;
      const int o_lo = ch * t.opc;
      const int no = std::min(t.opc, t.noctets - o_lo);
      for (int o = 0; o < no; ++o) {
        const int c0 = kGroup * (o_lo + o);
        const int nreal = std::min(kGroup, nchan - c0);
        // the reference channel whose delay every pattern is relative to:
        // channel kRefChan of the octet (the middle, which keeps the other
        // channels' relative delays small), or its last real channel when
        // the octet has fewer; padding channels read zeros at any shift
        const int cref = c0 + std::min(kRefChan, nreal - 1);
        // distinct relative patterns of the real channels
        std::vector<std::array<int32_t, kGroup>> pats;
        std::vector<int> pid(nd_cta);
        int32_t b = INT32_MAX, bmax = INT32_MIN;
        for (int i = 0; i < nd_cta; ++i) {
          const int32_t d0 = delay(tile, cref, i);
          b = std::min(b, d0);
          bmax = std::max(bmax, d0);
          std::array<int32_t, kGroup> rel{};
          for (int k = 0; k < nreal; ++k) rel[k] = delay(tile, c0 + k, i) - d0;
          auto it = std::find(pats.begin(), pats.end(), rel);
          pid[i] = static_cast<int>(it - pats.begin());
          if (it == pats.end()) pats.push_back(rel);
        }
        if (static_cast<int>(pats.size()) > kMaxPatterns) return 1;
        Octet O;
        O.row_off = row_words;
        O.npat = static_cast<int32_t>(pats.size());
        O.L = round_up(kTimeTile + bmax - b, 4);
        for (int k = 0; k < kGroup; ++k) {
          const int c = c0 + k;
          O.pad[k] = k >= nreal;
          int32_t emin = INT32_MAX, emax = INT32_MIN;
          for (int p = 0; p < O.npat; ++p) {
            emin = std::min(emin, pats[p][k]);
            emax = std::max(emax, pats[p][k]);
          }
          if (emax - emin > kMaxShift) return 1;
          for (int p = 0; p < O.npat; ++p) O.shift[p][k] = pats[p][k] - emin;
          if (!O.pad[k]) {
            // window: times b + emin .. b + emax + L - 1; for channels below
            // the reference it may start before the first time tile's first
            // sample (the kernel then clips the copy: no output reads there)
            start[c] = floor_to(b + emin, align);
            O.raw_off[k] = b + emin - start[c];
            need[c] = O.raw_off[k] + (emax - emin) + O.L;
            raw_stride = std::max(raw_stride, round_up(need[c], align));
          } else {
            O.raw_off[k] = 0;
          }
        }
        for (int p = 0; p < O.npat; ++p) O.lo[p] = INT32_MAX, O.hi[p] = INT32_MIN;
        for (int i = 0; i < nd_cta; ++i) {
          const int32_t w0 = delay(tile, cref, i) - b;
          A[o * nd_cta + i] = row_words + pid[i] * O.L + w0;
          O.lo[pid[i]] = std::min(O.lo[pid[i]], w0);
          O.hi[pid[i]] = std::max(O.hi[pid[i]], w0 + kTimeTile);
        }
        row_words += O.npat * O.L;
        octs.push_back(O);
      }
      rec[2] = no;
      prow_words = std::max(prow_words, row_words);
    }
    for (int c = 0; c < t.nchan_pad; ++c) {
      int32_t *m = &t.raw_meta[(static_cast<size_t>(tile) * t.nchan_pad + c) * 2];
      m[0] = start[c];
      m[1] = c < nchan ? need[c] : 0;
    }
  }
  // raw-buffer element offsets must fit 16 bits (zero area first)
  const int64_t raw_elems = static_cast<int64_t>(kGroup) * t.opc * raw_stride;
  if (kZeroElems + raw_elems + 32 + kMaxShift >= 0xffff) return 1;
  constexpr int kWarps = kBuildWarps;
  for (size_t rc = 0; rc < chunk_octets.size(); ++rc) {
    int32_t *rec = &t.recs[rc * t.rec_words];
    // A build unit covers 32 row words of the consecutive patterns p0 ..
    // p1-1 of one octet: those whose trials read any of the 32 words (the
    // patterns in between included).
    auto make_unit = [&](const Octet &O, int o, int first, int p0, int p1) {
      std::array<int32_t, kUnitWords> u{};
      u[0] = (O.row_off + p0 * O.L + first) | (std::min(32, O.L - first) << 20);
      // per channel, the smallest shift over the unit's patterns (the unit's
      // offsets and codes count from it) and the largest past it; the unit's
      // bound is the largest over its channels if at most 2 (the kernel then
      // loads each channel's candidate samples once and selects per
      // pattern), 0 otherwise (it loads each pattern's samples)
      int32_t base[kGroup];
      int32_t smax = 0;
      uint32_t chan_bounds = 0;
      for (int k = 0; k < kGroup; ++k) {
        int32_t lo = INT32_MAX, hi = 0;
        for (int p = p0; p < p1; ++p) {
          lo = std::min(lo, O.pad[k] ? 0 : O.shift[p][k]);
          hi = std::max(hi, O.pad[k] ? 0 : O.shift[p][k]);
        }
        base[k] = lo;
        chan_bounds |= static_cast<uint32_t>(hi - lo) << (2 * k);
        smax = std::max(smax, hi - lo);
      }
      const int32_t bound = smax <= 2 ? std::max(smax, 1) : 0;
      u[1] = (p1 - p0) | (O.L << 8) | (bound << 29);
      for (int k = 0; k < kGroup; ++k) {
        // element offsets from the start of the zero area; the raw buffer
        // follows it (kZeroElems elements)
        const uint32_t e =
            O.pad[k] ? 0u
                     : static_cast<uint32_t>(kZeroElems + (kGroup * o + k) * raw_stride +
                                             O.raw_off[k] + base[k] + first);
        u[2 + k / 2] |= static_cast<int32_t>(e << (16 * (k & 1)));
      }
      // pattern-major shift codes: word kCodesWord + q/2 for the unit's q-th
      // pattern, 16 bits per pattern (two per word), channel k's shift at
      // bits 2k .. 2k+1 of its half; the reference channel's shift is 0
      for (int p = p0; p < p1; ++p) {
        uint32_t code = 0;
        for (int k = 0; k < kGroup; ++k)
          code |= static_cast<uint32_t>(O.pad[k] ? 0 : O.shift[p][k] - base[k]) << (2 * k);
        const int q = p - p0;
        u[kCodesWord + q / 2] |= static_cast<int32_t>(code << (16 * (q & 1)));
      }
      u[kBoundsWord] = static_cast<int32_t>(chan_bounds);
      return u;
    };
    // instructions of a unit, roughly: a fixed part (header, addresses),
    // the candidate loads and per pattern and channel a select per
    // candidate past the first and an add (or, on the general path, 8 loads
    // and adds per pattern)
    auto cost = [](const std::array<int32_t, kUnitWords> &u) {
      const int32_t npat = u[1] & 0xff, bound = (u[1] >> 29) & 3;
      return 24 + (bound ? 8 * (bound + 1) + npat * (7 * (1 + 2 * bound) + 3) : 4 + 24 * npat);
    };
    struct Cand {
      std::array<int32_t, kUnitWords> whole, half[2];
      int cost;
      bool split;  // has two pattern halves (two or more patterns)
    };
    std::vector<Cand> cands;
    for (size_t o = 0; o < chunk_octets[rc].size(); ++o) {
      const Octet &O = chunk_octets[rc][o];
      for (int first = 0; first < O.L; first += 32) {
        int p0 = O.npat, p1 = 0;
        for (int p = 0; p < O.npat; ++p)
          if (O.lo[p] < first + 32 && O.hi[p] > first) p0 = std::min(p0, p), p1 = p + 1;
        if (p0 >= p1) continue;  // words past every trial's reach
        auto add = [&](int a, int z) {
          Cand c;
          c.whole = make_unit(O, static_cast<int>(o), first, a, z);
          c.cost = cost(c.whole);
          c.split = z - a >= 2;
          if (c.split) {
            const int pm = a + (z - a) / 2;
            c.half[0] = make_unit(O, static_cast<int>(o), first, a, pm);
            c.half[1] = make_unit(O, static_cast<int>(o), first, pm, z);
          }
          cands.push_back(c);
        };
        // a unit whose channels span three shifts selects among three
        // candidates per channel; where two units on either side of some
        // pattern cost less in all, it is built as those two
        const auto whole = make_unit(O, static_cast<int>(o), first, p0, p1);
        int best = cost(whole), cut = -1;
        if (((whole[1] >> 29) & 3) == 2) {
          for (int q = p0 + 1; q < p1; ++q) {
            const int c = cost(make_unit(O, static_cast<int>(o), first, p0, q)) +
                          cost(make_unit(O, static_cast<int>(o), first, q, p1));
            if (c < best) best = c, cut = q;
          }
        }
        if (cut < 0) {
          add(p0, p1);
        } else {
          add(p0, cut);
          add(cut, p1);
        }
      }
    }
    // The building warps meet once per chunk, so the chunk takes as long as
    // its busiest warp: costliest unit first onto the least loaded warp,
    // with the 0 .. kMaxSplits costliest units split in two pattern halves
    // (each half reloads its candidates), whichever count leaves the busiest
    // warp least loaded.
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
        const int w = static_cast<int>(
            std::min_element(ld.begin() + kFirstBuilder, ld.end()) - ld.begin());
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
      const int w = static_cast<int>(
          std::min_element(load.begin() + kFirstBuilder, load.end()) - load.begin());
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
  // queue skew: the reference channel of the order is the one whose largest
  // delay is nearest half the largest of any channel
  {
    int32_t maxd = 0;
    for (int64_t i = 0; i < static_cast<int64_t>(nchan) * ndm; ++i) maxd = std::max(maxd, delays[i]);
    int cmid = 0;
    int64_t best = INT64_MAX;
    for (int c = 0; c < nchan; ++c) {
      int32_t dc = 0;
      for (int d = 0; d < ndm; ++d) dc = std::max(dc, delays[static_cast<int64_t>(c) * ndm + d]);
      const int64_t gap = std::llabs(2 * static_cast<int64_t>(dc) - maxd);
      if (gap < best) best = gap, cmid = c;
    }
    t.skew.assign(t.ntiles, 0);
    for (int tile = 0; tile < t.ntiles; ++tile) {
      int32_t b = INT32_MAX;
      for (int i = 0; i < nd_cta; ++i) b = std::min(b, delay(tile, cmid, i));
      t.skew[tile] = b / kTimeTile;
      t.max_skew = std::max(t.max_skew, t.skew[tile]);
    }
  }
  t.raw_stride = raw_stride;
  t.prow_words = prow_words;
  t.smem_bytes = smem_bytes(t);
  if (t.smem_bytes > kMaxSmem) return 1;
  *tb = std::move(t);
  return 0;
}

}  // namespace ddo

// Host-side access to the tables for the CPU tests (not part of dd.h).
// info[0..11) = {ok, nd_cta, ntiles, nchunks, nchan_pad, rec_words, raw_stride,
// prow_words, smem_bytes, opc, esize}; recs / raw_meta may be NULL.
extern "C" int ddi_octet_tables(const int32_t *delays, int32_t nchan, int32_t ndm, int32_t nd_thr,
                                int32_t esize, int32_t *info, int32_t *recs, int32_t *raw_meta) {
  ddo::Tables t;
  const int rc = ddo::build_tables(delays, nchan, ndm, nd_thr, esize, &t);
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
  info[9] = t.opc;
  info[10] = t.esize;
  if (recs) std::copy(t.recs.begin(), t.recs.end(), recs);
  if (raw_meta) std::copy(t.raw_meta.begin(), t.raw_meta.end(), raw_meta);
  return 0;
}
