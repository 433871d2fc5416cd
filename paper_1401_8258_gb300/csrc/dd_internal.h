// dd_internal.h -- plan object and kernel launchers shared by the libdd
// translation units (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <vector>

#include "dd.h"
#include "dd_octet.h"
#include "dd_quad.h"

// A device array of plan tables, freed with the last plan that holds it:
// plans made with dd_plan_create_like share their source's tables.
struct DeviceTable {
  int32_t *ptr = nullptr;
  DeviceTable() = default;
  DeviceTable(const DeviceTable &) = delete;
  DeviceTable &operator=(const DeviceTable &) = delete;
  ~DeviceTable() {
    if (ptr) cudaFree(ptr);
  }
};
using SharedTable = std::shared_ptr<DeviceTable>;

// Device copies of the staged quad kernel's plan-time tables.  `tables`
// keeps the shape fields (its record and window vectors are emptied once
// uploaded); d_recs / d_raw_meta alias the shared device arrays.
struct QuadDevice {
  ddq::Tables tables;
  SharedTable recs_store, meta_store;
  int32_t *d_recs = nullptr;
  int32_t *d_raw_meta = nullptr;
};

// Device copies of the staged octet kernel's plan-time tables (and the work
// queue's per-DM-tile skews, after the window table in the same array).
struct OctetDevice {
  ddo::Tables tables;
  SharedTable recs_store, meta_store;
  int32_t *d_recs = nullptr;
  int32_t *d_raw_meta = nullptr;
  int32_t *d_skew = nullptr;
};

// Per-DM-row normalisation result written by the statistics kernels, with
// the row's candidate threshold for the current nsigma: the smallest value v
// (an int32 for integer rows, a float for real rows) whose snr,
// ((double)v - mean) / sigma in IEEE double, exceeds nsigma.  Because that
// double expression is monotone in v, "v >= threshold" decides exactly what
// "snr > nsigma" decides.
struct dd_row_stats {
  double mean;
  double sigma;
  int64_t ithr;  // integer rows: candidates are D >= ithr
  float fthr;    // real rows: candidates are D >= fthr
  int32_t any;   // 0: no sample of this row can be a candidate (sigma == 0)
};

struct dd_plan {
  int device = 0;
  int32_t nchan = 0;
  int32_t ndm = 0;
  int32_t dtype = DD_U8;
  double f_top = 0, df = 0, t_samp = 0;
  std::vector<double> dms;
  std::shared_ptr<std::vector<int32_t>> h_delays;  // [nchan][ndm] (shared by like plans)
  int32_t maxshift = 0;
  int sm_count = 0;

  SharedTable delays_store;       // device delay table (shared by like plans)
  int32_t *d_delays = nullptr;    // [nchan][ndm], aliases delays_store
  // sticky device status word (0 = ok); it lies in d_total's allocation
  // (word 2), so that one 16-byte copy brings a call's total and status back
  int32_t *d_error = nullptr;

  // detection workspace
  dd_row_stats *d_stats = nullptr;  // [ndm]
  int64_t *d_counts = nullptr;      // [ndm * nchunks] per-chunk candidate counts
  int64_t *d_offsets = nullptr;     // [ndm * nchunks] exclusive prefix of d_counts
  int64_t *d_total = nullptr;       // [2]: candidate total, then the status word d_error
  int64_t *h_total = nullptr;       // pinned [2]: the copy of d_total[0..1]
  int64_t *h_total_dev = nullptr;   // device address of h_total (mapped pinned memory)
  size_t chunk_cap = 0;             // entries allocated in d_counts / d_offsets
  std::vector<double> h_mean, h_sigma;
  bool stats_valid = false;

  // workspace of the fused path (dd_run with the staged kernel)
  int64_t *d_rowsums = nullptr;     // [ndm][2] exact S1, S2 from the dedispersion kernel
  int64_t *d_rowcount = nullptr;    // [ndm] candidates per row
  int64_t *d_rowoff = nullptr;      // [ndm] exclusive prefix of d_rowcount
  int32_t *d_tilemax = nullptr;     // [ndm * ntiles] largest output of each time tile
  int32_t *d_tilecount = nullptr;   // [ndm * ntiles] candidates per time tile
  size_t tile_cap = 0;              // entries allocated in d_tilemax / d_tilecount
  float4 *d_tilestats = nullptr;    // [ndm * ntiles] float rows: per-tile partial statistics
  size_t tilestats_cap = 0;         // entries allocated in d_tilestats

  // buffers owned for dd_process_host
  void *d_block = nullptr;
  size_t d_block_bytes = 0;
  void *d_out = nullptr;
  size_t d_out_bytes = 0;
  dd_candidate *d_cands = nullptr;
  size_t d_cands_cap = 0;

  QuadDevice *quad = nullptr;       // staged u8 kernel tables (null: not applicable)
  unsigned long long *d_next_item = nullptr;  // work-queue head of the staged kernels
  OctetDevice *octet = nullptr;     // staged f16/f32 kernel tables (null: not applicable)
  int32_t path = 0;                 // 0 = automatic, 1 = plain-load kernel only
  uint64_t wait_timeout_ns = 2000000000ull;  // bound on every device-side wait
  int32_t debug_skip_copies = 0;    // fault injection: staged kernel queues no copies

  // one-launch path for small float beams (dd_run): arrivals counter of its
  // grid barrier; each launch adds its CTAs' arrivals to `arrivals_base`
  unsigned long long *d_arrivals = nullptr;
  uint64_t arrivals_base = 0;
  // and each row's candidate count as published in its launch ([ndm]:
  // launch epoch << 24 | count; zero before the first launch)
  unsigned long long *d_published = nullptr;
  int32_t coop = 0;  // the device supports cooperative launches

  int64_t launches = 0;
  uint64_t ws_gen = 0;  // bumped whenever a workspace buffer is reallocated
};

// dd_execute_pitched for n plans on one device at once, on `stream`: the
// staged u8 work of plans with the same DM-tile width shares persistent
// launches (no row statistics), the rest runs as dd_execute_pitched would.
// Arguments per plan as for dd_execute_pitched; a timeout of a shared launch
// is recorded in the status word of its first plan.  Queues only.
int execute_plans_pitched(dd_plan *const *plans, int n, const void *const *block,
                          const int64_t *nsamp_in, const int64_t *pitch_elems, void *const *out,
                          const int64_t *out_pitch, void *stream);

namespace ddk {

// Element size of a dd_dtype.namespace ddk {

// Element size of a dd_dtype.
inline int elem_size(int32_t dtype) { return dtype == DD_U8 ? 1 : (dtype == DD_F16 ? 2 : 4); }

// Dedispersion: out[d][t] = sum_c block[c][t + delays[c][d]] for t < nsamp_out.
// Each launcher returns the number of kernels queued, or -1 with the CUDA
// error in *err.
// With tilestats non-null (float plans), also each (row, 256-sample time
// tile)'s partial statistics, as launch_dedisperse_octet.
int launch_dedisperse_direct(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                             void *out, int64_t out_pitch, float4 *tilestats, cudaStream_t stream,
                             cudaError_t *err);
// DM trials per thread of the plain-load kernel for this output length (16,
// or 4 when 16 would leave fewer than two CTAs per SM).
int direct_trials_per_thread(const dd_plan *p, int64_t nsamp_out);
// Staged quad kernel (u8): needs the plan's quad tables, a 16-byte aligned
// block, a pitch that is a multiple of 16 bytes and at most 65535 time tiles.
bool quad_supported(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out);
// With rowsums / tilemax non-null it also adds each row's exact sums
// (rowsums[2d] += sum D, rowsums[2d+1] += sum D^2; the caller zeroes them
// first) and writes the largest output of every (row, kTileSamples-sample
// time tile) to tilemax[d * ntiles + tile].
int launch_dedisperse_quad(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                           void *out, int64_t out_pitch, int64_t *rowsums, int32_t *tilemax,
                           cudaStream_t stream, cudaError_t *err);
// The staged kernel is persistent: one launch drains a queue of (beam, DM
// tile, time tile) items over up to ddq::kMaxBeams beams, which must share
// nd_thr (kNdThr, kNdThr/2 or kNdThr/4) and the staging depth copy_ahead
// (ddq::kMinCopyAhead .. kMaxCopyAhead); smem is the largest of the beams'
// shared-memory sizes at that depth.
ddq::Beam quad_beam(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                    void *out, int64_t out_pitch, int64_t *rowsums, int32_t *tilemax);
int launch_quad_beams(const ddq::Beam *beams, int nbeams, int nd_thr, int copy_ahead, int smem,
                      int device_sms,
                      unsigned long long *next_item, int32_t *status, uint64_t timeout_ns,
                      int32_t skip_copies, cudaStream_t stream, cudaError_t *err);
constexpr int kTileSamples = ddq::kTimeTile;
// Staged octet kernel (f16 / f32): needs the plan's octet tables, a 16-byte
// aligned block and a pitch of a whole number of 16-byte units.
bool octet_supported(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out);
// With tilestats non-null it also writes each (row, 256-sample time tile)'s
// partial statistics {K, sum (D - K), sum (D - K)^2, max D} (K the tile's
// first output) to tilestats[d * ntiles + tile] (octet_tiles(nsamp_out)
// tiles per row), for launch_tiled_detect_f32.
int launch_dedisperse_octet(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                            void *out, int64_t out_pitch, float4 *tilestats, cudaStream_t stream,
                            cudaError_t *err);
constexpr int kOctetTileSamples = ddo::kTimeTile;
inline int64_t octet_tiles(int64_t nsamp_out) {
  return (nsamp_out + kOctetTileSamples - 1) / kOctetTileSamples;
}
// The staged octet kernel is persistent too: one launch drains a queue of
// (beam, DM tile, time tile) items over up to ddo::kMaxBeams beams of one
// input dtype and one nd_thr (kNdThr or kNdThr/2); smem is the largest of
// the beams' shared-memory sizes.
ddo::Beam octet_beam(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out,
                     void *out, int64_t out_pitch, float4 *tilestats);
int launch_octet_beams(const ddo::Beam *beams, int nbeams, int32_t dtype, int nd_thr, int smem,
                       int device_sms, unsigned long long *next_item, int32_t *status,
                       uint64_t timeout_ns, int32_t skip_copies, cudaStream_t stream,
                       cudaError_t *err);
inline int64_t time_tiles(int64_t nsamp_out) { return (nsamp_out + kTileSamples - 1) / kTileSamples; }

// Detection passes over out[ndm][nsamp_out]; see dd_detect in dd.h.
constexpr int kDetectChunk = 4096;  // samples per (row, chunk) work unit
int launch_stats(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma,
                 cudaStream_t stream, cudaError_t *err);
int launch_candidates(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma,
                      dd_candidate *cands, int64_t capacity, cudaStream_t stream,
                      cudaError_t *err);
// Detection from the sums and tile maxima of the staged kernel (int32 rows):
// same statistics, thresholds and candidate list as launch_stats +
// launch_candidates, reading only the tiles that can hold a candidate.
int launch_tiled_detect(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma,
                        dd_candidate *cands, int64_t capacity, cudaStream_t stream,
                        cudaError_t *err);
// launch_tiled_detect for up to kMaxDetectBeams staged 8-bit beams at once,
// in two launches (count, then write with each row's offset summed in place
// and each beam's total stored to *total): the same statistics, thresholds
// and candidate lists.
struct DetectBeam {
  const int32_t *D;  // [ndm][n] outputs
  int64_t n;
  int32_t ntiles, ndm, row_begin;  // row_begin: set by the launcher
  const long long *rowsums;        // [ndm][2]
  const int32_t *tilemax;          // [ndm][ntiles]
  dd_row_stats *stats;             // [ndm]
  int32_t *tilecount;              // [ndm][ntiles]
  int64_t *rowcount;               // [ndm]
  dd_candidate *cands;
  int64_t capacity;
  int64_t *total;
};
constexpr int kMaxDetectBeams = 64;
int launch_tiled_detect_beams(const DetectBeam *beams, int nbeams, float nsigma,
                              cudaStream_t stream, cudaError_t *err);
// The same from the staged float kernel's per-tile partial statistics
// (float rows): each row's mean and rms combine its tiles' partials in a
// fixed order in FP64; candidates as launch_candidates.
int launch_tiled_detect_f32(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma,
                            dd_candidate *cands, int64_t capacity, cudaStream_t stream,
                            cudaError_t *err);

// One-launch dd_run for small float beams that the staged float kernel does
// not take: the plain-load kernel's sums and per-tile partials, the row
// statistics, counts and candidates of launch_tiled_detect_f32, in one
// cooperative launch with a grid barrier and a look-back over the rows'
// published counts (bounded waits).  The results equal those of
// launch_dedisperse_direct + launch_tiled_detect_f32 bit for bit.  The
// kernel writes the candidate total to the plan's pinned h_total[0] (and
// d_total[0]) once every row worker is done; a wait that ran out records the
// plan's status word and leaves h_total[0] as the host set it.
constexpr int64_t kSmallMaxOutputs = int64_t(1) << 22;  // ndm * nsamp_out
bool small_supported(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out);
int launch_run_small(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out, void *out,
                     float nsigma, dd_candidate *cands, int64_t capacity, cudaStream_t stream,
                     cudaError_t *err);

}  // namespace ddk
