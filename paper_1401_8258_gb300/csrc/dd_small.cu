// dd_small.cu -- dd_run in one launch for small float beams (the single-beam
// functional-test shape of Sec. 2.4: 64 wide channels at DM step 1, whose
// delay patterns the staged float kernel's tables do not take).
//
// For such a beam the work is a few microseconds and the cost of dd_run is
// its launches and host round trips.  Here the whole path -- dedispersion
// (Sec. 2.1.1), per-DM normalisation (Sec. 3.5) and n-sigma candidate
// extraction (Sec. 3.6) -- is one cooperative launch in three phases:
//   1. every CTA takes (time tile, DM group) items: the plain-load kernel's
//      channel sums (with 4 trials per thread on aligned rows from input
//      windows staged in shared memory, staged_sums; else direct_sums) and
//      its tile's partial statistics (tile_partials), then arrives at the
//      grid barrier;
//   2. the first min(grid, ndm) CTAs (the row workers) wait at the barrier
//      and take rows d: the row's mean, rms and threshold (row_stats_f32)
//      and its per-tile candidate counts (count_row_tiles), then publish
//      the row's count (the other CTAs are done).  When every worker has
//      one row that fits, the row's outputs and tile partials are copied into
//      shared memory (the partials in their own copy group, so the
//      statistics start while the row lands), phases 2 and 3 read them from
//      there, and the snr divisions of the row's first candidate tile are
//      issued before the look-back, whose wait hides their latency;
//   3. each row worker sums the earlier rows' published counts (a decoupled
//      look-back in place of a second grid barrier) and writes its row's
//      candidates at that position (write_row_tiles); the CTA of the
//      last row stores the total in device memory, and the last row worker
//      to finish copies it to the plan's pinned host word, which the host
//      polls (so dd_run returns without waiting for the launch to retire).
// The arithmetic is that of launch_dedisperse_direct followed by
// launch_tiled_detect_f32 (the same device functions), so outputs,
// statistics and candidates equal that path's bit for bit.
//
// The grid barrier: a 64-bit arrivals counter that only grows; launch k
// waits for base_k + grid arrivals, base_k being the arrivals of all earlier
// launches (kept by the host); the row counts are published tagged with
// epoch base_k + 1.  Every wait is bounded (globaltimer): a CTA whose wait
// runs out records the status word and returns, the CTAs waiting on it then
// run out too, the total is never stored, and the host resets the counter
// and the published counts.  With the plan's fault injection on, the barrier
// waits for one arrival more than the grid makes, so its waits run out.  The
// data other CTAs wrote before the barrier are read through L2
// (ld.global.cg).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "dd_detect_dev.cuh"
#include "dd_device.cuh"
#include "dd_direct_dev.cuh"
#include "dd_internal.h"

namespace {

static_assert(kDirectThreads == kTileThreads, "one CTA shape for all three phases");
static_assert(kDirectThreads == ddk::kOctetTileSamples, "a time tile is a statistics tile");

struct SmallArgs {
  const void *in;
  int64_t pitch;
  const int32_t *delays;
  int32_t nchan, ndm;
  int64_t nsamp_out;
  int32_t maxshift;        // nsamp_in = nsamp_out + maxshift
  int32_t aligned;         // rows start on 16-byte boundaries (staged windows)
  float *out;              // [ndm][nsamp_out]
  float4 *tilestats;       // [ndm][ntiles]
  dd_row_stats *stats;     // [ndm]
  int32_t *tilecount;      // [ndm][ntiles]
  int64_t *rowcount;       // [ndm]
  dd_candidate *cands;
  int64_t capacity;
  double thr;
  int64_t *total;          // device [1]
  int64_t *host_total;     // pinned host word, device-mapped
  int32_t *status;         // sticky status word
  unsigned long long *arrivals;
  unsigned long long base;  // arrivals of earlier launches
  unsigned long long *published;  // [ndm] epoch << 24 | row count (epoch = base + 1)
  uint64_t timeout_ns;
  int32_t ntiles, ngroups, nworkers;
  int32_t extra_wait;  // fault injection: the barrier waits for this many arrivals more
  int32_t row_smem;    // one row per worker, copied to shared memory for phases 2 and 3
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Arrive (thread 0, after the CTA's writes: the barrier orders them before
// its release) without waiting.
__device__ __forceinline__ void grid_arrive(unsigned long long *arrivals) {
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(arrivals) : "memory");
}

// Wait until the counter reaches `target` (thread 0 polls with acquire
// loads, bounded; the CTA barrier then orders the other threads' reads after
// it); false if the wait ran out (the status word is then set).  Whole CTA.
__device__ __forceinline__ bool grid_wait(const SmallArgs &a, unsigned long long target) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_acquire(a.arrivals) < target) {
      const uint64_t t0 = dddev::global_timer();
      while (ld_acquire(a.arrivals) < target) {
        if (dddev::global_timer() - t0 > a.timeout_ns) {
          atomicExch(a.status, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Row d's candidate count, published for this launch (thread 0, once the
// count is final): tagged with the launch's epoch, base + 1 (a count fits
// 24 bits: rows have at most kSmallMaxOutputs samples).
__device__ __forceinline__ void publish_count(const SmallArgs &a, int d, int64_t count) {
  const unsigned long long word = ((a.base + 1) << 24) | static_cast<unsigned long long>(count);
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(a.published + d), "l"(word) : "memory");
}

// Sum of the counts of rows 0 .. d-1 as published in this launch (decoupled
// look-back: each thread polls some rows with acquire loads until their
// words carry this launch's epoch, bounded); false if a wait ran out (the
// status word is then set).  Whole CTA; every thread gets the sum.
__device__ __forceinline__ bool rows_before_published(const SmallArgs &a, int d, int64_t *before) {
  __shared__ long long s_part[kDirectThreads / 32];
  __shared__ int s_fail;
  const unsigned long long epoch = (a.base + 1) & ((1ull << 40) - 1);
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  long long sum = 0;
  bool ok = true;
  for (int r = threadIdx.x; r < d && ok; r += kDirectThreads) {
    unsigned long long v = ld_acquire(a.published + r);
    if ((v >> 24) != epoch) {
      const uint64_t t0 = dddev::global_timer();
      while (((v = ld_acquire(a.published + r)) >> 24) != epoch) {
        if (dddev::global_timer() - t0 > a.timeout_ns) {
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    if (ok) sum += static_cast<long long>(v & 0xffffffull);
  }
  if (!ok) {
    s_fail = 1;
    atomicExch(a.status, 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = sum;
  __syncthreads();
  long long total = 0;
#pragma unroll
  for (int w = 0; w < kDirectThreads / 32; ++w) total += s_part[w];
  *before = total;
  const bool failed = s_fail != 0;
  __syncthreads();  // s_part / s_fail free for a later call
  return !failed;
}

// Phase 1 of the 4-trial variant on 16-byte aligned rows, with the input
// staged in shared memory: per delay stage of kDelayChans channels,
// the delays of the item's trials and each channel's smallest one (wmin);
// then sub-stages of nsub channels, each channel's window -- kWin4 samples
// from t0 + wmin rounded down to a 16-byte unit (t0 the tile's first
// output) -- copied with cp.async (16-byte units, all in flight at once;
// units past the row's last needed unit are zero-filled), after which the
// sums read the windows through a per-channel table of the trials' offsets:
// the same values added in the same channel order as direct_sums, so the
// same results.  A stage in which some channel's delays over the trials
// spread too far for a window, or rows that are not 16-byte aligned, are
// summed from global memory instead (direct_sums' loop).  The windows are
// 384 samples long, in sub-stages that fill 48 KB (32 f32 or 64 f16
// channels).  (The offsets are kept in groups of four trials, so the code
// takes any multiple of four.)

// Tile lists of phases 2 and 3 (rounds of this many tiles; small, to keep
// the kernel's static shared memory low).
constexpr int kRowList = 64, kL2List = 256;
constexpr int kWin4 = 384;  // samples per channel window, 4-trial variant
constexpr int kDyn4 = 48 * 1024;  // its window bytes (32 f32 / 64 f16 channels)

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Loads of phases 2 and 3 when the row lives in shared memory: the row's
// outputs, partials and counts are read from their shared copies (plain
// loads), the other rows' counts through L2.
struct RowLd {
  __device__ __forceinline__ float operator()(const float *p) const { return *p; }
  __device__ __forceinline__ float4 operator()(const float4 *p) const { return *p; }
  __device__ __forceinline__ int32_t operator()(const int32_t *p) const { return *p; }
  __device__ __forceinline__ int64_t operator()(const int64_t *p) const {
    return static_cast<int64_t>(__ldcg(reinterpret_cast<const long long *>(p)));
  }
};

template <typename T, int NDMS>
__device__ __forceinline__ void staged_sums(const SmallArgs &a, int d0, int64_t t0, bool live,
                                            float (&acc)[NDMS], T *s_win) {
  static_assert(NDMS % 4 == 0, "offsets in groups of four trials");
  constexpr int kQ = NDMS / 4;
  constexpr int kUnit = 16 / static_cast<int>(sizeof(T));  // samples per 16-byte unit
  __shared__ int32_t s_dl[kDelayChans][NDMS];
  __shared__ int32_t s_wmin[kDelayChans];
  __shared__ int4 s_off[kDelayChans][kQ];  // per channel: window offsets of the trials, less tid
  __shared__ int s_spread_ok;
  const T *in = static_cast<const T *>(a.in);
  const int64_t nsamp_in = a.nsamp_out + a.maxshift;
  // window geometry (compile-time, so that the copy loop's index
  // arithmetic is shifts and multiplies)
  constexpr int stride = kWin4, nsub = kDyn4 / (kWin4 * static_cast<int>(sizeof(T)));
  constexpr int units = stride / kUnit;
  static_assert(stride % kUnit == 0 && kDelayChans % nsub == 0, "window tiling");
  // the row's units that hold needed samples (within the row: the pitch is a
  // whole number of units, at least nsamp_in)
  const int64_t row_units = (nsamp_in + kUnit - 1) / kUnit;
  const int tid = threadIdx.x;
#pragma unroll
  for (int j = 0; j < NDMS; ++j) acc[j] = 0.f;
  for (int c0 = 0; c0 < a.nchan; c0 += kDelayChans) {
    const int nc = a.nchan - c0 < kDelayChans ? a.nchan - c0 : kDelayChans;
    __syncthreads();  // s_dl / s_wmin / s_win free from the previous stage
    if (tid == 0) s_spread_ok = a.aligned;
    // trials past ndm take the last trial's delays (in range; never stored)
    for (int i = tid; i < kDelayChans * NDMS; i += kDirectThreads) {
      const int cc = i / NDMS, j = i % NDMS;
      const int d = d0 + j < a.ndm ? d0 + j : a.ndm - 1;
      s_dl[cc][j] = cc < nc ? a.delays[static_cast<int64_t>(c0 + cc) * a.ndm + d] : 0;
    }
    __syncthreads();
    if (tid < kDelayChans) {
      int lo = s_dl[tid][0], hi = lo;
#pragma unroll
      for (int j = 1; j < NDMS; ++j) lo = min(lo, s_dl[tid][j]), hi = max(hi, s_dl[tid][j]);
      const int start = static_cast<int>((t0 + lo) % kUnit);  // offset inside the first unit
      s_wmin[tid] = lo;
      if (tid < nc && start + kDirectThreads - 1 + (hi - lo) >= stride) s_spread_ok = 0;
      // channel tid's window starts at sample (t0 + lo) rounded down to a unit:
      // output t0 + i of trial j reads element i + start + (delay_j - lo) of it
      const int base = (tid % nsub) * stride + start - lo;
#pragma unroll
      for (int q = 0; q < kQ; ++q)
        s_off[tid][q] = make_int4(base + s_dl[tid][4 * q], base + s_dl[tid][4 * q + 1],
                                  base + s_dl[tid][4 * q + 2], base + s_dl[tid][4 * q + 3]);
    }
    __syncthreads();
    if (!s_spread_ok) {  // uniform: this stage from global memory
      if (!live) continue;
      const T *base = in + static_cast<int64_t>(c0) * a.pitch + t0 + tid;
      for (int cc = 0; cc < nc; ++cc) {
        const T *row = base + static_cast<int64_t>(cc) * a.pitch;
#pragma unroll
        for (int j = 0; j < NDMS; ++j) acc[j] += DirectTraits<T>::load(row + s_dl[cc][j]);
      }
      continue;
    }
    const uint32_t win0 = dddev::smem_addr(s_win);
    for (int s0 = 0; s0 < nc; s0 += nsub) {
      const int ns = nc - s0 < nsub ? nc - s0 : nsub;
      if (s0 > 0) __syncthreads();  // every thread is past the previous sub-stage's sums
      for (int i = tid; i < ns * units; i += kDirectThreads) {
        const int cc = i / units, u = i % units;
        const int64_t unit = (t0 + s_wmin[s0 + cc]) / kUnit + u;
        const T *row = in + static_cast<int64_t>(c0 + s0 + cc) * a.pitch;
        const bool ok = unit < row_units;
        cp_async16(win0 + static_cast<uint32_t>((cc * stride + u * kUnit) * sizeof(T)),
                   ok ? row + unit * kUnit : row, ok ? 16u : 0u);
      }
      cp_async_wait_all();
      __syncthreads();
      if (live) {
        const T *wt = s_win + tid;
#pragma unroll 4
        for (int cc = 0; cc < ns; ++cc) {
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const int4 o = s_off[s0 + cc][q];
            acc[4 * q] += DirectTraits<T>::load_shared(wt + o.x);
            acc[4 * q + 1] += DirectTraits<T>::load_shared(wt + o.y);
            acc[4 * q + 2] += DirectTraits<T>::load_shared(wt + o.z);
            acc[4 * q + 3] += DirectTraits<T>::load_shared(wt + o.w);
          }
        }
      }
    }
  }
}

// Three CTAs per SM: 448 items (the 64 x 8192 single beam) run co-resident.
template <typename T, int NDMS>
__global__ void __launch_bounds__(kDirectThreads, 3)
dd_run_small(const __grid_constant__ SmallArgs a) {
  __shared__ PartialScratch<NDMS> s_part;
  extern __shared__ __align__(16) unsigned char s_dyn[];  // NDMS 4: windows, then a row
  const int64_t n = a.nsamp_out;
  const int ntiles = a.ntiles;
  // 1/n for the row statistics, its FP64 division under phase 1
  const double rn = __drcp_rn(static_cast<double>(n));

  // phase 1: sums and tile partials
  const int64_t nitems = static_cast<int64_t>(ntiles) * a.ngroups;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = static_cast<int>(item % ntiles);
    const int d0 = static_cast<int>(item / ntiles) * NDMS;
    const int64_t t = static_cast<int64_t>(tile) * kDirectThreads + threadIdx.x;
    const bool live = t < n;
    float acc[NDMS];
    if constexpr (NDMS <= 8) {
      staged_sums<T, NDMS>(a, d0, static_cast<int64_t>(tile) * kDirectThreads, live, acc,
                           reinterpret_cast<T *>(s_dyn));
    } else {
      __shared__ int32_t s_delay[kDelayChans][NDMS];
      direct_sums<T, NDMS>(static_cast<const T *>(a.in), a.pitch, a.delays, a.nchan, a.ndm, d0,
                           t, live, acc, s_delay);
    }
    if (live) {
#pragma unroll
      for (int j = 0; j < NDMS; ++j)
        if (d0 + j < a.ndm) a.out[static_cast<int64_t>(d0 + j) * n + t] = acc[j];
    }
    tile_partials<NDMS>(acc, live, d0, a.ndm, ntiles, tile, a.tilestats, s_part);
  }
  grid_arrive(a.arrivals);
  if (static_cast<int>(blockIdx.x) >= a.nworkers) return;
  if (!grid_wait(a, a.base + gridDim.x + a.extra_wait)) return;

  if (a.row_smem) {
    // one row per worker (d = blockIdx.x), kept in shared memory from here on
    const int d = blockIdx.x;
    float4 *s_ts = reinterpret_cast<float4 *>(s_dyn);          // the row's tile partials
    int32_t *s_tc = reinterpret_cast<int32_t *>(s_ts + ntiles);  // its per-tile counts
    float *s_row = reinterpret_cast<float *>(s_ts + ntiles + (ntiles + 3) / 4);  // its outputs
    const float4 *ts = a.tilestats + static_cast<int64_t>(d) * ntiles;
    // the tile partials first (one commit group), then the row in 16-byte
    // units from its start rounded down to a unit (a second group, landing
    // while the statistics are computed); the copy of the last unit stops
    // at the end of the last row
    for (int i = threadIdx.x; i < ntiles; i += kDirectThreads)
      cp_async16(dddev::smem_addr(s_ts + i), ts + i, 16u);
    cp_async_commit();
    const int64_t first = static_cast<int64_t>(d) * n;  // the row's first element
    const int64_t ufirst = first / 4, uend = (first + n + 3) / 4, all = static_cast<int64_t>(a.ndm) * n;
    for (int64_t u = ufirst + threadIdx.x; u < uend; u += kDirectThreads) {
      const int64_t rest = all - 4 * u;  // elements from this unit to the end of the last row
      cp_async16(dddev::smem_addr(s_row + 4 * (u - ufirst)), a.out + 4 * u,
                 static_cast<uint32_t>(rest < 4 ? 4 * rest : 16));
    }
    cp_async_commit();
    cp_async_wait_group<1>();
    __syncthreads();
    // phase 2: the row's statistics and per-tile counts
    const RowLd rl;
    const dd_row_stats st = row_stats_f32<kDirectThreads>(s_ts, n, ntiles, a.thr, rn, rl);
    cp_async_wait_group<0>();
    __syncthreads();
    s_row += first % 4;  // the row's element 0
    if (threadIdx.x == 0) a.stats[d] = st;
    const auto reaches = [&](int tt) { return s_ts[tt].w >= st.fthr; };
    count_row_tiles<float, kDirectThreads, decltype(reaches), RowLd, kRowList>(
        s_row, n, ntiles, st, reaches, s_tc, a.rowcount + d, rl);
    // publish the row's count (thread 0 wrote it)
    if (threadIdx.x == 0) publish_count(a, d, a.rowcount[d]);
    // the snr of this thread's candidate in the row's first tile with any:
    // its FP64 division runs while the CTA waits for the earlier rows' counts
    __syncthreads();  // s_tc complete
    int pre_tile = -1;
    float pre_snr = 0.f;
    for (int k0 = 0; k0 < ntiles && pre_tile < 0; k0 += 32) {
      const int kl = k0 + (threadIdx.x & 31);
      const unsigned any = __ballot_sync(0xffffffffu, kl < ntiles && s_tc[kl] != 0);
      if (any) pre_tile = k0 + __ffs(any) - 1;
    }
    if (pre_tile >= 0) {
      const int64_t t = static_cast<int64_t>(pre_tile) * kDirectThreads + threadIdx.x;
      if (t < n && is_candidate(s_row[t], st))
        pre_snr = static_cast<float>(snr_of(static_cast<double>(s_row[t]), st.mean, st.sigma));
    }
    // phase 3: the row's candidates, after the earlier rows' counts
    int64_t before = 0;
    if (!rows_before_published(a, d, &before)) return;
    const int64_t mine = a.rowcount[d];  // this CTA's write
    if (d == a.ndm - 1 && threadIdx.x == 0) *a.total = before + mine;
    if (mine > 0 && before < a.capacity)  // uniform across the CTA
      write_row_tiles<float, kDirectThreads, RowLd, kRowList>(s_row, n, ntiles, st, s_tc, before,
                                                             d, a.cands, a.capacity, rl,
                                                             pre_tile, &pre_snr);
  } else {
    // phase 2: row statistics and per-tile counts
    const L2Ld ld;
    for (int d = blockIdx.x; d < a.ndm; d += a.nworkers) {
      const float4 *ts = a.tilestats + static_cast<int64_t>(d) * ntiles;
      const dd_row_stats st = row_stats_f32<kDirectThreads>(ts, n, ntiles, a.thr, rn, ld);
      if (threadIdx.x == 0) a.stats[d] = st;
      const auto reaches = [&](int tt) { return ld(ts + tt).w >= st.fthr; };
      count_row_tiles<float, kDirectThreads, decltype(reaches), L2Ld, kL2List>(
          a.out + static_cast<int64_t>(d) * n, n, ntiles, st, reaches,
          a.tilecount + static_cast<int64_t>(d) * ntiles, a.rowcount + d, ld);
      if (threadIdx.x == 0) publish_count(a, d, a.rowcount[d]);  // thread 0 wrote it
    }

    // phase 3: candidates, rows in order, each after the earlier rows' counts
    for (int d = blockIdx.x; d < a.ndm; d += a.nworkers) {
      int64_t before = 0;
      if (!rows_before_published(a, d, &before)) return;
      const int64_t mine = ld(a.rowcount + d);
      if (d == a.ndm - 1 && threadIdx.x == 0) *a.total = before + mine;
      if (mine == 0 || before >= a.capacity) continue;  // uniform across the CTA
      // stats[d] and the tile counts were written by this CTA in phase 2
      const dd_row_stats st = a.stats[d];
      write_row_tiles<float, kDirectThreads, L2Ld, kL2List>(
          a.out + static_cast<int64_t>(d) * n, n, ntiles, st,
          a.tilecount + static_cast<int64_t>(d) * ntiles, before, d, a.cands, a.capacity, ld);
    }
  }
  // the last row worker to get here stores the total on the host: every
  // output, statistic and candidate has been written by then
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long before = atomicAdd(a.arrivals, 1ull);
    if (before == a.base + gridDim.x + a.nworkers - 1) {
      __threadfence();
      const long long total = __ldcg(reinterpret_cast<const long long *>(a.total));
      *reinterpret_cast<volatile long long *>(a.host_total) = total;
      __threadfence_system();
    }
  }
}

using SmallKernel = void (*)(SmallArgs);

// Kernel variant for (input dtype, trials per thread: 4 or 16).
SmallKernel small_kernel(int32_t dtype, int ndms) {
  if (dtype == DD_F16) return ndms == 16 ? dd_run_small<uint16_t, 16> : dd_run_small<uint16_t, 4>;
  return ndms == 16 ? dd_run_small<float, 16> : dd_run_small<float, 4>;
}

// Dynamic shared memory: the 4-trial variant stages its windows in kDyn4
// bytes, then a row (outputs, tile partials and counts) in phases 2 and 3;
// the 16-trial one none.
static_assert(kDelayChans * kWin4 * 2 <= kDyn4 && 32 * kWin4 * 4 <= kDyn4, "4-trial windows");

// Co-resident CTAs per SM of each variant (queried once per process; every
// device of the process is a GB300, the one target of this library).
int resident_per_sm(int32_t dtype, int ndms) {
  static std::once_flag once;
  static int n[2][2] = {{0, 0}, {0, 0}};
  std::call_once(once, [] {
    for (int f = 0; f < 2; ++f)
      for (int w = 0; w < 2; ++w) {
        const void *k = reinterpret_cast<const void *>(small_kernel(f ? DD_F16 : DD_F32, w ? 16 : 4));
        const int dyn = w ? 0 : kDyn4;
        int b = 0;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kDirectThreads, dyn) != cudaSuccess)
          b = 0;
        n[f][w] = b;
      }
    cudaGetLastError();
  });
  return n[dtype == DD_F16 ? 1 : 0][ndms == 16 ? 1 : 0];
}

struct SmallShape {
  int ndms;          // trials per thread
  int dyn;           // dynamic shared memory per CTA
  int64_t resident;  // co-resident CTAs on the device
};

// 16 trials per thread when that already gives two CTAs per SM (as the
// plain-load kernel), else 4 with staged windows.
SmallShape small_shape(const dd_plan *p, int64_t nsamp_out) {
  const int ndms = ddk::direct_trials_per_thread(p, nsamp_out);
  const int64_t resident = static_cast<int64_t>(resident_per_sm(p->dtype, ndms)) * p->sm_count;
  return {ndms, ndms == 16 ? 0 : kDyn4, resident};
}

}  // namespace

namespace ddk {

bool small_supported(const dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out) {
  if (p->dtype == DD_U8 || p->path != 0 || !p->coop || !p->d_arrivals) return false;
  if (static_cast<int64_t>(p->ndm) * nsamp_out > kSmallMaxOutputs) return false;
  if (octet_supported(p, block, pitch, nsamp_out)) return false;
  return small_shape(p, nsamp_out).resident > 0;
}

int launch_run_small(dd_plan *p, const void *block, int64_t pitch, int64_t nsamp_out, void *out,
                     float nsigma, dd_candidate *cands, int64_t capacity, cudaStream_t stream,
                     cudaError_t *err) {
  const SmallShape sh = small_shape(p, nsamp_out);
  const int ndms = sh.ndms;
  const int64_t ntiles = (nsamp_out + kDirectThreads - 1) / kDirectThreads;
  const int ngroups = (p->ndm + ndms - 1) / ndms;
  const int64_t nitems = ntiles * ngroups;
  const int grid = static_cast<int>(nitems < sh.resident ? nitems : sh.resident);
  SmallArgs a;
  a.in = block;
  a.pitch = pitch;
  a.delays = p->d_delays;
  a.nchan = p->nchan;
  a.ndm = p->ndm;
  a.nsamp_out = nsamp_out;
  a.maxshift = p->maxshift;
  a.aligned = (reinterpret_cast<uintptr_t>(block) % 16 == 0 &&
               (pitch * ddk::elem_size(p->dtype)) % 16 == 0) ? 1 : 0;
  a.out = static_cast<float *>(out);
  a.tilestats = p->d_tilestats;
  a.stats = p->d_stats;
  a.tilecount = p->d_tilecount;
  a.rowcount = p->d_rowcount;
  a.cands = cands;
  a.capacity = capacity;
  a.thr = static_cast<double>(nsigma);
  a.total = p->d_total;
  a.host_total = p->h_total_dev;
  a.status = p->d_error;
  a.arrivals = p->d_arrivals;
  a.base = p->arrivals_base;
  a.published = p->d_published;
  a.timeout_ns = p->wait_timeout_ns;
  a.ntiles = static_cast<int32_t>(ntiles);
  a.ngroups = ngroups;
  a.nworkers = grid < p->ndm ? grid : p->ndm;
  a.extra_wait = p->debug_skip_copies ? 1 : 0;
  // shared row layout: ntiles partials (16 B), the counts rounded up to
  // 16 B, then the row in 16-byte units (up to 3 elements before it, 3 after)
  a.row_smem = (a.nworkers == p->ndm && reinterpret_cast<uintptr_t>(out) % 16 == 0 &&
                ntiles * static_cast<int64_t>(sizeof(float4)) + (ntiles + 3) / 4 * 16 +
                        (nsamp_out + 6) * 4 <= sh.dyn)
                   ? 1 : 0;
  void *args[] = {&a};
  *err = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(small_kernel(p->dtype, ndms)),
                                     dim3(grid), dim3(kDirectThreads), args, sh.dyn, stream);
  if (*err != cudaSuccess) return -1;
  p->arrivals_base += static_cast<uint64_t>(grid) + static_cast<uint64_t>(a.nworkers);
  return 1;
}

}  // namespace ddk
