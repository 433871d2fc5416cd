/*
 * dd.h -- C ABI of libdd: brute-force incoherent dedispersion of a
 * channelised filterbank block, per-DM-trial normalisation and n-sigma
 * candidate extraction on one NVIDIA GB300 (sm_103a).
 *
 * Method (A. Magro, "A Real-Time, GPU-Based, Non-Imaging Back-End for Radio
 * Telescopes", 2013):
 *   D[d][t] = sum_{c=0}^{nchan-1} I[c][t + delay(c,d)]        (Sec. 2.1.1, brute-force equation)
 *   delay(c,d) = round(DM_d * dT(c)),
 *   dT(c) = K * ((f_top - c*df)^-2 - f_top^-2) / t_samp       (Sec. 2.1.1, deltaT equation)
 *   K = 4.148808e3 MHz^2 pc^-1 cm^3 s                          (Sec. 1.2.1, dispersion constant)
 *   valid output length nsamp_out = nsamp_in - maxshift        (Sec. 3.4, maxshift overlap)
 *   per-DM mean and rms, snr = (D - mean)/rms                  (Sec. 3.5, normalisation)
 *   candidates = (DM, time, intensity) with snr > nsigma       (Sec. 3.6, thresholding)
 *
 * Conventions fixed by this library where the text is silent:
 *   - channel c has centre frequency f_top - c*df (df > 0), so channel 0 is
 *     the band top and has delay 0;
 *   - round() is round half away from zero; dT(c) and DM_d*dT(c) are formed
 *     in IEEE double, left to right, with no fused multiply-add;
 *   - rms is the population standard deviation (1/N) about the mean of the
 *     row, no detrending; the threshold is strict (snr > nsigma); rows with
 *     rms == 0 yield no candidates; candidates are ordered by (dm_idx, t).
 *
 * Layouts:
 *   block  [nchan][pitch] elements, time fastest (channel 0 = band top);
 *          elements u8 (DD_U8), IEEE binary16 bits (DD_F16) or f32 (DD_F32).
 *   out    [ndm][nsamp_out], dense rows; int32 for DD_U8 input (exact sums),
 *          f32 for DD_F16 / DD_F32 input (f32 accumulation).
 *   delays [nchan][ndm] int32 (channel-major: one channel's DM trials are
 *          contiguous).
 *
 * Errors: every entry point returns DD_OK (0) or a negative dd_status; none
 * throws, aborts or exits.  Argument errors are detected synchronously before
 * anything is queued.  Device-side faults caught by the kernels themselves
 * (bounded waits that ran out) are recorded in the plan and reported by the
 * next synchronising call (dd_detect, dd_sync, dd_process_host).
 *
 * Threads and streams: a plan may be used by one host thread at a time; work
 * queued with one plan on different streams must not overlap in time
 * (the plan's workspace is shared).  Use one plan per concurrent beam.
 */
#ifndef DD_H
#define DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { DD_U8 = 0, DD_F16 = 1, DD_F32 = 2 } dd_dtype;

typedef enum {
  DD_OK = 0,
  DD_ERR_ARG = -1,            /* invalid argument (null pointer, bad geometry, non-finite DM) */
  DD_ERR_SIZE = -2,           /* size out of range (nsamp_in <= maxshift, pitch < nsamp_in, ...) */
  DD_ERR_DTYPE = -3,          /* unknown input dtype */
  DD_ERR_CUDA = -4,           /* a CUDA runtime call failed */
  DD_ERR_OOM = -5,            /* device or host allocation failed */
  DD_ERR_OVERFLOW = -6,       /* more candidates than capacity; the first capacity are written */
  DD_ERR_DEVICE_TIMEOUT = -7, /* a bounded device wait ran out; results of that launch are invalid */
  DD_ERR_RANGE = -8           /* a delay does not fit in int32, or a sum may overflow int32 */
} dd_status;

/* One detection: DM trial index, output sample (arrival sample at f_top,
 * relative to the block), dedispersed value D[dm_idx][t] and its snr. */
typedef struct {
  int32_t dm_idx;
  int32_t t;
  float value;
  float snr;
} dd_candidate;

typedef struct dd_plan dd_plan; /* opaque; owns the device delay table and workspace */

/* Host-only delay table, Sec. 2.1.1 deltaT equation, with the conventions
 * above.  delays_out: host int32 [nchan][ndm] (caller-owned); maxshift_out:
 * largest delay.  Needs no GPU.  DD_ERR_ARG for nchan < 1, ndm < 1, df <= 0,
 * t_samp <= 0, a band whose bottom channel frequency is <= 0, or a DM that is
 * negative or not finite; DD_ERR_RANGE if a delay exceeds INT32_MAX. */
int dd_compute_delays(int32_t nchan, double f_top_mhz, double chan_width_mhz,
                      double t_samp_s, const double *dm_list, int32_t ndm,
                      int32_t *delays_out, int32_t *maxshift_out);

/* Create a plan on CUDA device `device` for blocks of `nchan` channels of
 * in_dtype samples and the DM trials dm_list[0..ndm) (host array, copied).
 * Computes the delay table (dd_compute_delays) and uploads it once
 * (Sec. 3.4: delays are computed once at start-up and stored channel/DM
 * order).  *out receives the plan, or NULL on error. */
int dd_plan_create(dd_plan **out, int32_t nchan, double f_top_mhz, double chan_width_mhz,
                   double t_samp_s, const double *dm_list, int32_t ndm, int32_t in_dtype,
                   int32_t device);

/* Free the plan and all device memory it owns.  NULL-safe.  Synchronises the
 * plan's device first. */
int dd_plan_destroy(dd_plan *p);

/* A plan of the same geometry as `src` (channels, band, sampling, DM list,
 * input dtype, device, kernel path and tile width) that shares src's
 * plan-time tables -- the delay table and the staged kernels' records and
 * windows, read only -- instead of building and storing its own; its
 * workspaces, statistics and status word are its own, so the two plans may
 * be run independently (each on one stream at a time), in the same batch or
 * stream wave.  For the identical beams of a multi-beam receiver (the
 * thesis's back-end dedisperses several beams of one geometry per GPU,
 * Sec. 3.4).  Shared tables are freed with the last plan that holds them;
 * retuning a plan (dd_plan_autotune) gives it tables of its own.  Returns
 * DD_ERR_ARG for a NULL argument, DD_ERR_OOM / DD_ERR_CUDA on failure. */
int dd_plan_create_like(dd_plan **out, const dd_plan *src);

/* A plan for an explicit delay table instead of the dispersion law: host
 * int32 delays[nchan][ndm] (channel-major, copied), every entry in
 * 0 .. 2^30; out[d][t] = sum_c block[c][t + delays[c][d]] with the same
 * kernels, layouts and detection as dd_plan_create.  The thesis's two-step
 * approximations (subband and tree dedispersion, Sec. 2.1) are brute-force
 * sums over such tables.  DD_ERR_ARG for a null table or a negative or
 * larger entry. */
int dd_plan_create_from_delays(dd_plan **out, int32_t nchan, int32_t ndm, const int32_t *delays,
                               int32_t in_dtype, int32_t device);

/* Largest delay of the plan (maxshift, Sec. 3.4). */
int dd_plan_max_delay(const dd_plan *p, int32_t *maxshift);

/* Valid output length nsamp_in - maxshift (Sec. 3.4); DD_ERR_SIZE if
 * nsamp_in <= maxshift. */
int dd_plan_nsamp_out(const dd_plan *p, int64_t nsamp_in, int64_t *nsamp_out);

/* Copy the plan's delay table to host_out, int32 [nchan][ndm]. */
int dd_plan_delays(const dd_plan *p, int32_t *host_out);

/* Dedisperse one block (Sec. 2.1.1) on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).
 *   block: device pointer, [nchan][pitch_elems] elements of the plan's dtype,
 *          of which the first nsamp_in of each row are read;
 *   out:   device pointer, [ndm][nsamp_out] with nsamp_out = nsamp_in - maxshift,
 *          int32 (DD_U8) or float (DD_F16, DD_F32); every element is written.
 * Asynchronous: returns once the kernel is queued.  Caller owns block and out
 * and must keep them alive until the stream reaches this work.  For DD_U8,
 * DD_ERR_RANGE if nchan * 255 could overflow int32.  Any 16-byte-aligned
 * block with a pitch of a whole number of 16-byte units takes the staged
 * (bulk-copy) kernel; other layouts take a plain-load kernel with identical
 * results. */
int dd_execute(dd_plan *p, const void *block, int64_t nsamp_in, int64_t pitch_elems,
               void *out, void *stream);

/* dd_execute with output rows `out_pitch` elements apart (out_pitch >=
 * nsamp_out; DD_ERR_ARG otherwise): row d starts at out + d * out_pitch, and
 * only its first nsamp_out elements are written.  Lets a caller place the
 * rows of several plans into one interleaved array (the subband variant,
 * dd_subband.h, does this). */
int dd_execute_pitched(dd_plan *p, const void *block, int64_t nsamp_in, int64_t pitch_elems,
                       void *out, int64_t out_pitch, void *stream);

/* Normalise and threshold a dedispersed block (Sec. 3.5, 3.6) on `stream`.
 *   out:   device pointer to [ndm][nsamp_out] as written by dd_execute;
 *   cands: device pointer to `capacity` dd_candidate slots (may be NULL when
 *          capacity == 0); filled in (dm_idx, t) order;
 *   count: host pointer; receives the total number of candidates found, even
 *          if it exceeds capacity.
 * Per-DM mean and rms: for DD_U8 plans from exact integer sums S1, S2 and
 * the finaliser mean = S1/N, rms = sqrt((double)(N*S2 - S1^2))/N (128-bit
 * exact numerator, round-to-nearest conversion); for float plans from double
 * sums about a per-row shift.  snr = ((double)D - mean)/rms in IEEE double.
 * Synchronises `stream` once (to return *count).  Returns DD_ERR_OVERFLOW if
 * *count > capacity (the first `capacity` candidates are still written), or
 * DD_ERR_DEVICE_TIMEOUT if an earlier launch on this plan reported one. */
int dd_detect(dd_plan *p, const void *out, int64_t nsamp_out, float nsigma, dd_candidate *cands,
              int64_t capacity, int64_t *count, void *stream);

/* The whole path on device buffers in one call: dd_execute(block -> out)
 * followed by dd_detect(out) (Sec. 2.1.1, 3.5, 3.6), with the same results --
 * every element of out, the same candidates in (dm_idx, t) order, the same
 * per-DM mean and rms (dd_get_stats), *count and status codes as those two
 * calls.  Arguments as for dd_execute and dd_detect; `event` is an optional
 * cudaEvent_t (NULL = none) recorded on `stream` right after the
 * dedispersion kernel, for timing the phases.  When the staged kernel runs,
 * it also accumulates each DM row's exact integer sums and the largest value
 * of each 512-sample time tile as it writes out, so the detection reads out
 * only in the tiles that can hold a candidate instead of twice in full; the
 * float kernels keep per-tile partial statistics the same way.  Synchronises
 * `stream` once -- except for small float beams that the staged float kernel
 * does not take, whose whole path runs as one cooperative launch: dd_run
 * then returns as soon as that launch has stored the count in host memory,
 * when every output, statistic and candidate is written, without waiting
 * for the launch to retire (later work on `stream` is ordered after it). */
int dd_run(dd_plan *p, const void *block, int64_t nsamp_in, int64_t pitch_elems, void *out,
           float nsigma, dd_candidate *cands, int64_t capacity, int64_t *count, void *stream,
           void *event);

/* Batches: several beams, each with its own plan (geometry, DM list, dtype),
 * processed together.  The thesis runs one beam per GPU kernel (Sec. 2.4) and
 * several beams per GPU (Sec. 3.4, Ch. 6); here the staged u8 kernel is
 * persistent, so one launch drains the work items (DM tile x time tile) of
 * up to 64 beams, with the costliest beams queued first, and small or
 * uneven beams no longer leave most of the GPU idle.
 *
 * dd_batch_create: `plans` (host array of nplans >= 1 plan pointers, all on
 * one device) must outlive the batch; a plan may appear once.
 * dd_batch_run: for beam i, block[i], nsamp_in[i], pitch_elems[i], out[i],
 * cands[i] (device, capacity[i] slots, NULL when capacity[i] == 0) as for
 * dd_run with plans[i]; counts[i] (host) receives beam i's total.  Results
 * per beam are identical to dd_run.  Synchronises `stream` once.  Returns the
 * first error, else DD_ERR_OVERFLOW if any count exceeds its capacity (every
 * beam's first capacity[i] candidates are still written), else DD_OK. */
typedef struct dd_batch dd_batch;
int dd_batch_create(dd_batch **out, dd_plan *const *plans, int32_t nplans);
/* The batch's launch sequence is captured into a CUDA graph after the first
 * run of an argument set and replayed (one graph launch on `stream`) while
 * the arguments, the plans' workspaces and their kernel settings (path,
 * wait timeout, fault injection) stay the same; anything else runs directly
 * and re-captures.  dd_batch_graph_replays: runs served by the graph. */
int dd_batch_graph_replays(const dd_batch *b, int64_t *replays);
int dd_batch_destroy(dd_batch *b);
int dd_batch_run(dd_batch *b, const void *const *block, const int64_t *nsamp_in,
                 const int64_t *pitch_elems, void *const *out, float nsigma,
                 dd_candidate *const *cands, const int64_t *capacity, int64_t *counts,
                 void *stream);

/* Streams (Sec. 3.4: each block is dedispersed together with the previous
 * block's last maxshift samples, kept on the device, so that the output runs
 * on without gaps).  A stream belongs to one plan and takes blocks of
 * `block_samples` samples per channel; before its first block the history is
 * zeros.  Push k of a stream writes out[ndm][block_samples] = the dedispersed
 * samples k*block_samples - maxshift .. (k+1)*block_samples - maxshift - 1 of
 * the stream (zeros before sample 0), with detection as in dd_run.
 *
 * dd_stream_bytes: device bytes one stream of this plan and block length
 * needs (its double buffer, one output block, detection workspace), for
 * admission against free memory.
 * dd_streams_push: one block for each of n streams (distinct plans, one
 * device) in one wave -- block[i] a device array [nchan][pitch_elems[i]] of
 * the plan's dtype, out[i], cands[i], capacity[i], counts[i] as for
 * dd_batch_run; the staged u8 beams of the wave share persistent launches.
 * Synchronises `stream` once; status codes as for dd_batch_run. */
typedef struct dd_stream dd_stream;
int dd_stream_bytes(const dd_plan *p, int64_t block_samples, int64_t *bytes);
int dd_stream_create(dd_stream **out, dd_plan *p, int64_t block_samples);
int dd_stream_destroy(dd_stream *s);
int dd_streams_push(dd_stream *const *streams, int32_t n, const void *const *block,
                    const int64_t *pitch_elems, void *const *out, float nsigma,
                    dd_candidate *const *cands, const int64_t *capacity, int64_t *counts,
                    void *stream);

/* Host copies of the per-DM mean and rms computed by the last dd_detect,
 * dd_run or dd_batch_run on this plan (double[ndm] each; either pointer may
 * be NULL). */
int dd_get_stats(const dd_plan *p, double *mean, double *sigma);

/* Synchronise `stream` and return the plan's sticky device status
 * (DD_OK or DD_ERR_DEVICE_TIMEOUT), clearing it. */
int dd_sync(dd_plan *p, void *stream);

/* Whole path on host buffers: copy `host_block` ([nchan][pitch_elems],
 * host memory, pinned for full speed) to plan-owned device memory, dedisperse
 * and detect (dd_run) and copy the candidates back to
 * `host_cands` (host, `capacity` slots).  *count as for dd_detect.  The plan
 * grows its device buffers on first use for a given nsamp_in / pitch and keeps
 * them until destroyed.  Synchronises `stream` before returning. */
int dd_process_host(dd_plan *p, const void *host_block, int64_t nsamp_in, int64_t pitch_elems,
                    float nsigma, dd_candidate *host_cands, int64_t capacity, int64_t *count,
                    void *stream);

/* Host pipes: dd_process_host over a sequence of host blocks with the copy
 * of each block overlapped with the previous block's dedispersion (the
 * thesis's double-buffered input, filled while the GPU works on the previous
 * buffer, Sec. 4.2).  A pipe belongs to one plan and
 * takes blocks of one shape ([nchan][pitch_elems] host memory, the first
 * nsamp_in samples of each row used; pinned memory lets the copies run
 * asynchronously) and owns two device input buffers, one output and a
 * candidate buffer of `capacity` slots, and its own copy stream.
 *
 * dd_host_pipe_push queues the copy of `host_block` on the copy stream, then,
 * if an earlier block's result is still due, runs dd_run with `nsigma` on
 * that block on `stream` while the new copy is in flight and copies its
 * candidates to `host_cands` (host, `capacity` slots): *has_result = 1 and
 * *count = its total; otherwise *has_result = 0.  dd_host_pipe_flush returns
 * the last pushed block's result the same way (*has_result = 0 when none is
 * due).  So push k returns block k-1's result, and one flush after the last
 * push returns the last block's.  host_block must stay unchanged until the
 * next push or flush returns.  Each result equals dd_process_host of its
 * block; status codes as for dd_process_host (DD_ERR_OVERFLOW when the total
 * exceeds capacity; the first capacity candidates are still returned).
 * Synchronises `stream` before returning.  Not thread-safe; the plan must
 * not be used elsewhere while the pipe runs, and must outlive it. */
typedef struct dd_host_pipe dd_host_pipe;
int dd_host_pipe_create(dd_host_pipe **out, dd_plan *p, int64_t nsamp_in, int64_t pitch_elems,
                        float nsigma, int64_t capacity);
int dd_host_pipe_destroy(dd_host_pipe *q);
int dd_host_pipe_push(dd_host_pipe *q, const void *host_block, dd_candidate *host_cands,
                      int64_t *count, int32_t *has_result, void *stream);
int dd_host_pipe_flush(dd_host_pipe *q, dd_candidate *host_cands, int64_t *count,
                       int32_t *has_result, void *stream);

/* Number of kernel launches queued by this plan since creation (all entry
 * points); used to account for device work. */
int dd_plan_launch_count(const dd_plan *p, int64_t *launches);

/* Autotuning (plan time).  The thesis sets the accumulators per thread and
 * threads per block by a hand sweep for its GPU (Sec. 2.4); here each staged
 * kernel is compiled for several tile widths (u8: 64, 32 or 16 DM trials per
 * CTA; f16/f32: 128 or 64) and the u8 kernel also for staging depths 1, 2
 * and 3 (input windows queued that many channel chunks ahead of the chunk
 * being built), and the plan takes the widest width whose delay patterns
 * fit, at depth 2.  dd_plan_autotune instead times every width (and, for
 * u8, every depth) that fits, on a scratch block of nsamp_in samples of the
 * plan's geometry (allocated and freed here; the choice depends on the
 * channel / DM geometry, so a shorter block tunes faster), and keeps the
 * fastest.  *dms_per_cta receives the chosen width (0: no staged width fits;
 * the plain-load kernel stays; dd_plan_kernel_info reports the depth), and
 * *ms_per_launch (may be NULL) its median time.  Results of dd_execute /
 * dd_run do not depend on the width or depth.  Synchronous. */
int dd_plan_autotune(dd_plan *p, int64_t nsamp_in, int32_t *dms_per_cta, float *ms_per_launch);

/* Kernel selection: path 0 (default) lets dd_execute take the staged kernel
 * whenever the plan and the block's layout allow it; path 1 forces the
 * plain-load kernel (same results; used to cross-check the two). */
int dd_plan_set_path(dd_plan *p, int32_t path);

/* Upper bound, in nanoseconds, on every device-side wait of the staged
 * kernel (default 2e9).  A wait that runs out makes the launch record
 * DD_ERR_DEVICE_TIMEOUT (reported by the next synchronising call) and leave
 * its output unwritten.  DD_ERR_ARG below 1000 ns. */
int dd_plan_set_wait_timeout(dd_plan *p, int64_t timeout_ns);

/* Staging depth of the staged u8 kernel (1..3 channel chunks of input
 * windows queued ahead of the chunk being built; 2 by default, else what
 * dd_plan_autotune picked).  DD_ERR_ARG for a depth outside 1..3 or a plan
 * without the staged u8 kernel; DD_ERR_SIZE if that depth's buffers exceed
 * a CTA's shared memory (the depth is then unchanged).  Results do not
 * depend on it. */
int dd_plan_set_staging_depth(dd_plan *p, int32_t copy_ahead);

/* Fault injection for tests of the timeout path: with skip_copies != 0 the
 * staged kernel queues none of its bulk copies, so its first bounded wait
 * runs out, and dd_run's one-launch path for small float beams waits at its
 * grid barrier for one arrival more than its grid makes, so that wait
 * runs out (no device fault, no hang).  0 restores normal operation. */
int dd_plan_inject_fault(dd_plan *p, int32_t skip_copies);

/* Which kernel dd_execute would use for `block` / `pitch_elems`:
 * *staged = 1 for the staged (bulk-copy) kernel, 0 for the plain-load one;
 * *dms_per_cta, *smem_bytes and *copy_ahead describe the staged kernel's
 * tiling and staging depth (0 when the plan has none; the depth is 0 for the
 * f16/f32 kernel, whose depth is fixed).  Any of the last three may be
 * NULL. */
int dd_plan_kernel_info(const dd_plan *p, const void *block, int64_t pitch_elems,
                        int32_t *staged, int32_t *dms_per_cta, int32_t *smem_bytes,
                        int32_t *copy_ahead);

/* dd_detect without allocation.  The thesis has no counterpart: this entry
 * point exists for callers that must not allocate device memory at run time
 * -- for example a process whose device memory is entirely reserved up front
 * by another allocator (a framework's caching allocator), or a real-time loop
 * that may not call cudaMalloc because it can synchronise the device and stall
 * the stream -- and that therefore cannot create a plan.
 *
 * It runs the same normalisation and threshold passes as dd_detect on
 *   out: device pointer, [ndm][nsamp_out], int32 when in_dtype is DD_U8,
 *        float when it is DD_F16 or DD_F32 (the dd_execute output types),
 * writes up to `capacity` candidates to the device array `cands` in (dm_idx,
 * t) order and the total found to the host pointer *count, with the same
 * statistics, threshold rule and status codes as dd_detect.
 *
 * Scratch memory: one file-scope device array of 4.5 MiB (per-row statistics,
 * per-chunk counts and offsets), which every GPU that loads the library keeps
 * until the process exits.  Limits: ndm <= 16384 and
 * ndm * ceil(nsamp_out / 4096) <= 262144; larger sizes return DD_ERR_SIZE
 * before anything is queued.  The call makes no cudaMalloc, cudaFree or other
 * allocating call; it runs on the calling thread's current device.  Its first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress), and so does the first call after that device's
 * context has been re-created (for example by cudaDeviceReset): make those
 * first calls before any stream capture.  Every call uses the same array and leaves its contents behind (nothing in
 * it needs to start at zero): calls whose work overlaps on the GPU -- on
 * different streams, or from different host threads -- race and must be
 * serialised by the caller.  Synchronises `stream` once (to return *count). */
int dd_detect_noalloc(const void *out, int32_t in_dtype, int32_t ndm, int64_t nsamp_out,
                      float nsigma, dd_candidate *cands, int64_t capacity, int64_t *count,
                      void *stream);

/* Static description of a status code. */
const char *dd_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
