/*
 * lof.h -- C ABI of the GB300-native LOFAR Online Flagger (LOF) hot path.
 *
 * The operation is the real-time flagger of "Towards Exascale Real-Time RFI
 * Mitigation" (van Nieuwpoort, 2017), applied independently to every "unit":
 * one (station, polarisation, subband) block of n_chan channels x n_time
 * samples (pre-correlation placement, Section 3), or one beam-formed Stokes I
 * subband (post-beam-forming placement).  Per unit, in this order:
 *   a1  power P[c,t] = re^2 + im^2 of the complex voltages (Section 4: complex
 *       input is turned into power before flagging); Stokes I input is already
 *       power;
 *   a2  time-integrated spectrum S[c] = sum_t P[c,t] (Section 3: for frequency
 *       flagging the time axis is summed away entirely);
 *   a3  median and robust stddev of S (Section 4.2);
 *   a4  SumThreshold over S (Section 2.1) -> whole channels flagged;
 *   a5  median and robust stddev pooled over every sample of the channels the
 *       frequency pass kept (Section 4: frequency flagging first protects the
 *       statistics);
 *   a6  SumThreshold along time in every kept channel, windows 1, 2, 4, ...,
 *       max_window (Section 2.1);
 *   a7  history flagger per channel (Section 4.1): the mean of the unflagged
 *       samples against mean + k * stddev of the means of earlier blocks;
 *   a8  mask = frequency | time | history flags; flagged samples of the output
 *       are zeroed (flagged data is removed before the beam former, Section 3).
 * SumThreshold (Section 2.1): threshold_I = median + stddev * factor_I *
 * sensitivity with factor_I = start_threshold * p^(log2 I) / I.  A window of I
 * samples is flagged when the sum of its samples, flagged ones counted as
 * threshold_I, exceeds I * threshold_I; windows of one size see the flags of
 * the smaller sizes only; windows lie inside the row.  "stddev" is
 * 1.482602218505602 * MAD (population stddev when the MAD is 0).
 *
 * Integer voltages give bit-exact masks: powers and window sums are exact
 * integers, and every threshold is the same binary64 formula, compared as an
 * integer table floor((I - n_flagged) * threshold_I).
 *
 * Conventions
 *  - Every call returns an int status (LOF_OK or a negative LOF_ERR_*) and
 *    never aborts; lof_last_error() gives a message for the last failure.
 *  - Calls are asynchronous on the caller's CUDA stream (a cudaStream_t passed
 *    as void*, NULL = legacy default stream).  Device-side failures (a bounded
 *    wait that timed out, an internal limit) set an error word in the context;
 *    the next call, or lof_status(), returns them.
 *  - The caller owns every data buffer (device memory, e.g. from PyTorch);
 *    the context owns the history rings and its scratch memory.
 *  - One context must not be used from two host threads at once, nor have two
 *    lof_flag_block calls in flight on different streams at the same time
 *    (they share scratch); calls on one stream are ordered.
 */
#ifndef LOF_H
#define LOF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lof_ctx lof_ctx;

enum {
  LOF_OK = 0,
  LOF_ERR_INVALID = -1,     /* bad argument, pointer, alignment or shape */
  LOF_ERR_NOMEM = -2,       /* device or host allocation failed */
  LOF_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  LOF_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
  LOF_ERR_STATE = -5,       /* call out of order (e.g. history not sized) */
  LOF_ERR_UNSUPPORTED = -6  /* valid request this build does not implement */
};

/* Sample types.  CI8 / CI16: complex voltages, interleaved (re, im) int8 or
 * int16 pairs, one element = one complex sample; results are exact (integer
 * window sums against an integer threshold table).  F32: Stokes I power
 * (Section 4: the power is given); non-finite samples are flagged on entry.
 * F32 statistics agree with binary64 within 1e-6 relative and window sums
 * are float32 trees of at most 64 terms, so a flag can differ from binary64
 * arithmetic only where a window sum lies within ~1e-6 of its threshold.
 * CF32: complex float32 visibilities (interleaved re, im; the post-correlation
 * placement of Section 3), one element = one complex sample of 8 bytes; the
 * power re^2 + im^2 is formed in float32 and flagged like F32 (same
 * tolerance; non-finite re or im flags the sample; a flagged sample's output
 * is 0 + 0i). */
enum { LOF_CI8 = 1, LOF_CI16 = 2, LOF_F32 = 3, LOF_CF32 = 4 };

enum { LOF_SIGMA_MAD = 0, LOF_SIGMA_STD = 1, LOF_SIGMA_WINSOR = 2 };

enum { LOF_TIME_PER_CHANNEL = 0, LOF_TIME_INTEGRATED = 1, LOF_TIME_2D = 2 };

enum { LOF_SCOPE_POOLED = 0, LOF_SCOPE_CHANNEL = 1 };

typedef struct {
  double p;                /* Section 2.1, default 1.5 */
  double sensitivity;      /* Section 2.1, default 1.0 */
  double start_threshold;  /* Section 2.1, default 6 ("6 sigma" at I = 1) */
  int32_t max_window;      /* largest SumThreshold window, power of two <= 64; default 64 */
  int32_t history_len;     /* history ring capacity per channel, 1..1024; default 60 */
  int32_t history_min;     /* stored means needed before the history test; default 8 */
  double history_k;        /* history threshold = mean + k * stddev; default 6 */
  int32_t sigma_estimator; /* Section 4.2 statistics: LOF_SIGMA_MAD (default, 1.4826 * MAD),
                              LOF_SIGMA_STD (population stddev) or LOF_SIGMA_WINSOR (the
                              lowest and highest n / 10 values clamped to the nearest kept
                              order statistic, population stddev of the clamped values times
                              1.2138796046717422, which makes it estimate sigma of normal
                              data).  Each falls back to the plain stddev when it is 0.
                              LOF_SIGMA_WINSOR takes integer units and n_time <= 16384; it
                              runs on the exact-statistics unit kernel (one CTA per unit) */
  int32_t enable_freq;     /* frequency pass on (1) / off (0) */
  int32_t enable_time;     /* time pass on / off */
  int32_t enable_history;  /* history flagger on / off */
  int32_t sir_percent;     /* Section 2.2 scale-invariant rank operator on the final mask,
                              eta in percent (0 = off, the default; at most 99): a sample
                              is flagged when some interval holding it, along time or
                              then along frequency, is at least (100 - eta)% flagged.
                              Needs the mask output of every unit; runs after the history
                              values are staged (it changes the mask, the data and
                              n_flag_total, not the history) */
  int32_t time_mode;       /* LOF_TIME_PER_CHANNEL (default): SumThreshold along time on
                              every kept channel with the pooled statistics;
                              LOF_TIME_INTEGRATED (Section 3): the frequency direction
                              integrated fully -- one series of the summed powers of the
                              kept channels, its own median and sigma, one SumThreshold,
                              a flagged time step flagged in every kept channel.
                              Integer units only, n_time <= 16384.
                              LOF_TIME_2D (Sections 2.1 and 3 mention a 2-D flagger that
                              integrates partially): replaces both passes -- the powers are
                              summed into cells of integ_chan x integ_time samples, one
                              median and sigma are taken over the cells, and for each window
                              size SumThreshold runs along time on every row of cells and
                              then along frequency on every column (enable_time /
                              enable_freq switch the directions); a flagged cell flags all
                              of its samples; median_f, sigma_f, n_chan_freq are reported as
                              0 and median_t, sigma_t are the cells' statistics.  Integer
                              units; the cell sizes divide n_chan and n_time; at most 16384
                              cells per unit */
  int32_t stats_scope;     /* statistics of the per-channel time pass (Section 4.2 reading):
                              LOF_SCOPE_POOLED (default) -- one median and sigma pooled over
                              the unit's kept channels; LOF_SCOPE_CHANNEL -- each kept
                              channel's own median and sigma over its own samples (the
                              unit's median_t and sigma_t are then reported as 0).
                              LOF_SCOPE_CHANNEL takes integer units, time_mode
                              LOF_TIME_PER_CHANNEL and n_time <= 16384 */
  int32_t integ_chan;      /* LOF_TIME_2D: channels per cell (default 1) */
  int32_t integ_time;      /* LOF_TIME_2D: samples per cell (default 1); integ_chan *
                              integ_time <= 65536 */
} lof_params;

/* Per-unit results, written by lof_flag_block when lof_unit.stats != NULL
 * (device memory).  Medians and sigmas are the values the thresholds used. */
typedef struct {
  double median_f, sigma_f; /* spectrum statistics (a3); 0 in LOF_TIME_2D */
  double median_t, sigma_t; /* pooled statistics of the time pass (a5); those of the
                               integrated series (LOF_TIME_INTEGRATED), of the cells
                               (LOF_TIME_2D); 0 with LOF_SCOPE_CHANNEL */
  int64_t n_chan_freq;      /* channels flagged by the frequency pass */
  int64_t n_flag_time;      /* samples flagged by the time pass (the 2-D pass in LOF_TIME_2D) */
  int64_t n_chan_hist;      /* channels flagged by the history flagger */
  int64_t n_flag_total;     /* ones in the mask */
} lof_unit_stats;

/* One unit.  All pointers are device pointers owned by the caller.
 *  in    : n_chan rows of n_time samples; row c starts at in + c*in_row_stride
 *          elements.  Must be aligned to the element size.
 *  out   : same layout (out_row_stride); receives in with flagged samples set
 *          to zero.  NULL = no data output.  out == in (same strides) flags in
 *          place: only flagged samples are written.
 *  mask  : uint8 0/1 per sample, row c at mask + c*mask_row_stride.  NULL = none.
 *  history_slot: first of n_chan consecutive history slots of the context, or
 *          -1 for no history (the history flagger is then skipped for the unit).
 *  stats : optional device lof_unit_stats*, or NULL.
 * Limits: 1 <= n_chan <= 2048, 1 <= n_time; the flag words of one row (one
 * bit per sample) must fit a CTA's shared memory, and a float32 row's flag
 * words times 8 as well (n_time up to ~400000 with the default tuning; see
 * lof_max_time()). */
typedef struct {
  const void *in;
  void *out;
  uint8_t *mask;
  int32_t n_chan, n_time;
  int64_t in_row_stride, out_row_stride, mask_row_stride;
  int64_t history_slot;
  lof_unit_stats *stats;
} lof_unit;

/* Fill *p with the defaults above. */
void lof_default_params(lof_params *p);

/* Create a context on CUDA device cuda_device with n_history_slots history
 * channels (each a ring of history_len binary64 means, Section 4.1, sized as
 * in the paper's storage estimate: slots x history_len x 8 bytes).  Allocates
 * device memory; runs no kernel except memsets.  *out receives the context. */
int lof_create(const lof_params *params, int cuda_device, int64_t n_history_slots,
               lof_ctx **out);

/* Flag one block of n_units units of sample type dtype (steps a1-a8 above) in
 * ONE persistent kernel launch on cuda_stream.  units is a host array, read
 * during the call.  History rings are read, not modified: the value each
 * channel would add to its ring is staged and committed by
 * lof_history_update (the paper processes seconds out of order, Section 4.1,
 * so the commit is a separate step).  block_seq is an opaque sequence number
 * recorded with the staged values.  Returns LOF_ERR_INVALID for bad
 * descriptors (nothing launched), or a pending device error. */
int lof_flag_block(lof_ctx *ctx, int dtype, const lof_unit *units, int n_units,
                   uint64_t block_seq, void *cuda_stream);

/* Same operation with HOST buffers: in/out/mask/stats of every unit are host
 * pointers (pinned memory gives asynchronous copies).  Inputs are copied to
 * context-owned device staging memory, flagged, and out/mask/stats copied
 * back.  The units are taken in up to 16 chunks of whole units: a chunk's
 * uploads run on an internal copy stream, its flag launch on cuda_stream
 * (after those uploads) and its downloads on a second internal copy stream
 * (after that launch), so the copies of neighbouring chunks overlap the
 * kernel; each chunk's uploads are issued after the previous chunk's launch.
 * Consecutive units whose host buffers are contiguous move as one copy.  The
 * copies start after the work already queued on cuda_stream, and cuda_stream
 * waits for the last download: the call returns after enqueueing, and
 * synchronising cuda_stream covers all of it.  Host buffers must stay valid
 * until then. */
int lof_flag_block_host(lof_ctx *ctx, int dtype, const lof_unit *units, int n_units,
                        uint64_t block_seq, void *cuda_stream);

/* Section 4.1 commit: for every channel of the given units (history_slot >= 0)
 * append the value staged by the last lof_flag_block to its ring, dropping the
 * oldest once history_len means are held, and refresh the cached
 * mean + k*stddev threshold.  Channels with nothing staged are unchanged. */
int lof_history_update(lof_ctx *ctx, const lof_unit *units, int n_units, void *cuda_stream);

/* Copy n slots starting at slot0 of the history to / from host memory:
 * values[n][history_len] oldest -> newest (unused tail zero) and counts[n].
 * Synchronous (waits for the context's work).  For checkpointing and tests. */
int lof_history_export(lof_ctx *ctx, int64_t slot0, int64_t n, double *values, int32_t *counts);
int lof_history_import(lof_ctx *ctx, int64_t slot0, int64_t n, const double *values,
                       const int32_t *counts);

/* Wait for cuda_stream and return the first device-side error recorded by the
 * context's kernels (LOF_ERR_TIMEOUT, ...) or LOF_OK; clears it. */
int lof_status(lof_ctx *ctx, void *cuda_stream);

/* Work counters of the last lof_flag_block on ctx (not of graph replays):
 * counts[0] = units whose pooled time-pass statistics needed another pass
 * over their data after the first counting pass (the counts near the previous
 * block's median and MAD did not pin them down, or the block left its value
 * window), counts[1] = such passes that read a unit's kept rows again.
 * Waits for cuda_stream.  Instrumentation of the exact
 * selection (Section 4.2 asks for O(N) medians); results never depend on it. */
int lof_block_counters(lof_ctx *ctx, void *cuda_stream, int64_t *counts);

/* Largest n_time a unit of dtype may have with the current tuning. */
int lof_max_time(const lof_ctx *ctx, int dtype);

/* Launch-shape knobs (an autotuner sweeps them; results do not depend on
 * them).  0 keeps the current value. */
typedef struct {
  int32_t threads;         /* threads per CTA: 128 or 256 (default) */
  int32_t ctas_per_sm;     /* resident CTAs per SM: 1 to 4 (default 2) */
  int32_t tile_bytes;      /* cap on the shared-memory bytes of a CTA */
  int32_t fine_bins;       /* counters per exact-selection refinement round */
  int32_t flag_rows;       /* rows per time-pass task (tile height), 1..64 (default 64) */
  int32_t stat_samples;    /* samples per statistics task, >= 1024 (default 262144;
                              at most 64 rows) */
  int32_t schedule;        /* window schedule of the time pass (Section 2.1's window sizes
                              over a row): LOF_SCHED_SET plus any of
                              LOF_SCHED_PACKED (rows whose values fit run in the packed
                              low-bit form, one warp per 1024-sample segment in registers;
                              without it every row takes the general path, exact 64-bit
                              window sums over a shared-memory prefix), LOF_SCHED_BOUND64
                              (the 64-sample windows are first screened by an exact bound on
                              sums of blocks of four; without it every window is tested) and
                              LOF_SCHED_COALESCED (the masked data of a segment leaves with
                              coalesced 16-byte stores; without it one bulk copy per lane),
                              and for the statistics LOF_SCHED_VALUE_WINDOW (a unit whose
                              history slot holds the previous block's median m and MAD d,
                              with d small enough, counts its pooled powers value by value
                              in a window of 4096 values around m plus one count below it,
                              and resolves median and MAD from those counts; a block whose
                              statistics leave the window is counted again in full), and for
                              Stokes I (LOF_F32) units LOF_SCHED_F32_CLUSTER (one thread-block
                              cluster of 16, or 8, CTAs per unit holds the unit in shared
                              memory, read from global memory once, where it fits: at most 256
                              channels; otherwise, or without it, one CTA per unit; the input is
                              read once, but the unit's statistics passes then wait on cluster
                              barriers, so it is off by default).
                              Default LOF_SCHED_SET | LOF_SCHED_PACKED | LOF_SCHED_BOUND64 |
                              LOF_SCHED_COALESCED | LOF_SCHED_VALUE_WINDOW */
} lof_tuning;
enum {
  LOF_SCHED_PACKED = 1,
  LOF_SCHED_BOUND64 = 2,
  LOF_SCHED_COALESCED = 4,
  LOF_SCHED_VALUE_WINDOW = 8,
  LOF_SCHED_F32_CLUSTER = 16,
  LOF_SCHED_SET = 0x80
};
int lof_set_tuning(lof_ctx *ctx, const lof_tuning *t);
int lof_get_tuning(const lof_ctx *ctx, lof_tuning *t);

/* Autotuner: times lof_flag_block on these units (reps timed launches after
 * one warm-up, median) for every candidate launch shape -- threads per CTA,
 * CTAs per SM, rows per time-pass task, samples per statistics task -- and
 * then, with the fastest shape, every window schedule (the packed or the
 * general time pass, the bound on the 64-sample windows on or off, coalesced
 * or bulk data stores, value-window statistics on or off), and keeps the fastest in the context (*best, *best_ms
 * if not NULL).  Results never depend on the tuning.  Synchronous; stages
 * history values like any lof_flag_block call (do not commit them).  Float
 * units have no launch shape; for F32 the cluster bit is tried both ways. */
int lof_autotune(lof_ctx *ctx, int dtype, const lof_unit *units, int n_units, int reps,
                 void *cuda_stream, lof_tuning *best, float *best_ms);

/* Graph form of a block (the batching pattern for fixed buffers: every
 * station x polarisation x subband of a real-time pipeline, re-flagged each
 * block in the same device buffers).  lof_graph_create builds and uploads the
 * descriptors of n_units units once (pointers, shapes and strides are fixed
 * from then on; the data in the buffers changes freely) and captures the
 * device-side steps of lof_flag_block -- state reset, the one persistent
 * launch, the error-word copy -- in a CUDA graph, with the context's current
 * tuning and parameters.  lof_graph_launch replays it on cuda_stream with the
 * given block sequence number; history values are staged in the context's
 * slots exactly as by lof_flag_block (commit them with lof_history_update).
 * Replays of one graph must be ordered on one stream.  lof_graph_launch
 * returns a device-side error of the previous replay once it has finished;
 * lof_graph_status waits for cuda_stream and returns it. */
typedef struct lof_graph lof_graph;
int lof_graph_create(lof_ctx *ctx, int dtype, const lof_unit *units, int n_units,
                     lof_graph **out);
int lof_graph_launch(lof_graph *graph, uint64_t block_seq, void *cuda_stream);
int lof_graph_status(lof_graph *graph, void *cuda_stream);
int lof_graph_destroy(lof_graph *graph);

/* Flag one block of units like lof_flag_block, without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate memory while they run -- real-time processing threads that
 * cannot afford cudaMalloc/cudaFree (which block and synchronise the device),
 * processes with a fixed allocation budget, or hosts without a memory pool.
 * It needs no context: params may be NULL (defaults; otherwise checked as
 * lof_create checks them), and the history flagger is unavailable (every unit
 * must have history_slot = -1).  Its scratch is
 * one file-scope device array of 64 MiB that every GPU which loads the
 * library holds until the process exits (about 40 KB per unit plus 9 bytes
 * per channel); host-side descriptors live in fixed static arrays (at most
 * 1024 units and 262144 tasks per call).  A block
 * that does not fit is rejected with LOF_ERR_INVALID and a message
 * (lof_last_error(NULL)); nothing is launched then.
 * The first call on each device looks up the device address of the array
 * (with that device current); make that first call before any stream
 * capture.  The unit descriptors are uploaded from fixed host arrays that
 * the next call reuses, so while cuda_stream is capturing the call returns
 * LOF_ERR_INVALID and enqueues nothing; the upload copies from pageable host
 * memory and may wait for work already queued on cuda_stream.  All calls
 * share the array and it keeps the last call's contents:
 * each call clears what must start at zero, but calls whose work overlaps on
 * the GPU (different streams, or different host threads without ordering)
 * race on it -- serialise them.  status: optional DEVICE int that receives
 * the device-side status of this call (0 = ok, else a device error code) when
 * the stream reaches it; NULL = not reported.  Returns LOF_OK when the work
 * was enqueued on cuda_stream. */
int lof_flag_block_noalloc(const lof_params *params, int dtype, const lof_unit *units, int n_units,
                           int *status, void *cuda_stream);

/* Message for the last failed call on ctx (or of lof_create when ctx is NULL). */
const char *lof_last_error(const lof_ctx *ctx);

int lof_destroy(lof_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
