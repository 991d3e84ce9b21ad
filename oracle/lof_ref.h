/*
 * lof_ref.h -- ORACLE for the LOFAR Online Flagger (LOF) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded CPU
 * restatement of what the flagger computes, written from the paper
 * ("Towards Exascale Real-Time RFI Mitigation", van Nieuwpoort, 2017):
 *   Section 2.1  SumThreshold and its threshold schedule,
 *   Section 4    power first, frequency flagging on the time-integrated
 *                spectrum, then time flagging,
 *   Section 4.1  the history flagger,
 *   Section 4.2  medians / MAD / standard deviations.
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may use
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Arithmetic: every floating-point step is one IEEE binary64 operation in the
 * order written (build with -ffp-contract=off, no fast-math).  For integer
 * voltages all powers, sums and medians are integers (or halves) below 2^53,
 * so they are exact in binary64.
 *
 * Pins: tests/test_oracle_pins.py and tests/test_oracle_invariants.py check
 * every function here against the paper's printed thresholds (6 and 4.5
 * sigma), hand-worked SumThreshold examples, a brute-force window enumerator,
 * numpy/scipy statistics and closed-form flag rates.
 */
#ifndef LOF_REF_H
#define LOF_REF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { LOF_REF_CI8 = 1, LOF_REF_CI16 = 2, LOF_REF_F32 = 3,
       LOF_REF_CF32 = 4 /* complex float32 visibilities (post-correlation) */ };
enum { LOF_REF_SIGMA_MAD = 0, LOF_REF_SIGMA_STD = 1, LOF_REF_SIGMA_WINSOR = 2 };

typedef struct {
  double p;               /* Section 2.1: 1.5 */
  double sensitivity;     /* Section 2.1: 1.0 */
  double start_threshold; /* Section 2.1: 6 (the "6 sigma" of the first iteration) */
  int max_window;         /* largest window, a power of two (64) */
  int history_len;        /* ring capacity H (60) */
  int history_min;        /* entries needed before the history test runs (4) */
  double history_k;       /* history threshold multiplier (6) */
  int sigma_estimator;    /* LOF_REF_SIGMA_MAD, LOF_REF_SIGMA_STD or LOF_REF_SIGMA_WINSOR */
  int enable_freq, enable_time, enable_history;
  int sir_percent;        /* Section 2.2 SIR operator, eta in percent (0 = off) */
  int time_mode;          /* 0: time pass per channel; 1: on the frequency-integrated series;
                             2: two-dimensional SumThreshold on integration cells */
  int stats_scope;        /* time-pass statistics: 0 pooled over the unit; 1 per channel */
  int integ_chan, integ_time; /* time_mode 2: channels x samples summed into one cell (1 = none);
                                 each divides the unit's size in its direction */
} lof_ref_params;

typedef struct {
  double median_f, sigma_f; /* statistics of the time-integrated spectrum */
  double median_t, sigma_t; /* pooled statistics for the time pass */
  int64_t n_chan_freq;      /* channels flagged by the frequency pass */
  int64_t n_flag_time;      /* samples newly flagged by the time pass */
  int64_t n_chan_hist;      /* channels flagged by the history flagger */
  int64_t n_flag_total;     /* mask ones */
} lof_ref_stats;

/* Section 2.1: factor_I for I = 2^k. */
double lof_ref_factor(const lof_ref_params *pr, int k);
/* Section 2.1: threshold_I = median + stddev * factor_I * sensitivity. */
double lof_ref_threshold(const lof_ref_params *pr, double median, double sigma, int k);
/* Median of n values (sorts a private copy). */
double lof_ref_median(const double *x, int64_t n);
/* Robust sigma: 1/Phi^-1(3/4) * MAD, falling back to the population standard
 * deviation when the MAD is 0; is_int selects exact integer moments.
 * Writes the median to *median. */
double lof_ref_sigma(const lof_ref_params *pr, const double *x, int64_t n, int is_int,
                     double *median);
/* Section 2.1: one-dimensional SumThreshold over v[0..L).  flags[] holds the
 * entry flags on input and the result on output. */
void lof_ref_sum_threshold(const lof_ref_params *pr, const double *v, int64_t L, double median,
                           double sigma, uint8_t *flags);

/* Section 2.2: the scale-invariant rank operator on one line of a mask,
 * f[i * stride] for i < L (values 0/1).  Output g[i * gstride] = 1 exactly when
 * some interval [a, b) holding i has at least (100 - percent)% of its samples
 * flagged in f.  f and g may be the same array. */
void lof_ref_sir(const uint8_t *f, int64_t L, int64_t stride, int percent, uint8_t *g,
                 int64_t gstride);

/* One unit (C channels x T samples, time fastest) through the whole hot path.
 * in/out/mask strides are in elements of the respective array.  ring holds
 * the history of each channel oldest -> newest (C x history_len values, with
 * ring_count[c] valid entries); it is read only.  pending[c] / has_pending[c]
 * receive the value the history flagger stages for each channel.  out, mask,
 * ring, pending, stats may be NULL.  Returns 0, or -1 on invalid arguments. */
int lof_ref_flag_unit(const lof_ref_params *pr, int dtype, const void *in, int C, int T,
                      int64_t in_stride, void *out, int64_t out_stride, uint8_t *mask,
                      int64_t mask_stride, const double *ring, const int32_t *ring_count,
                      double *pending, uint8_t *has_pending, lof_ref_stats *stats);

/* Section 4.1: append each staged value to its channel's ring (dropping the
 * oldest entry once history_len entries are held). */
void lof_ref_history_commit(const lof_ref_params *pr, int C, double *ring, int32_t *ring_count,
                            const double *pending, const uint8_t *has_pending);

#ifdef __cplusplus
}
#endif
#endif
