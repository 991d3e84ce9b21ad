/*
 * lof_ref.c -- ORACLE for the LOFAR Online Flagger hot path (test
 * infrastructure only; see lof_ref.h).  Plain loops in the paper's order and
 * notation, one binary64 operation per written step.
 *
 * Readings of points the paper leaves open (each is restated in the design
 * notes of the repository):
 *  - factor_I = startThreshold * p^(log2 I) / I, with startThreshold = 6, the
 *    only reading that yields the printed 6 sigma (I=1) and 4.5 sigma (I=2)
 *    of Section 2.1;
 *  - a window of I samples is flagged when the sum of its samples, with every
 *    already-flagged sample replaced by threshold_I, exceeds I*threshold_I
 *    (upper side only, strict '>'), i.e. sum_unflagged > (I - n_flagged) *
 *    threshold_I;
 *  - all windows of one size are judged against the flags of the previous
 *    sizes only (snapshot), windows lie fully inside the row;
 *  - "stddev" is the robust 1.4826*MAD (population stddev when the MAD is 0);
 *  - the winsorized estimator (sigma_estimator = 2; Section 4.2 lists
 *    winsorized means among the statistics) clamps the lowest and the highest
 *    k = floor(n / 10) of the n values to the nearest kept order statistic
 *    (10% winsorizing on each side), takes the population stddev of the
 *    clamped values and scales it by 1/sqrt(c) so that it estimates sigma of
 *    normal data (population stddev when the result is 0);
 *  - time-pass statistics pool every sample of the channels the frequency
 *    pass left unflagged (Section 4: flagging frequency first clears strong
 *    narrow-band interference, which would otherwise spoil these statistics);
 *  - the history flagger keeps one ring of per-channel means, multiplier k,
 *    ties flag (a channel is kept only when its mean is strictly below the
 *    threshold, as in the paper's code);
 *  - the integrated time mode (Section 3, time_mode = 1) sums the powers of the
 *    channels kept by the frequency pass into one series G[t] (entry-flagged
 *    samples left out), takes the statistics of its T values and runs
 *    SumThreshold on it; a flagged time step is flagged in every kept channel;
 *  - the per-channel statistics scope (stats_scope = 1, time_mode 0) gives
 *    each kept channel's time pass the median and sigma of that channel's own
 *    samples instead of the pooled ones (the unit's median_t and sigma_t are
 *    then reported as 0);
 *  - the two-dimensional mode (time_mode = 2; Sections 2.1 and 3 mention a 2-D
 *    flagger that integrates partially in one or both directions) replaces
 *    both one-dimensional passes: the powers are summed into cells of
 *    integ_chan channels x integ_time samples, one median and sigma are taken
 *    over the cells, and for each window size I SumThreshold runs along time
 *    on every row of cells and then along frequency on every column; a
 *    flagged cell flags all of its samples (enable_time / enable_freq switch
 *    the two directions);
 *  - the SIR operator (Section 2.2, optional) is the scale-invariant rank
 *    operator the section names, with eta = sir_percent / 100: a sample is
 *    flagged when an interval around it is at least (1 - eta) flagged.  It
 *    runs on the final mask, along time on every channel and then along
 *    frequency on every time step, after the history values are staged.
 */
#include "lof_ref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* 1/Phi^-1(3/4): scales the MAD of normal data to its standard deviation. */
static const double MAD_TO_SIGMA = 1.482602218505602;

/* 1/sqrt(c), c = the variance of a standard normal winsorized at its 10% and
 * 90% quantiles +-z (z = Phi^-1(0.9) = 1.2815515655446004):
 * c = 0.8 - 2 z phi(z) + 0.2 z^2 = 0.6786545589528744. */
static const double WINSOR_TO_SIGMA = 1.2138796046717422;

/* Section 2.1: factor_I = startThreshold * p^(log2 I) / I, I = 2^k.
 * p^k is formed by k successive multiplications. */
double lof_ref_factor(const lof_ref_params *pr, int k) {
  double pk = 1.0;
  for (int i = 0; i < k; ++i) pk = pk * pr->p;
  double f = pr->start_threshold * pk;
  return f / (double)((int64_t)1 << k);
}

/* Section 2.1: threshold_I = median + stddev * factor_I * sensitivity. */
double lof_ref_threshold(const lof_ref_params *pr, double median, double sigma, int k) {
  double a = sigma * lof_ref_factor(pr, k);
  double b = a * pr->sensitivity;
  return median + b;
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Textbook median: middle order statistic, or the mean of the two middle
 * ones for even n (Section 4.2 lists medians among the statistics). */
double lof_ref_median(const double *x, int64_t n) {
  if (n <= 0) return 0.0;
  double *s = (double *)malloc((size_t)n * sizeof(double));
  memcpy(s, x, (size_t)n * sizeof(double));
  qsort(s, (size_t)n, sizeof(double), cmp_double);
  double m = (n % 2) ? s[n / 2] : (s[n / 2 - 1] + s[n / 2]) * 0.5;
  free(s);
  return m;
}

/* Population standard deviation.  Integer data: exact moments,
 * M = n*sum(x^2) - (sum x)^2 in 128-bit integers, sigma = sqrt(M / n^2).
 * Float data: two sequential passes (mean, then squared deviations). */
static double population_std(const double *x, int64_t n, int is_int) {
  if (n <= 0) return 0.0;
  if (is_int) {
    unsigned __int128 s1 = 0, s2 = 0;
    for (int64_t i = 0; i < n; ++i) {
      unsigned __int128 v = (unsigned __int128)(uint64_t)x[i];
      s1 += v;
      s2 += v * v;
    }
    unsigned __int128 M = (unsigned __int128)(uint64_t)n * s2 - s1 * s1;
    double nn = (double)n * (double)n;
    return sqrt((double)M / nn);
  }
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = s + x[i];
  double mu = s / (double)n;
  double q = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = x[i] - mu;
    q = q + d * d;
  }
  return sqrt(q / (double)n);
}

/* Section 4.2 statistics: median and a robust stddev.  The MAD is the median
 * of |x - median|. */
double lof_ref_sigma(const lof_ref_params *pr, const double *x, int64_t n, int is_int,
                     double *median) {
  if (n <= 0) {
    *median = 0.0;
    return 0.0;
  }
  double m = lof_ref_median(x, n);
  *median = m;
  if (pr->sigma_estimator == LOF_REF_SIGMA_STD) return population_std(x, n, is_int);
  if (pr->sigma_estimator == LOF_REF_SIGMA_WINSOR) {
    /* winsorize: order statistics k and n-1-k bound the clamped values */
    double *s = (double *)malloc((size_t)n * sizeof(double));
    memcpy(s, x, (size_t)n * sizeof(double));
    qsort(s, (size_t)n, sizeof(double), cmp_double);
    const int64_t k = n / 10;
    const double lo = s[k], hi = s[n - 1 - k];
    for (int64_t i = 0; i < n; ++i) s[i] = x[i] < lo ? lo : (x[i] > hi ? hi : x[i]);
    double sw = population_std(s, n, is_int);
    free(s);
    if (sw > 0.0) return WINSOR_TO_SIGMA * sw;
    return population_std(x, n, is_int);
  }
  double *d = (double *)malloc((size_t)n * sizeof(double));
  for (int64_t i = 0; i < n; ++i) d[i] = fabs(x[i] - m);
  double mad = lof_ref_median(d, n);
  free(d);
  if (mad > 0.0) return MAD_TO_SIGMA * mad;
  return population_std(x, n, is_int);
}

/* Section 2.1 SumThreshold, one dimension.  For I = 1, 2, 4, ... up to
 * min(max_window, L): every window [t, t+I) fully inside the row is judged
 * against the flags left by the smaller windows; it is flagged when the sum
 * of its unflagged samples exceeds (I - n_flagged) * threshold_I.  A sigma
 * that is not positive flags nothing. */
void lof_ref_sum_threshold(const lof_ref_params *pr, const double *v, int64_t L, double median,
                           double sigma, uint8_t *flags) {
  if (!(sigma > 0.0) || L <= 0) return;
  uint8_t *next = (uint8_t *)malloc((size_t)L);
  for (int k = 0;; ++k) {
    int64_t I = (int64_t)1 << k;
    if (I > pr->max_window || I > L) break;
    double thr = lof_ref_threshold(pr, median, sigma, k);
    memcpy(next, flags, (size_t)L);
    for (int64_t t = 0; t + I <= L; ++t) {
      int64_t nf = 0;
      double su = 0.0;
      for (int64_t j = t; j < t + I; ++j) {
        if (flags[j])
          nf++;
        else
          su = su + v[j];
      }
      double limit = (double)(I - nf) * thr;
      if (su > limit)
        for (int64_t j = t; j < t + I; ++j) next[j] = 1;
    }
    memcpy(flags, next, (size_t)L);
  }
  free(next);
}

/* One window size of Section 2.1 on a line of L values v[i * stride], flags
 * f[i * stride]: every window [t, t + I) is judged against the flags on entry
 * and fires when the sum of its unflagged values exceeds
 * (I - n_flagged) * thr; the fired windows are flagged afterwards. */
static void st_one_size(const double *v, int64_t L, int64_t stride, int64_t I, double thr,
                        uint8_t *f) {
  uint8_t *next = (uint8_t *)malloc((size_t)(L > 0 ? L : 1));
  for (int64_t i = 0; i < L; ++i) next[i] = f[i * stride];
  for (int64_t t = 0; t + I <= L; ++t) {
    int64_t nf = 0;
    double su = 0.0;
    for (int64_t j = t; j < t + I; ++j) {
      if (f[j * stride])
        nf++;
      else
        su = su + v[j * stride];
    }
    double limit = (double)(I - nf) * thr;
    if (su > limit)
      for (int64_t j = t; j < t + I; ++j) next[j] = 1;
  }
  for (int64_t i = 0; i < L; ++i) f[i * stride] = next[i];
  free(next);
}

/* Section 2.2: scale-invariant rank operator on one line.  With integer
 * weights w = +percent for a flagged sample and -(100 - percent) for an
 * unflagged one, an interval [a, b) is at least (100 - percent)% flagged
 * exactly when its weight sum is >= 0.  With prefix sums Q[0] = 0,
 * Q[i + 1] = Q[i] + w[i], sample x lies in such an interval exactly when
 * max_{b > x} Q[b] >= min_{a <= x} Q[a] (the sum over [a, b) is Q[b] - Q[a]);
 * both extremes come from one pass each, so the operator is linear in L. */
void lof_ref_sir(const uint8_t *f, int64_t L, int64_t stride, int percent, uint8_t *g,
                 int64_t gstride) {
  if (L <= 0) return;
  int64_t *Q = (int64_t *)malloc((size_t)(L + 1) * sizeof(int64_t));
  int64_t *Qmax = (int64_t *)malloc((size_t)(L + 1) * sizeof(int64_t));
  Q[0] = 0;
  for (int64_t i = 0; i < L; ++i)
    Q[i + 1] = Q[i] + (f[i * stride] ? (int64_t)percent : -(int64_t)(100 - percent));
  /* Qmax[i] = max of Q[b] over b >= i */
  Qmax[L] = Q[L];
  for (int64_t i = L - 1; i >= 0; --i) Qmax[i] = Q[i] > Qmax[i + 1] ? Q[i] : Qmax[i + 1];
  int64_t qmin = Q[0];
  for (int64_t x = 0; x < L; ++x) {
    if (Q[x] < qmin) qmin = Q[x];         /* min of Q[a] over a <= x */
    g[x * gstride] = (uint8_t)(Qmax[x + 1] >= qmin);
  }
  free(Q);
  free(Qmax);
}

/* Section 4: the power of one sample (complex input is turned into power
 * before flagging); non-finite Stokes I values (or a non-finite part of a
 * complex visibility) are reported through *bad. */
static double sample_power(int dtype, const void *in, int64_t idx, int *bad) {
  *bad = 0;
  if (dtype == LOF_REF_CI8) {
    const int8_t *p = (const int8_t *)in + 2 * idx;
    double re = (double)p[0], im = (double)p[1];
    return re * re + im * im;
  }
  if (dtype == LOF_REF_CI16) {
    const int16_t *p = (const int16_t *)in + 2 * idx;
    double re = (double)p[0], im = (double)p[1];
    return re * re + im * im;
  }
  if (dtype == LOF_REF_CF32) {
    const float *p = (const float *)in + 2 * idx;
    if (!isfinite(p[0]) || !isfinite(p[1])) {
      *bad = 1;
      return 0.0;
    }
    double re = (double)p[0], im = (double)p[1];
    return re * re + im * im;
  }
  float f = ((const float *)in)[idx];
  if (!isfinite(f)) {
    *bad = 1;
    return 0.0;
  }
  return (double)f;
}

static void write_out(int dtype, const void *in, int64_t iidx, void *out, int64_t oidx,
                      int flagged) {
  if (dtype == LOF_REF_CI8) {
    const int8_t *s = (const int8_t *)in + 2 * iidx;
    int8_t *d = (int8_t *)out + 2 * oidx;
    d[0] = flagged ? 0 : s[0];
    d[1] = flagged ? 0 : s[1];
  } else if (dtype == LOF_REF_CI16) {
    const int16_t *s = (const int16_t *)in + 2 * iidx;
    int16_t *d = (int16_t *)out + 2 * oidx;
    d[0] = flagged ? 0 : s[0];
    d[1] = flagged ? 0 : s[1];
  } else if (dtype == LOF_REF_CF32) {
    const float *s = (const float *)in + 2 * iidx;
    float *d = (float *)out + 2 * oidx;
    d[0] = flagged ? 0.0f : s[0];
    d[1] = flagged ? 0.0f : s[1];
  } else {
    float v = ((const float *)in)[iidx];
    ((float *)out)[oidx] = flagged ? 0.0f : v;
  }
}

/* Section 4.1: mean and population stddev of the stored per-channel means,
 * summed oldest -> newest; threshold = mean + k * stddev. */
static double history_threshold(const double *ring, int count, double k) {
  double s = 0.0;
  for (int i = 0; i < count; ++i) s = s + ring[i];
  double mu = s / (double)count;
  double q = 0.0;
  for (int i = 0; i < count; ++i) {
    double d = ring[i] - mu;
    q = q + d * d;
  }
  double sd = sqrt(q / (double)count);
  return mu + k * sd;
}

int lof_ref_flag_unit(const lof_ref_params *pr, int dtype, const void *in, int C, int T,
                      int64_t in_stride, void *out, int64_t out_stride, uint8_t *mask,
                      int64_t mask_stride, const double *ring, const int32_t *ring_count,
                      double *pending, uint8_t *has_pending, lof_ref_stats *stats) {
  if (!pr || !in || C < 0 || T < 0) return -1;
  if (dtype != LOF_REF_CI8 && dtype != LOF_REF_CI16 && dtype != LOF_REF_F32 &&
      dtype != LOF_REF_CF32)
    return -1;
  const int is_int = dtype == LOF_REF_CI8 || dtype == LOF_REF_CI16;
  const int64_t N = (int64_t)C * T;
  lof_ref_stats st;
  memset(&st, 0, sizeof st);

  /* power and entry flags */
  double *P = (double *)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
  uint8_t *F = (uint8_t *)calloc((size_t)(N > 0 ? N : 1), 1);
  for (int c = 0; c < C; ++c)
    for (int t = 0; t < T; ++t) {
      int bad;
      P[(int64_t)c * T + t] = sample_power(dtype, in, (int64_t)c * in_stride + t, &bad);
      F[(int64_t)c * T + t] = (uint8_t)bad;
    }

  /* Section 3: the spectrum for frequency flagging sums each channel over all
   * of its time samples. */
  uint8_t *Fc = (uint8_t *)calloc((size_t)(C > 0 ? C : 1), 1);
  double *S = (double *)malloc((size_t)(C > 0 ? C : 1) * sizeof(double));
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (int t = 0; t < T; ++t)
      if (!F[(int64_t)c * T + t]) s = s + P[(int64_t)c * T + t];
    S[c] = s;
  }
  if (pr->time_mode != 2) { /* the 2-D mode has no separate frequency pass */
    if (C > 0) st.sigma_f = lof_ref_sigma(pr, S, C, is_int, &st.median_f);
    if (pr->enable_freq && C > 0) lof_ref_sum_threshold(pr, S, C, st.median_f, st.sigma_f, Fc);
    for (int c = 0; c < C; ++c) st.n_chan_freq += Fc[c];
  }

  if (pr->time_mode == 2) {
    /* Two-dimensional SumThreshold on integration cells. */
    const int Fi = pr->integ_chan, Ti = pr->integ_time;
    const int Cg = (Fi > 0 && C % Fi == 0) ? C / Fi : -1;
    const int Tg = (Ti > 0 && T % Ti == 0) ? T / Ti : -1;
    if (Cg < 0 || Tg < 0) {
      free(P);
      free(F);
      free(Fc);
      free(S);
      return -1;
    }
    const int64_t NG = (int64_t)Cg * Tg;
    double *V = (double *)calloc((size_t)(NG > 0 ? NG : 1), sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)(NG > 0 ? NG : 1), sizeof(int64_t));
    uint8_t *Fg = (uint8_t *)calloc((size_t)(NG > 0 ? NG : 1), 1);
    /* a cell's value: the sum of its unflagged powers; a cell with none is flagged */
    for (int c = 0; c < C; ++c)
      for (int t = 0; t < T; ++t)
        if (!F[(int64_t)c * T + t]) {
          const int64_t g = (int64_t)(c / Fi) * Tg + t / Ti;
          V[g] = V[g] + P[(int64_t)c * T + t];
          cnt[g]++;
        }
    int64_t nu = 0;
    double *U = (double *)malloc((size_t)(NG > 0 ? NG : 1) * sizeof(double));
    for (int64_t g = 0; g < NG; ++g) {
      if (cnt[g] == 0)
        Fg[g] = 1;
      else
        U[nu++] = V[g];
    }
    if (nu > 0) st.sigma_t = lof_ref_sigma(pr, U, nu, is_int, &st.median_t);
    if (nu > 0 && st.sigma_t > 0.0) {
      for (int k = 0;; ++k) {
        const int64_t I = (int64_t)1 << k;
        if (I > pr->max_window || (I > Tg && I > Cg)) break;
        const double thr = lof_ref_threshold(pr, st.median_t, st.sigma_t, k);
        if (pr->enable_time && I <= Tg) /* along time, every row of cells */
          for (int g = 0; g < Cg; ++g) st_one_size(V + (int64_t)g * Tg, Tg, 1, I, thr, Fg + (int64_t)g * Tg);
        if (pr->enable_freq && I <= Cg) /* then along frequency, every column */
          for (int h = 0; h < Tg; ++h) st_one_size(V + h, Cg, Tg, I, thr, Fg + h);
      }
    }
    for (int c = 0; c < C; ++c)
      for (int t = 0; t < T; ++t)
        if (Fg[(int64_t)(c / Fi) * Tg + t / Ti] && !F[(int64_t)c * T + t]) {
          F[(int64_t)c * T + t] = 1;
          st.n_flag_time++;
        }
    free(U);
    free(V);
    free(cnt);
    free(Fg);
  } else if (pr->time_mode == 1) {
    /* Section 3: for time-domain flagging the frequency axis is summed away
     * entirely, over the channels the frequency pass kept. */
    double *G = (double *)malloc((size_t)(T > 0 ? T : 1) * sizeof(double));
    uint8_t *Ft = (uint8_t *)calloc((size_t)(T > 0 ? T : 1), 1);
    int nkept = 0;
    for (int c = 0; c < C; ++c) nkept += !Fc[c];
    for (int t = 0; t < T; ++t) {
      double g = 0.0;
      for (int c = 0; c < C; ++c)
        if (!Fc[c] && !F[(int64_t)c * T + t]) g = g + P[(int64_t)c * T + t];
      G[t] = g;
    }
    if (T > 0 && nkept > 0) {
      st.sigma_t = lof_ref_sigma(pr, G, T, is_int, &st.median_t);
      if (pr->enable_time) lof_ref_sum_threshold(pr, G, T, st.median_t, st.sigma_t, Ft);
    }
    for (int c = 0; c < C; ++c) {
      if (Fc[c]) continue;
      for (int t = 0; t < T; ++t)
        if (Ft[t] && !F[(int64_t)c * T + t]) {
          F[(int64_t)c * T + t] = 1;
          st.n_flag_time++;
        }
    }
    free(G);
    free(Ft);
  } else {
    /* Section 4 / 4.2: statistics for the time pass pool the samples of the
     * channels left unflagged by the frequency pass. */
    int64_t nu = 0;
    double *U = (double *)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    for (int c = 0; c < C; ++c) {
      if (Fc[c]) continue;
      for (int t = 0; t < T; ++t)
        if (!F[(int64_t)c * T + t]) U[nu++] = P[(int64_t)c * T + t];
    }
    if (nu > 0) st.sigma_t = lof_ref_sigma(pr, U, nu, is_int, &st.median_t);
    free(U);

    /* Section 2.1 in the time direction, one channel at a time, with the
     * pooled statistics or (per-channel scope) the channel's own. */
    uint8_t *entry = (uint8_t *)malloc((size_t)(T > 0 ? T : 1));
    double *V = (double *)malloc((size_t)(T > 0 ? T : 1) * sizeof(double));
    for (int c = 0; c < C; ++c) {
      if (Fc[c] || !pr->enable_time || nu == 0) continue;
      uint8_t *row = F + (int64_t)c * T;
      double m = st.median_t, sg = st.sigma_t;
      if (pr->stats_scope == 1) {
        int64_t nv = 0;
        for (int t = 0; t < T; ++t)
          if (!row[t]) V[nv++] = P[(int64_t)c * T + t];
        if (nv == 0) continue;
        sg = lof_ref_sigma(pr, V, nv, is_int, &m);
      }
      memcpy(entry, row, (size_t)T);
      lof_ref_sum_threshold(pr, P + (int64_t)c * T, T, m, sg, row);
      for (int t = 0; t < T; ++t) st.n_flag_time += (row[t] && !entry[t]);
    }
    free(V);
    free(entry);
    if (pr->stats_scope == 1) st.median_t = st.sigma_t = 0.0;
  }

  /* Section 4.1: the history flagger, per channel. */
  uint8_t *Fh = (uint8_t *)calloc((size_t)(C > 0 ? C : 1), 1);
  for (int c = 0; c < C; ++c) {
    if (has_pending) has_pending[c] = 0;
    if (Fc[c]) continue;
    double s = 0.0;
    int64_t n = 0;
    for (int t = 0; t < T; ++t)
      if (!F[(int64_t)c * T + t]) {
        s = s + P[(int64_t)c * T + t];
        n++;
      }
    if (n == 0) continue;
    double cur = s / (double)n;
    double staged = cur;
    if (pr->enable_history && ring && ring_count && ring_count[c] >= pr->history_min &&
        ring_count[c] > 0) {
      double thr = history_threshold(ring + (int64_t)c * pr->history_len, ring_count[c],
                                     pr->history_k);
      if (!(cur < thr)) {
        staged = thr;
        Fh[c] = 1;
      }
    }
    if (pending) pending[c] = staged;
    if (has_pending) has_pending[c] = 1;
    st.n_chan_hist += Fh[c];
  }

  /* The final mask; Section 2.2: the optional SIR operator extends its flagged
   * ranges, along time on every channel, then along frequency. */
  uint8_t *Mk = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
  for (int c = 0; c < C; ++c)
    for (int t = 0; t < T; ++t)
      Mk[(int64_t)c * T + t] = (uint8_t)(Fc[c] || Fh[c] || F[(int64_t)c * T + t]);
  if (pr->sir_percent > 0) {
    for (int c = 0; c < C; ++c) lof_ref_sir(Mk + (int64_t)c * T, T, 1, pr->sir_percent, Mk + (int64_t)c * T, 1);
    for (int t = 0; t < T; ++t) lof_ref_sir(Mk + t, C, T, pr->sir_percent, Mk + t, T);
  }

  /* Apply: flagged data is removed (zeroed) and the mask is reported. */
  for (int c = 0; c < C; ++c)
    for (int t = 0; t < T; ++t) {
      int f = Mk[(int64_t)c * T + t];
      st.n_flag_total += f;
      if (mask) mask[(int64_t)c * mask_stride + t] = (uint8_t)f;
      if (out) write_out(dtype, in, (int64_t)c * in_stride + t, out, (int64_t)c * out_stride + t, f);
    }

  if (stats) *stats = st;
  free(Mk);
  free(P);
  free(F);
  free(Fc);
  free(S);
  free(Fh);
  return 0;
}

void lof_ref_history_commit(const lof_ref_params *pr, int C, double *ring, int32_t *ring_count,
                            const double *pending, const uint8_t *has_pending) {
  const int H = pr->history_len;
  for (int c = 0; c < C; ++c) {
    if (!has_pending[c]) continue;
    double *r = ring + (int64_t)c * H;
    if (ring_count[c] < H) {
      r[ring_count[c]] = pending[c];
      ring_count[c] += 1;
    } else {
      for (int i = 1; i < H; ++i) r[i - 1] = r[i];
      r[H - 1] = pending[c];
    }
  }
}
