// lof_integ.cu -- exact-statistics unit kernel for integer voltage units, one
// CTA per unit, in four modes:
//   0  the integrated time mode (lof_params.time_mode = 1): Section 3 sums
//      the time axis away for frequency flagging and the frequency axis away
//      for time-domain flagging (steps a1-a8 below);
//   1  the per-channel statistics scope (stats_scope = 1): each kept channel's
//      time pass with the median and sigma of its own powers;
//   2  the pooled per-channel time pass with statistics selected exactly from
//      the unit in global memory (the winsorized estimator, which the
//      histogram statistics of the block kernel do not provide);
//   3  the two-dimensional mode (time_mode = 2): SumThreshold on cells of
//      summed powers, along time and then along frequency for each window.
// Every mode supports the three sigma estimators (MAD, stddev, winsorized).
// The integrated mode, step by step:
//   a1  powers re^2 + im^2 (exact integers)
//   a2  row sums S[c] and the column series over all channels, one pass
//   a3  median and sigma of S (Section 4.2; bitonic sort, exact)
//   a4  SumThreshold over S (Section 2.1) -> channel flags
//   a5  the series G[t] over the kept channels (flagged rows subtracted) and
//       its median and sigma (radix selection on 64-bit keys, exact)
//   a6  SumThreshold over G -> time flags, applied to every kept channel
//   a7  history test per channel (Section 4.1; binary64 mean of the unflagged
//       samples, exact integer sum)
//   a8  mask and masked data
// Sums of integer powers are exact in binary64 here (G <= 2048 * 2^31 and
// window sums <= 2^53; the kernel adds them in 64-bit integers and converts
// once), so the decisions equal those of the binary64 oracle.
#include <cstdint>

#include <cuda_runtime.h>

#include "lof_internal.h"

namespace lofk {
namespace {

constexpr int kNtI = 512, kNwI = kNtI / 32;
constexpr int kIntegMaxT = 16384;
constexpr unsigned kFullI = 0xFFFFFFFFu;
constexpr double kMadToSigma = 1.482602218505602;
// 1/sqrt(c): c = 0.8 - 2 z phi(z) + 0.2 z^2 = 0.6786545589528744 is the
// variance of a standard normal clamped at its 10% / 90% quantiles +-z,
// z = 1.2815515655446004, so the clamped stddev times this estimates sigma.
constexpr double kWinsorToSigma = 1.2138796046717422;
constexpr int kEstStd = 1, kEstWinsor = 2;  // KParams::sigma_std holds the estimator

// shared memory layout (bytes)
constexpr int kOffS = 0;                                  // u64 S[kMaxChan]
constexpr int kOffSrt = kOffS + 8 * kMaxChan;             // u64 sort buffer [kMaxChan]
constexpr int kOffG = kOffSrt + 8 * kMaxChan;             // u64 G[kIntegMaxT]
constexpr int kOffHist = kOffG + 8 * kIntegMaxT;          // u32 [2][2048] (two ranks)
constexpr int kOffFc = kOffHist + 4 * 2 * 2048;           // u8 [kMaxChan]
constexpr int kOffFcn = kOffFc + kMaxChan;                // u8 [kMaxChan]
constexpr int kOffFt = kOffFcn + kMaxChan;                // u8 [kIntegMaxT]
constexpr int kOffFn = kOffFt + kIntegMaxT;               // u8 [kIntegMaxT]
constexpr int kIntegSmem = kOffFn + kIntegMaxT;
static_assert(kIntegSmem <= 227 * 1024 - 1024, "one CTA per SM");

struct IntegShared {
  long long kw[65];      // integer window thresholds of one window size (I <= 64)
  uint32_t ctot[128];    // chunk totals of the selection histograms (32 bins a chunk)
  double median_f, sigma_f, median_t, sigma_t;
  unsigned long long cnt_time, cnt_total, cnt_hist;
  unsigned long long pref[2];
  long long rank[2];
  int nrank, nkept, nfc;
  unsigned long long s1lo[kNwI], s1hi[kNwI], s2lo[kNwI], s2hi[kNwI];
  unsigned long long rs[kNwI], orw[kNwI];
  int rn[kNwI];
  int fh;
};

template <int DT>
__device__ __forceinline__ uint32_t ipow(const uint8_t* row, int t) {
  if constexpr (DT == LOF_CI16) {
    const uint32_t w = reinterpret_cast<const uint32_t*>(row)[t];
    const int re = static_cast<int16_t>(w & 0xFFFFu), im = static_cast<int16_t>(w >> 16);
    return static_cast<uint32_t>(re * re) + static_cast<uint32_t>(im * im);
  } else {
    const uint32_t h = reinterpret_cast<const uint16_t*>(row)[t];
    const int re = static_cast<int8_t>(h & 0xFFu), im = static_cast<int8_t>(h >> 8);
    return static_cast<uint32_t>(re * re + im * im);
  }
}

// Sum of the powers of the samples of one 16-byte vector (4 ci16 or 8 ci8).
template <int DT>
__device__ __forceinline__ unsigned long long vec_power_sum(const uint4& v) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  unsigned long long s = 0ull;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if constexpr (DT == LOF_CI16) {
      const int re = static_cast<int16_t>(w[j] & 0xFFFFu), im = static_cast<int16_t>(w[j] >> 16);
      s += static_cast<unsigned long long>(static_cast<uint32_t>(re * re) + static_cast<uint32_t>(im * im));
    } else {
      uint32_t p = 0u;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t x = (w[j] >> (16 * h)) & 0xFFFFu;
        const int re = static_cast<int8_t>(x & 0xFFu), im = static_cast<int8_t>(x >> 8);
        p += static_cast<uint32_t>(re * re + im * im);
      }
      s += p;
    }
  }
  return s;
}

// Calls fn(t, power) for every sample of a row, lanes in parallel: 16-byte
// vector loads (four per lane issued before any is used) where the row is
// 16-byte aligned, plain loads for the rest.
template <int DT, class FN>
__device__ __forceinline__ void row_powers(const uint8_t* row, int T, bool vec, FN fn) {
  constexpr int VS = DT == LOF_CI16 ? 4 : 8, U = 4, STEP = 32 * VS * U;
  const int lane = threadIdx.x & 31;
  int t0 = 0;
  if (vec) {
    for (; t0 + STEP <= T; t0 += STEP) {
      uint4 v[U];
#pragma unroll
      for (int k = 0; k < U; ++k)
        v[k] = __ldg(reinterpret_cast<const uint4*>(row) + (t0 + k * 32 * VS) / VS + lane);
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const uint32_t w[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
        for (int j = 0; j < VS; ++j) {
          const int t = t0 + k * 32 * VS + lane * VS + j;
          uint32_t p;
          if constexpr (DT == LOF_CI16) {
            const int re = static_cast<int16_t>(w[j] & 0xFFFFu), im = static_cast<int16_t>(w[j] >> 16);
            p = static_cast<uint32_t>(re * re) + static_cast<uint32_t>(im * im);
          } else {
            const uint32_t h = (w[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
            const int re = static_cast<int8_t>(h & 0xFFu), im = static_cast<int8_t>(h >> 8);
            p = static_cast<uint32_t>(re * re + im * im);
          }
          fn(t, p);
        }
      }
    }
  }
  for (int t = t0 + lane; t < T; t += 32) fn(t, ipow<DT>(row, t));
}

__device__ __forceinline__ double u128_to_double_i(unsigned __int128 m) {
  const unsigned long long hi = static_cast<unsigned long long>(m >> 64);
  const unsigned long long lo = static_cast<unsigned long long>(m);
  if (hi == 0) return __ull2double_rn(lo);
  const int s = __clzll(static_cast<long long>(hi));
  unsigned long long top = s ? ((hi << s) | (lo >> (64 - s))) : hi;
  const unsigned long long rest = s ? (lo << s) : lo;
  top |= (rest != 0ull) ? 1ull : 0ull;
  return ldexp(__ull2double_rn(top), 64 - s);
}

// Population stddev of n integers from exact moments (the oracle's integer
// form): sqrt((n * S2 - S1^2) / n^2).  Whole CTA; v(i) gives value i.
template <class V>
__device__ double exact_std(long long n, V v, IntegShared& f) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned __int128 s1 = 0, s2 = 0;
  for (long long i = tid; i < n; i += kNtI) {
    const unsigned __int128 x = v(i);
    s1 += x;
    s2 += x * x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(kFullI, static_cast<unsigned long long>(s1), o);
    const unsigned long long b = __shfl_xor_sync(kFullI, static_cast<unsigned long long>(s1 >> 64), o);
    const unsigned long long c = __shfl_xor_sync(kFullI, static_cast<unsigned long long>(s2), o);
    const unsigned long long d = __shfl_xor_sync(kFullI, static_cast<unsigned long long>(s2 >> 64), o);
    s1 += (static_cast<unsigned __int128>(b) << 64) | a;
    s2 += (static_cast<unsigned __int128>(d) << 64) | c;
  }
  if (lane == 0) {
    f.s1lo[warp] = static_cast<unsigned long long>(s1);
    f.s1hi[warp] = static_cast<unsigned long long>(s1 >> 64);
    f.s2lo[warp] = static_cast<unsigned long long>(s2);
    f.s2hi[warp] = static_cast<unsigned long long>(s2 >> 64);
  }
  __syncthreads();
  unsigned __int128 t1 = 0, t2 = 0;
  for (int w = 0; w < kNwI; ++w) {
    t1 += (static_cast<unsigned __int128>(f.s1hi[w]) << 64) | f.s1lo[w];
    t2 += (static_cast<unsigned __int128>(f.s2hi[w]) << 64) | f.s2lo[w];
  }
  __syncthreads();
  if (n <= 0) return 0.0;
  const unsigned __int128 M = static_cast<unsigned __int128>(n) * t2 - t1 * t1;
  const double nn = __dmul_rn(static_cast<double>(n), static_cast<double>(n));
  return __dsqrt_rn(__ddiv_rn(u128_to_double_i(M), nn));
}

// Bitonic sort of n (power of two) u64 keys, ascending (whole CTA).
__device__ void sort_u64(unsigned long long* a, int n) {
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += kNtI) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long x = a[i], y = a[l];
          if (((i & k) == 0) == (x > y)) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
}

// Order statistics r0 <= r1 of n u64 keys key(i) (whole CTA): radix selection
// with digits of 11 bits (the last of 9), one histogram per open rank.  Every
// key is below 2^bits: the digits above are all zero and their passes, which
// would leave the prefix at 0 and the ranks unchanged, are skipped.
template <class K>
__device__ void select2(long long n, long long r0, long long r1, K key, uint32_t* hist, IntegShared& f,
                        unsigned long long* k0, unsigned long long* k1, int bits = 64) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    f.pref[0] = f.pref[1] = 0ull;
    f.rank[0] = r0;
    f.rank[1] = r1;
    f.nrank = r0 == r1 ? 1 : 2;
  }
  __syncthreads();
  int first = 0;
  while (first < 5 && 53 - 11 * first >= bits) ++first;
  for (int pass = first; pass < 6; ++pass) {  // bits 63..53, 52..42, 41..31, 30..20, 19..9, 8..0
    const int nb = pass < 5 ? 11 : 9;
    const int sh = pass < 5 ? 53 - 11 * pass : 0;
    const int hs = sh + nb;
    for (int i = tid; i < 2 * 2048; i += kNtI) hist[i] = 0u;
    __syncthreads();
    const unsigned long long p0 = f.pref[0], p1 = f.pref[1];
    const bool two = f.nrank == 2, same = !two || p0 == p1;
    for (long long i = tid; i < n; i += kNtI) {
      const unsigned long long x = key(i);
      const unsigned long long hi = hs >= 64 ? 0ull : (x >> hs);
      const uint32_t dig = static_cast<uint32_t>((x >> sh) & ((1ull << nb) - 1ull));
      if (hi == p0) atomicAdd(&hist[dig], 1u);
      if (!same && hi == p1) atomicAdd(&hist[2048 + dig], 1u);
    }
    __syncthreads();
    // the histograms' chunk totals (32 bins a chunk), one warp a chunk
    const int nch = (1 << nb) / 32, nh = same ? 1 : 2;
    for (int c = warp; c < nh * nch; c += kNwI) {
      uint32_t x = hist[(c / nch) * 2048 + (c % nch) * 32 + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFullI, x, o);
      if (lane == 0) f.ctot[c] = x;
    }
    __syncthreads();
    if (warp < f.nrank) {
      const uint32_t* h = hist + (same ? 0 : 2048 * warp);
      const uint32_t* ct = f.ctot + (same ? 0 : nch * warp);
      long long rk = f.rank[warp], base = 0;
      uint32_t digit = 0;
      // the rank's chunk from the chunk totals, then its bin inside the chunk
      auto find = [&](const uint32_t* cnts, int n, int& at) {
        for (int b0 = 0; b0 < n; b0 += 32) {
          const uint32_t cnt = b0 + lane < n ? cnts[b0 + lane] : 0u;
          uint32_t incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullI, incl, o);
            if (lane >= o) incl += y;
          }
          const uint32_t tot = __shfl_sync(kFullI, incl, 31);
          if (rk < base + tot) {
            const unsigned hit = __ballot_sync(kFullI, rk < base + static_cast<long long>(incl));
            const int l = __ffs(hit) - 1;
            at = b0 + l;
            rk -= base + __shfl_sync(kFullI, incl - cnt, l);
            base = 0;
            return true;
          }
          base += tot;
        }
        return false;
      };
      int chunk = 0, bin = 0;
      if (find(ct, nch, chunk) && find(h + 32 * chunk, 32, bin)) digit = static_cast<uint32_t>(32 * chunk + bin);
      if (lane == 0) {
        f.pref[warp] = (f.pref[warp] << nb) | digit;
        f.rank[warp] = rk;
      }
    }
    __syncthreads();
    if (tid == 0 && f.nrank == 1) {
      f.pref[1] = f.pref[0];
      f.rank[1] = f.rank[0];
    }
    __syncthreads();
  }
  *k0 = f.pref[0];
  *k1 = f.pref[1];
}

// Bit length of the largest of n u64 values v(i) (whole CTA).
template <class V>
__device__ int key_bits(long long n, V v, IntegShared& f) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long o = 0;
  for (long long i = tid; i < n; i += kNtI) o |= v(i);
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) o |= __shfl_xor_sync(kFullI, o, k);
  if (lane == 0) f.orw[warp] = o;
  __syncthreads();
  unsigned long long a = 0;
  for (int w = 0; w < kNwI; ++w) a |= f.orw[w];
  __syncthreads();
  return a ? 64 - __clzll(static_cast<long long>(a)) : 0;
}

// Winsorized sigma of n u64 values v(i) given the order statistics lo = v_(k)
// and hi = v_(n-1-k), k = n / 10: the population stddev of the values clamped
// to [lo, hi] times kWinsorToSigma (the plain stddev when that is 0).
template <class V>
__device__ double winsor_sigma(long long n, V v, unsigned long long lo, unsigned long long hi, IntegShared& f) {
  const double sw = exact_std(n, [&](long long i) {
    const unsigned long long x = v(i);
    return x < lo ? lo : (x > hi ? hi : x);
  }, f);
  return sw > 0.0 ? __dmul_rn(kWinsorToSigma, sw) : exact_std(n, v, f);
}

// Section 4.2 median and sigma of n u64 values v(i), exact: the median as
// m2 / 2 with m2 = the sum of the two middle values (twice the middle one for
// odd n); the MAD from the keys |2 v - m2| = 2 |v - median|; the winsorized
// sigma from the order statistics n / 10 and n - 1 - n / 10.
template <class V>
__device__ void stats_u64(const KParams& kp, long long n, V v, uint32_t* hist, IntegShared& f,
                          double* med, double* sig) {
  const int bits = key_bits(n, v, f);
  const long long ra = (n & 1) ? n / 2 : n / 2 - 1, rb = n / 2;
  unsigned long long a, b;
  select2(n, ra, rb, v, hist, f, &a, &b, bits);
  const unsigned long long m2 = a + b;
  *med = __dmul_rn(static_cast<double>(m2), 0.5);
  if (kp.sigma_std == kEstStd) {
    *sig = exact_std(n, v, f);
    return;
  }
  if (kp.sigma_std == kEstWinsor) {
    const long long k = n / 10;
    unsigned long long lo, hi;
    select2(n, k, n - 1 - k, v, hist, f, &lo, &hi, bits);
    *sig = winsor_sigma(n, v, lo, hi, f);
    return;
  }
  auto dev = [&](long long i) {
    const unsigned long long x2 = 2ull * v(i);
    return x2 >= m2 ? x2 - m2 : m2 - x2;
  };
  unsigned long long da, db;
  select2(n, ra, rb, dev, hist, f, &da, &db, bits + 1);
  const double mad = __dmul_rn(static_cast<double>(da + db), 0.25);
  *sig = mad > 0.0 ? __dmul_rn(kMadToSigma, mad) : exact_std(n, v, f);
}

// threshold_I = median + sigma * factor_I * sensitivity (Section 2.1)
__device__ __forceinline__ double thr_i(const KParams& kp, double m, double s, int k) {
  return __dadd_rn(m, __dmul_rn(__dmul_rn(s, kp.factor[k]), kp.sensitivity));
}

// Section 2.1 SumThreshold over v[0..L) (whole CTA), flags in / out in fl,
// next as scratch: a window fires when the sum of its unflagged values exceeds
// (I - n) * thr_I.  The values are integers and every window sum is at most
// 2^51 (64 spectrum sums of at most 2^14 powers of at most 2^31, or 64 series
// values of at most 2^11 such powers), so the sum is accumulated in 64-bit
// integers and converted once: the same number as a binary64 sum, whose every
// partial sum is exact, at a fraction of the binary64 operations.
template <class V>
__device__ void st_1d(const KParams& kp, V v, int L, double med, double sig, uint8_t* fl,
                      uint8_t* next, long long* Kw) {
  if (!(sig > 0.0) || L <= 0) return;
  for (int k = 0;; ++k) {
    const int I = 1 << k;
    if (I > (1 << kp.max_log_window) || I > L) break;
    const double thr = thr_i(kp, med, sig, k);
    for (int i = threadIdx.x; i < L; i += kNtI) next[i] = fl[i];
    // the binary64 test su > (I - n) * thr as the integer one su > Kw[n]
    // (su is exact and at most 2^51; Kw[n] = floor of the product, -1 below 0)
    for (int n = threadIdx.x; n <= I; n += kNtI) {
      const double P = __dmul_rn(static_cast<double>(I - n), thr);
      Kw[n] = P < 0.0 ? -1ll : (P >= 9.0e18 ? 0x7FFFFFFFFFFFFFFFll : __double2ll_rd(P));
    }
    __syncthreads();
    // each thread slides over its run of window starts (each value enters and
    // leaves its window sum once) against the flags on entry
    const int nw = L - I + 1, per = (nw + kNtI - 1) / kNtI;
    const int t0 = threadIdx.x * per, t1 = min(nw, t0 + per);
    if (t0 < t1) {
      unsigned long long su = 0ull;
      int nf = 0, done = 0;
      for (int j = t0; j < t0 + I - 1; ++j) {
        if (fl[j]) ++nf;
        else su += v(j);
      }
      for (int t = t0; t < t1; ++t) {
        const int e = t + I - 1;
        if (fl[e]) ++nf;
        else su += v(e);
        if (static_cast<long long>(su) > Kw[nf]) {
          for (int j = max(t, done); j < t + I; ++j) next[j] = 1;
          done = t + I;
        }
        if (fl[t]) --nf;
        else su -= v(t);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L; i += kNtI) fl[i] = next[i];
    __syncthreads();
  }
}

// Section 4.1 history test of one channel (one thread): cur = the mean of its
// n unflagged powers (sum s, exact); once the ring holds history_min means the
// channel is flagged unless cur is below the cached mean + k * stddev.  The
// value the commit will append (cur, or the threshold when flagged) is staged;
// a channel with no unflagged sample stages nothing.  Returns the flag.
__device__ bool stage_history(const KParams& kp, long long h, unsigned long long s, int n) {
  bool fh = false;
  if (n > 0) {
    const double cur = __ddiv_rn(static_cast<double>(s), static_cast<double>(n));
    double staged = cur;
    if (kp.enable_history && h >= 0) {
      const int cnt = kp.hist.count[h];
      if (cnt >= kp.history_min && cnt > 0) {
        const double thr = kp.hist.thr[h];
        if (!(cur < thr)) {
          fh = true;
          staged = thr;
        }
      }
    }
    if (h >= 0) {
      kp.hist.pend[h] = staged;
      kp.hist.pend_flag[h] = 1;
      kp.hist.pend_seq[h] = kp.block_seq;
    }
  } else if (h >= 0) {
    kp.hist.pend_flag[h] = 0;
  }
  return fh;
}

// a3, a4 for a unit whose row sums are in S: exact median and sigma of the
// spectrum (bitonic sort of the C sums, deviations as |2x - m2|) and the
// frequency SumThreshold -> Fc (whole CTA).
__device__ void freq_stage(const KParams& kp, unsigned long long* S, unsigned long long* srt, int C,
                           uint8_t* Fc, uint8_t* Fcn, IntegShared& f) {
  const int tid = threadIdx.x;
  {
    int n2 = 1;
    while (n2 < C) n2 <<= 1;
    for (int i = tid; i < n2; i += kNtI) srt[i] = i < C ? S[i] : ~0ull;
    __syncthreads();
    sort_u64(srt, n2);
    const long long ra = (C & 1) ? C / 2 : C / 2 - 1, rb = C / 2;
    const unsigned long long m2 = srt[ra] + srt[rb];
    const double med = __dmul_rn(static_cast<double>(m2), 0.5);
    double sig;
    if (kp.sigma_std == kEstStd) {
      sig = exact_std(C, [&](long long i) { return S[i]; }, f);
    } else if (kp.sigma_std == kEstWinsor) {
      const unsigned long long lo = srt[C / 10], hi = srt[C - 1 - C / 10];
      sig = winsor_sigma(C, [&](long long i) { return S[i]; }, lo, hi, f);
    } else {
      __syncthreads();
      for (int i = tid; i < n2; i += kNtI) {
        if (i < C) {
          const unsigned long long x2 = 2ull * S[i];
          srt[i] = x2 >= m2 ? x2 - m2 : m2 - x2;
        } else {
          srt[i] = ~0ull;
        }
      }
      __syncthreads();
      sort_u64(srt, n2);
      const double mad = __dmul_rn(static_cast<double>(srt[ra] + srt[rb]), 0.25);
      sig = mad > 0.0 ? __dmul_rn(kMadToSigma, mad) : exact_std(C, [&](long long i) { return S[i]; }, f);
    }
    if (tid == 0) {
      f.median_f = med;
      f.sigma_f = sig;
    }
    __syncthreads();
  }
  // a4: frequency SumThreshold
  if (kp.enable_freq) st_1d(kp, [&](int i) { return S[i]; }, C, f.median_f, f.sigma_f, Fc, Fcn, f.kw);
  __syncthreads();
}

template <int DT>
__device__ void integ_unit(const KParams& kp, const DevUnit& u, uint8_t* smem, IntegShared& f) {
  constexpr int ES = DT == LOF_CI16 ? 4 : 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int C = u.C, T = u.T;
  unsigned long long* S = reinterpret_cast<unsigned long long*>(smem + kOffS);
  unsigned long long* srt = reinterpret_cast<unsigned long long*>(smem + kOffSrt);
  unsigned long long* G = reinterpret_cast<unsigned long long*>(smem + kOffG);
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + kOffHist);
  uint8_t* Fc = smem + kOffFc;
  uint8_t* Fcn = smem + kOffFcn;
  uint8_t* Ft = smem + kOffFt;
  uint8_t* Fn = smem + kOffFn;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  const bool vin = (u.flags & kUnitInVec) != 0;
  for (int i = tid; i < T; i += kNtI) {
    G[i] = 0ull;
    Ft[i] = 0;
  }
  for (int i = tid; i < C; i += kNtI) Fc[i] = 0;
  if (tid == 0) f.cnt_time = f.cnt_total = f.cnt_hist = 0ull;
  __syncthreads();
  // a1, a2: row sums and the column series over every channel
  for (int c = warp; c < C; c += kNwI) {
    const uint8_t* row = gin + static_cast<int64_t>(c) * u.in_stride * ES;
    unsigned long long s = 0;
    row_powers<DT>(row, T, vin, [&](int t, uint32_t p) {
      s += p;
      atomicAdd(&G[t], static_cast<unsigned long long>(p));
    });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFullI, s, o);
    if (lane == 0) S[c] = s;
  }
  __syncthreads();
  freq_stage(kp, S, srt, C, Fc, Fcn, f);
  // a5: the series over the kept channels and its statistics
  for (int c = warp; c < C; c += kNwI) {
    if (!Fc[c]) continue;
    const uint8_t* row = gin + static_cast<int64_t>(c) * u.in_stride * ES;
    row_powers<DT>(row, T, vin, [&](int t, uint32_t p) { atomicAdd(&G[t], 0ull - static_cast<unsigned long long>(p)); });
  }
  if (tid == 0) {
    int nk = 0;
    for (int c = 0; c < C; ++c) nk += !Fc[c];
    f.nkept = nk;
    f.nfc = C - nk;
  }
  __syncthreads();
  double med_t = 0.0, sig_t = 0.0;
  if (f.nkept > 0) {
    stats_u64(kp, T, [&](long long i) { return G[i]; }, hist, f, &med_t, &sig_t);
    // a6: SumThreshold over the series
    if (kp.enable_time) st_1d(kp, [&](int i) { return G[i]; }, T, med_t, sig_t, Ft, Fn, f.kw);
  }
  __syncthreads();
  // a7, a8: per channel.  A kept row is summed for the history test while its
  // mask and data are written as if the test keeps it (one pass over it); the
  // rare row the test flags is then rewritten whole.
  const bool inplace = (u.flags & kUnitInPlace) != 0;
  const bool vout = vin && (u.flags & kUnitOutVec) && (u.flags & kUnitMaskVec) && !inplace;
  constexpr int VS = ES == 4 ? 4 : 8;
  for (int c = warp; c < C; c += kNwI) {
    const uint8_t* row = gin + static_cast<int64_t>(c) * u.in_stride * ES;
    const long long h = u.hist_slot >= 0 ? u.hist_slot + c : -1;
    uint8_t* mr = u.mask ? u.mask + static_cast<int64_t>(c) * u.mask_stride : nullptr;
    uint8_t* orow = u.out ? static_cast<uint8_t*>(u.out) + static_cast<int64_t>(c) * u.out_stride * ES : nullptr;
    auto put = [&](int t, bool fl) {  // one sample's mask and data
      if (mr) mr[t] = fl ? 1 : 0;
      if (orow) {
        if (ES == 4) {
          if (fl) reinterpret_cast<uint32_t*>(orow)[t] = 0u;
          else if (!inplace) reinterpret_cast<uint32_t*>(orow)[t] = reinterpret_cast<const uint32_t*>(row)[t];
        } else {
          if (fl) reinterpret_cast<uint16_t*>(orow)[t] = 0;
          else if (!inplace) reinterpret_cast<uint16_t*>(orow)[t] = reinterpret_cast<const uint16_t*>(row)[t];
        }
      }
    };
    bool full = Fc[c] != 0;
    if (!full) {
      unsigned long long s = 0;
      int n = 0;
      int tv = 0;
      if (vout && mr && orow) {
        for (; tv + 32 * VS <= T; tv += 32 * VS) {
          const int t = tv + lane * VS;
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + static_cast<size_t>(t) * ES));
          uint32_t w[4] = {v.x, v.y, v.z, v.w}, mb[2] = {0u, 0u};
#pragma unroll
          for (int j = 0; j < VS; ++j) {
            uint32_t pw;
            if constexpr (DT == LOF_CI16) {
              const int re = static_cast<int16_t>(w[j] & 0xFFFFu), im = static_cast<int16_t>(w[j] >> 16);
              pw = static_cast<uint32_t>(re * re) + static_cast<uint32_t>(im * im);
            } else {
              const uint32_t hh = (w[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
              const int re = static_cast<int8_t>(hh & 0xFFu), im = static_cast<int8_t>(hh >> 8);
              pw = static_cast<uint32_t>(re * re + im * im);
            }
            if (Ft[t + j]) {
              if (ES == 4) w[j] = 0u;
              else w[j >> 1] &= (j & 1) ? 0x0000FFFFu : 0xFFFF0000u;
              mb[j >> 2] |= 1u << (8 * (j & 3));
            } else {
              s += pw;
              ++n;
            }
          }
          *reinterpret_cast<uint4*>(orow + static_cast<size_t>(t) * ES) = make_uint4(w[0], w[1], w[2], w[3]);
          if (VS == 4) *reinterpret_cast<uint32_t*>(mr + t) = mb[0];
          else *reinterpret_cast<uint2*>(mr + t) = make_uint2(mb[0], mb[1]);
        }
      }
      for (int t = tv + lane; t < T; t += 32) {
        const bool fl = Ft[t] != 0;
        if (!fl) {
          s += ipow<DT>(row, t);
          ++n;
        }
        put(t, fl);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(kFullI, s, o);
        n += __shfl_xor_sync(kFullI, n, o);
      }
      bool fh = false;
      if (lane == 0) {
        fh = stage_history(kp, h, s, n);
        atomicAdd(&f.cnt_time, static_cast<unsigned long long>(T - n));
        if (fh) atomicAdd(&f.cnt_hist, 1ull);
        atomicAdd(&f.cnt_total, fh ? static_cast<unsigned long long>(T) : static_cast<unsigned long long>(T - n));
      }
      full = __shfl_sync(kFullI, fh ? 1 : 0, 0) != 0;
      __syncwarp();  // the row's first writes, by every lane, before a rewrite
    } else if (lane == 0) {
      if (h >= 0) kp.hist.pend_flag[h] = 0;
      atomicAdd(&f.cnt_total, static_cast<unsigned long long>(T));
    }
    if (full)
      for (int t = lane; t < T; t += 32) put(t, true);
  }
  __syncthreads();
  if (tid == 0 && u.stats) {
    u.stats->median_f = f.median_f;
    u.stats->sigma_f = f.sigma_f;
    u.stats->median_t = med_t;
    u.stats->sigma_t = sig_t;
    u.stats->n_chan_freq = f.nfc;
    u.stats->n_flag_time = static_cast<long long>(f.cnt_time);
    u.stats->n_chan_hist = static_cast<long long>(f.cnt_hist);
    u.stats->n_flag_total = static_cast<long long>(f.cnt_total);
  }
  __syncthreads();
}


// The per-channel time pass (Section 2.1 along time on every kept channel):
// the frequency stage as above; then, with POOLED, one median and sigma over
// every power of the kept channels, selected exactly from the unit in global
// memory, else (the per-channel statistics scope) each kept channel's own;
// then, one kept channel at a time with the whole CTA, SumThreshold along its
// row, the history test and the output.
template <int DT, bool POOLED>
__device__ void chan_unit(const KParams& kp, const DevUnit& u, uint8_t* smem, IntegShared& f) {
  constexpr int ES = DT == LOF_CI16 ? 4 : 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int C = u.C, T = u.T;
  unsigned long long* S = reinterpret_cast<unsigned long long*>(smem + kOffS);
  unsigned long long* srt = reinterpret_cast<unsigned long long*>(smem + kOffSrt);
  unsigned long long* R = reinterpret_cast<unsigned long long*>(smem + kOffG);  // one row's powers
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + kOffHist);
  uint8_t* Fc = smem + kOffFc;
  uint8_t* Fcn = smem + kOffFcn;
  uint8_t* Ft = smem + kOffFt;
  uint8_t* Fn = smem + kOffFn;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  const bool vin = (u.flags & kUnitInVec) != 0;
  const bool inplace = (u.flags & kUnitInPlace) != 0;
  for (int i = tid; i < C; i += kNtI) Fc[i] = 0;
  if (tid == 0) f.cnt_time = f.cnt_total = f.cnt_hist = 0ull;
  __syncthreads();
  for (int c = warp; c < C; c += kNwI) {
    const uint8_t* row = gin + static_cast<int64_t>(c) * u.in_stride * ES;
    unsigned long long sum = 0;
    row_powers<DT>(row, T, vin, [&](int, uint32_t p) { sum += p; });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFullI, sum, o);
    if (lane == 0) S[c] = sum;
  }
  __syncthreads();
  freq_stage(kp, S, srt, C, Fc, Fcn, f);
  double med_p = 0.0, sig_p = 0.0;
  if constexpr (POOLED) {
    // the kept channels' indices, in order, in the (now free) sort buffer
    int* kidx = reinterpret_cast<int*>(srt);
    if (tid == 0) {
      int nk = 0;
      for (int c = 0; c < C; ++c)
        if (!Fc[c]) kidx[nk++] = c;
      f.nkept = nk;
    }
    __syncthreads();
    const long long nu = static_cast<long long>(f.nkept) * T;
    if (nu > 0)
      stats_u64(kp, nu, [&](long long i) {
        const uint32_t ii = static_cast<uint32_t>(i);  // nu <= 2048 * 16384
        const int r = static_cast<int>(ii / static_cast<uint32_t>(T));
        const int t = static_cast<int>(ii - static_cast<uint32_t>(r) * static_cast<uint32_t>(T));
        return static_cast<unsigned long long>(
            ipow<DT>(gin + static_cast<int64_t>(kidx[r]) * u.in_stride * ES, t));
      }, hist, f, &med_p, &sig_p);
    __syncthreads();
  }
  int nfc = 0;
  for (int c = 0; c < C; ++c) {
    const uint8_t* row = gin + static_cast<int64_t>(c) * u.in_stride * ES;
    const long long h = u.hist_slot >= 0 ? u.hist_slot + c : -1;
    uint8_t* mr = u.mask ? u.mask + static_cast<int64_t>(c) * u.mask_stride : nullptr;
    uint8_t* orow = u.out ? static_cast<uint8_t*>(u.out) + static_cast<int64_t>(c) * u.out_stride * ES : nullptr;
    const bool kept = !Fc[c];
    nfc += !kept;
    if (kept) {
      for (int t = tid; t < T; t += kNtI) {
        R[t] = ipow<DT>(row, t);
        Ft[t] = 0;
      }
      __syncthreads();
      double med = med_p, sig = sig_p;
      if constexpr (!POOLED) stats_u64(kp, T, [&](long long i) { return R[i]; }, hist, f, &med, &sig);
      if (kp.enable_time) st_1d(kp, [&](int i) { return R[i]; }, T, med, sig, Ft, Fn, f.kw);
      __syncthreads();
      unsigned long long sum = 0;
      int n = 0;
      for (int t = tid; t < T; t += kNtI)
        if (!Ft[t]) {
          sum += R[t];
          ++n;
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(kFullI, sum, o);
        n += __shfl_xor_sync(kFullI, n, o);
      }
      if (lane == 0) {
        f.rs[warp] = sum;
        f.rn[warp] = n;
      }
      __syncthreads();
      if (tid == 0) {
        unsigned long long st = 0;
        int nt = 0;
        for (int w = 0; w < kNwI; ++w) {
          st += f.rs[w];
          nt += f.rn[w];
        }
        const bool fh = stage_history(kp, h, st, nt);
        f.cnt_time += static_cast<unsigned long long>(T - nt);
        if (fh) f.cnt_hist += 1ull;
        f.cnt_total += fh ? static_cast<unsigned long long>(T) : static_cast<unsigned long long>(T - nt);
        f.fh = fh ? 1 : 0;
      }
      __syncthreads();
    } else if (tid == 0) {
      if (h >= 0) kp.hist.pend_flag[h] = 0;
      f.cnt_total += static_cast<unsigned long long>(T);
    }
    const bool full = !kept || f.fh;
    for (int t = tid; t < T; t += kNtI) {
      const bool fl = full || Ft[t];
      if (mr) mr[t] = fl ? 1 : 0;
      if (orow) {
        if (ES == 4) {
          if (fl) reinterpret_cast<uint32_t*>(orow)[t] = 0u;
          else if (!inplace) reinterpret_cast<uint32_t*>(orow)[t] = reinterpret_cast<const uint32_t*>(row)[t];
        } else {
          if (fl) reinterpret_cast<uint16_t*>(orow)[t] = 0;
          else if (!inplace) reinterpret_cast<uint16_t*>(orow)[t] = reinterpret_cast<const uint16_t*>(row)[t];
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && u.stats) {
    u.stats->median_f = f.median_f;
    u.stats->sigma_f = f.sigma_f;
    u.stats->median_t = med_p;
    u.stats->sigma_t = sig_p;
    u.stats->n_chan_freq = nfc;
    u.stats->n_flag_time = static_cast<long long>(f.cnt_time);
    u.stats->n_chan_hist = static_cast<long long>(f.cnt_hist);
    u.stats->n_flag_total = static_cast<long long>(f.cnt_total);
  }
  __syncthreads();
}


// One window size of Section 2.1 along n_lines lines of L cells of the grid V
// (line r starts at cell r * line_stride, its cells step apart), flags in fl
// and next as scratch (whole CTA): every window is judged against the flags
// on entry and fires when the sum of its unflagged cells exceeds
// (I - n) * thr.  Cell sums are at most 2^16 powers of at most 2^31, so a
// window sum is at most 2^53: exact in 64-bit integers and in binary64, and
// the test is the integer one su > Kw[n], Kw[n] = floor((I - n) * thr) (the
// binary64 product), -1 where that is negative.  One thread per line slides
// the unflagged sum and the flagged count along it (each cell enters and
// leaves once); a fired window at t flags cells t .. t + I - 1, which the
// slide marks as it passes them.
__device__ void st_grid_lines(const unsigned long long* V, uint8_t* fl, uint8_t* next, int NG, int n_lines,
                              int L, int step, int line_stride, int I, double thr, long long* Kw) {
  for (int i = threadIdx.x; i < NG; i += kNtI) next[i] = fl[i];
  for (int n = threadIdx.x; n <= I; n += kNtI) {
    const double P = __dmul_rn(static_cast<double>(I - n), thr);
    Kw[n] = P < 0.0 ? -1ll : (P >= 9.0e18 ? 0x7FFFFFFFFFFFFFFFll : __double2ll_rd(P));
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n_lines; r += kNtI) {
    const int b = r * line_stride;
    unsigned long long su = 0ull;
    int nf = 0;
    for (int j = 0; j < I - 1; ++j) {
      const int i = b + j * step;
      if (fl[i]) ++nf;
      else su += V[i];
    }
    int until = 0;  // cells below it lie in a fired window
    for (int t = 0; t < L; ++t) {
      if (t + I - 1 < L) {
        const int ie = b + (t + I - 1) * step;  // the window at t: cells t .. t + I - 1
        if (fl[ie]) ++nf;
        else su += V[ie];
        if (static_cast<long long>(su) > Kw[nf]) until = t + I;
        const int il = b + t * step;
        if (fl[il]) --nf;
        else su -= V[il];
      }
      if (t < until) next[b + t * step] = 1;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NG; i += kNtI) fl[i] = next[i];
  __syncthreads();
}

// The same test along the rows of cells (the time direction: lines of L
// contiguous cells): one warp per line, each lane sliding over its run of
// window starts, the window sum at its first start summed directly, so the
// lanes of a warp read cells of one row (few shared-memory bank conflicts)
// and all warps of the CTA take lines.
__device__ void st_grid_rows(const unsigned long long* V, uint8_t* fl, uint8_t* next, int NG, int n_lines,
                             int L, int I, double thr, long long* Kw) {
  for (int i = threadIdx.x; i < NG; i += kNtI) next[i] = fl[i];
  for (int n = threadIdx.x; n <= I; n += kNtI) {
    const double P = __dmul_rn(static_cast<double>(I - n), thr);
    Kw[n] = P < 0.0 ? -1ll : (P >= 9.0e18 ? 0x7FFFFFFFFFFFFFFFll : __double2ll_rd(P));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = L - I + 1, per = (nw + 31) / 32;
  for (int r = warp; r < n_lines; r += kNwI) {
    const int b = r * L, t0 = lane * per, t1 = min(nw, t0 + per);
    if (t0 >= t1) continue;
    unsigned long long su = 0ull;
    int nf = 0, done = 0;
    for (int j = t0; j < t0 + I - 1; ++j) {
      if (fl[b + j]) ++nf;
      else su += V[b + j];
    }
    for (int t = t0; t < t1; ++t) {
      const int e = b + t + I - 1;
      if (fl[e]) ++nf;
      else su += V[e];
      if (static_cast<long long>(su) > Kw[nf]) {
        for (int j = max(t, done); j < t + I; ++j) next[b + j] = 1;
        done = t + I;
      }
      if (fl[b + t]) --nf;
      else su -= V[b + t];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NG; i += kNtI) fl[i] = next[i];
  __syncthreads();
}

// The two-dimensional mode (time_mode = 2): powers summed into cells of Fi
// channels x Ti samples (Fi divides C, Ti divides T, at most kIntegMaxT
// cells), one median and sigma over the cells, then for I = 1, 2, 4, ...
// SumThreshold along time on every row of cells and then along frequency on
// every column (enable_time / enable_freq); a flagged cell flags its samples.
// No separate frequency pass; the history test and the output per channel as
// in the other modes.
template <int DT>
__device__ void grid_unit(const KParams& kp, const DevUnit& u, uint8_t* smem, IntegShared& f, int Fi, int Ti) {
  constexpr int ES = DT == LOF_CI16 ? 4 : 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int C = u.C, T = u.T;
  // the host validates the cells; a launch with others reports an error and
  // touches nothing
  if (Fi < 1 || Ti < 1 || C % Fi || T % Ti || static_cast<long long>(C / Fi) * (T / Ti) > kIntegMaxT) {
    if (tid == 0 && atomicCAS(kp.err, 0, kErrInternal) == 0) {
      kp.err_info[0] = 800;
      kp.err_info[1] = static_cast<int>(kp.block_seq);
    }
    return;
  }
  const int Cg = C / Fi, Tg = T / Ti, NG = Cg * Tg;
  unsigned long long* V = reinterpret_cast<unsigned long long*>(smem + kOffG);
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + kOffHist);
  uint8_t* Fg = smem + kOffFt;
  uint8_t* Fn = smem + kOffFn;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  const bool vin = (u.flags & kUnitInVec) != 0;
  const bool inplace = (u.flags & kUnitInPlace) != 0;
  for (int i = tid; i < NG; i += kNtI) {
    V[i] = 0ull;
    Fg[i] = 0;
  }
  if (tid == 0) f.cnt_time = f.cnt_total = f.cnt_hist = 0ull;
  __syncthreads();
  // Rows of at least 32 cells: each lane sums whole cells of the row (cells
  // [lane * gpl, lane * gpl + gpl)) in registers and adds each cell once;
  // rows of fewer cells sample by sample.
  constexpr int VS = DT == LOF_CI16 ? 4 : 8;
  const int gpl = (Tg + 31) / 32;
  const bool chunked = Tg >= 32;
  const bool vcell = vin && Ti % VS == 0;  // 16-byte vectors within every cell
  const int g0 = lane * gpl, g1 = min(Tg, g0 + gpl);
  for (int c = warp; c < C; c += kNwI) {
    const uint8_t* row = gin + static_cast<int64_t>(c) * u.in_stride * ES;
    unsigned long long* vr = V + (c / Fi) * Tg;
    if (chunked && vcell) {
      // the lane's cells are one run of 16-byte vectors: eight loads in flight
      const int vpc = Ti / VS, nvec = (g1 - g0) * vpc;
      const uint4* vb = reinterpret_cast<const uint4*>(row + static_cast<size_t>(g0) * Ti * ES);
      unsigned long long sc = 0ull;
      int kc = 0, g = g0;
      for (int k0 = 0; k0 < nvec; k0 += 8) {
        uint4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (k0 + j < nvec) v[j] = __ldg(vb + k0 + j);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (k0 + j < nvec) {
            sc += vec_power_sum<DT>(v[j]);
            if (++kc == vpc) {
              atomicAdd(&vr[g], sc);
              sc = 0ull;
              kc = 0;
              ++g;
            }
          }
        }
      }
    } else if (chunked) {
      for (int g = g0; g < g1; ++g) {
        unsigned long long sc = 0ull;
        for (int t = g * Ti; t < g * Ti + Ti; ++t) sc += ipow<DT>(row, t);
        atomicAdd(&vr[g], sc);
      }
    } else {
      row_powers<DT>(row, T, vin, [&](int t, uint32_t p) {
        atomicAdd(&vr[t / Ti], static_cast<unsigned long long>(p));
      });
    }
  }
  __syncthreads();
  double med = 0.0, sig = 0.0;
  stats_u64(kp, NG, [&](long long i) { return V[i]; }, hist, f, &med, &sig);
  if (sig > 0.0) {
    for (int k = 0;; ++k) {
      const int I = 1 << k;
      if (I > (1 << kp.max_log_window) || (I > Tg && I > Cg)) break;
      const double thr = thr_i(kp, med, sig, k);
      long long* Kw = reinterpret_cast<long long*>(hist);  // the selection's histogram is free here
      if (kp.enable_time && I <= Tg) st_grid_rows(V, Fg, Fn, NG, Cg, Tg, I, thr, Kw);
      if (kp.enable_freq && I <= Cg) st_grid_lines(V, Fg, Fn, NG, Tg, Cg, Tg, 1, I, thr, Kw);
    }
  }
  // per channel: the history test on the unflagged samples, mask and data
  const bool vout_cell = vcell && (!u.mask || (u.flags & kUnitMaskVec)) &&
                         (!u.out || inplace || (u.flags & kUnitOutVec));
  for (int c = warp; c < C; c += kNwI) {
    const uint8_t* row = gin + static_cast<int64_t>(c) * u.in_stride * ES;
    const uint8_t* fr = Fg + (c / Fi) * Tg;
    const long long h = u.hist_slot >= 0 ? u.hist_slot + c : -1;
    uint8_t* mr = u.mask ? u.mask + static_cast<int64_t>(c) * u.mask_stride : nullptr;
    uint8_t* orow = u.out ? static_cast<uint8_t*>(u.out) + static_cast<int64_t>(c) * u.out_stride * ES : nullptr;
    auto put = [&](int t, bool fl) {
      if (mr) mr[t] = fl ? 1 : 0;
      if (orow) {
        if (ES == 4) {
          if (fl) reinterpret_cast<uint32_t*>(orow)[t] = 0u;
          else if (!inplace) reinterpret_cast<uint32_t*>(orow)[t] = reinterpret_cast<const uint32_t*>(row)[t];
        } else {
          if (fl) reinterpret_cast<uint16_t*>(orow)[t] = 0;
          else if (!inplace) reinterpret_cast<uint16_t*>(orow)[t] = reinterpret_cast<const uint16_t*>(row)[t];
        }
      }
    };
    unsigned long long s = 0;
    int n = 0;
    if (vout_cell) {
      // the row's 16-byte vectors, lane L taking vectors L, L + 32, ... (coalesced
      // loads and stores), eight in flight; the cell of vector k is k / vpc,
      // tracked from one step to the next without a division
      const int vpc = Ti / VS, nv = T / VS, qd = 32 / vpc, rd = 32 % vpc;
      int g = lane / vpc, kc = lane - (lane / vpc) * vpc;
      for (int k0 = 0; k0 < nv; k0 += 8 * 32) {
        uint4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = k0 + 32 * j + lane;
          if (k < nv) v[j] = __ldg(reinterpret_cast<const uint4*>(row) + k);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = k0 + 32 * j + lane;
          if (k < nv) {
            const bool fl = fr[g] != 0;
            const int t = k * VS;
            if (mr) {
              if constexpr (VS == 4) *reinterpret_cast<uint32_t*>(mr + t) = fl ? 0x01010101u : 0u;
              else *reinterpret_cast<uint2*>(mr + t) = fl ? make_uint2(0x01010101u, 0x01010101u) : make_uint2(0u, 0u);
            }
            if (fl) {
              if (orow) *reinterpret_cast<uint4*>(orow + t * ES) = make_uint4(0u, 0u, 0u, 0u);
            } else {
              s += vec_power_sum<DT>(v[j]);
              n += VS;
              if (orow && !inplace) *reinterpret_cast<uint4*>(orow + t * ES) = v[j];
            }
          }
          g += qd;
          kc += rd;
          if (kc >= vpc) {
            kc -= vpc;
            ++g;
          }
        }
      }
    } else if (chunked) {
      for (int g = g0; g < g1; ++g) {
        const bool fl = fr[g] != 0;
        for (int t = g * Ti; t < g * Ti + Ti; ++t) {
          if (!fl) {
            s += ipow<DT>(row, t);
            ++n;
          }
          put(t, fl);
        }
      }
    } else {
      for (int t = lane; t < T; t += 32) {
        const bool fl = fr[t / Ti] != 0;
        if (!fl) {
          s += ipow<DT>(row, t);
          ++n;
        }
        put(t, fl);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(kFullI, s, o);
      n += __shfl_xor_sync(kFullI, n, o);
    }
    bool fh = false;
    if (lane == 0) {
      fh = stage_history(kp, h, s, n);
      atomicAdd(&f.cnt_time, static_cast<unsigned long long>(T - n));
      if (fh) atomicAdd(&f.cnt_hist, 1ull);
      atomicAdd(&f.cnt_total, fh ? static_cast<unsigned long long>(T) : static_cast<unsigned long long>(T - n));
    }
    const bool full = __shfl_sync(kFullI, fh ? 1 : 0, 0) != 0;
    __syncwarp();  // the row's first writes, by every lane, before a rewrite
    if (full)
      for (int t = lane; t < T; t += 32) put(t, true);
  }
  __syncthreads();
  if (tid == 0 && u.stats) {
    u.stats->median_f = 0.0;
    u.stats->sigma_f = 0.0;
    u.stats->median_t = med;
    u.stats->sigma_t = sig;
    u.stats->n_chan_freq = 0;
    u.stats->n_flag_time = static_cast<long long>(f.cnt_time);
    u.stats->n_chan_hist = static_cast<long long>(f.cnt_hist);
    u.stats->n_flag_total = static_cast<long long>(f.cnt_total);
  }
  __syncthreads();
}

// MODE 0: integrated time mode; MODE 1: per-channel statistics scope; MODE 2:
// pooled per-channel time pass; MODE 3: two-dimensional mode on cells of
// cells.x channels x cells.y samples (the other modes ignore cells).
template <int DT, int MODE>
__global__ void __launch_bounds__(kNtI, 1) lof_integ_kernel(const KParams kp, const int2 cells) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ IntegShared f;
  for (int ui = blockIdx.x; ui < kp.n_units; ui += gridDim.x) {
    if constexpr (MODE == 0) integ_unit<DT>(kp, kp.units[ui], smem, f);
    else if constexpr (MODE == 3) grid_unit<DT>(kp, kp.units[ui], smem, f, cells.x, cells.y);
    else chan_unit<DT, MODE == 2>(kp, kp.units[ui], smem, f);
  }
}

}  // namespace
}  // namespace lofk

extern "C" int lofk_integ_max_time() { return lofk::kIntegMaxT; }

// The integrated time mode (mode 0), the per-channel statistics scope (mode 1),
// the pooled per-channel pass with exact statistics (mode 2) or the
// two-dimensional mode on cells of cell_chan x cell_time samples (mode 3)
// over n_units integer units (one CTA per unit).  The kernel's arguments are
// (KParams, int2 cells).
extern "C" int lofk_launch_integ(int dtype, const lofk::KParams* kp, int n_units, int n_sm, void* stream,
                                 int mode, int cell_chan, int cell_time) {
  using namespace lofk;
  if (n_units <= 0) return 0;
  if (mode < 0 || mode > 3 || cell_chan < 1 || cell_time < 1) return static_cast<int>(cudaErrorInvalidValue);
  const void* ks[2][4] = {{reinterpret_cast<const void*>(&lof_integ_kernel<LOF_CI16, 0>),
                           reinterpret_cast<const void*>(&lof_integ_kernel<LOF_CI16, 1>),
                           reinterpret_cast<const void*>(&lof_integ_kernel<LOF_CI16, 2>),
                           reinterpret_cast<const void*>(&lof_integ_kernel<LOF_CI16, 3>)},
                          {reinterpret_cast<const void*>(&lof_integ_kernel<LOF_CI8, 0>),
                           reinterpret_cast<const void*>(&lof_integ_kernel<LOF_CI8, 1>),
                           reinterpret_cast<const void*>(&lof_integ_kernel<LOF_CI8, 2>),
                           reinterpret_cast<const void*>(&lof_integ_kernel<LOF_CI8, 3>)}};
  const void* k = ks[dtype == LOF_CI16 ? 0 : 1][mode];
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kIntegSmem) != cudaSuccess)
    return -2;
  const int grid = n_units < n_sm ? n_units : n_sm;
  int2 cells = make_int2(cell_chan, cell_time);
  void* args[] = {const_cast<KParams*>(kp), &cells};
  const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(kNtI), args, static_cast<size_t>(kIntegSmem),
                                         static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? 0 : static_cast<int>(e);
}
