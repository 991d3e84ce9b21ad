// lof_f32.cu -- the flagger for float32 units: Stokes I power (LOF_F32), or
// complex float32 visibilities (LOF_CF32, the post-correlation placement of
// Section 3) whose power |V|^2 = re^2 + im^2 is formed in float32 on load.
//
// One CTA flags one unit at a time (units are independent; a launch takes a
// whole block of units, grid-strided).  Steps, in the order of the paper's
// Section 4 pipeline:
//   a1  P = the input (non-finite samples count as flagged and are excluded)
//   a2  row sums S[c] over the finite samples, binary64
//   a3  median and 1.4826*MAD of S (bitonic sort in shared memory)
//   a4  SumThreshold over S (Section 2.1), binary64 window sums in the order
//       of the definition
//   a5  median and MAD of the finite samples of the kept channels: exact
//       order statistics by three radix-select passes over monotone 32-bit
//       keys of the floats (two ranks at once for an even count); the MAD is
//       taken over float32 keys of |x - median|, formed in float32 from the
//       median split into two floats (error about a unit in the last place)
//   a6  SumThreshold along time, one warp per 1024-sample row segment (rows
//       longer than 1024 overlap by a 120-sample halo, as in the integer
//       path): flagged samples are replaced by threshold_I and the window
//       sums are built by doubling (S_2I(j) = S_I(j) + S_I(j + I)) in
//       float32, so each sum is a balanced tree of at most 64 terms
//       (relative error <= 6 * 2^-24); a window fires when its sum exceeds
//       I * threshold_I
//   a7  history test per channel (binary64 mean of the unflagged samples)
//   a8  mask bytes and the masked data
// Float results match the binary64 oracle except for samples whose deciding
// window sum lies within a relative 1e-5 of its threshold (and the windows a
// changed flag touches later).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lof_internal.h"

namespace lofk {
namespace {

constexpr unsigned kFullF = 0xFFFFFFFFu;
constexpr int kHaloF = 120;   // sum over window sizes of (I - 1)
constexpr int kNplF = 32;     // samples per lane in the time pass
constexpr int kNtF = 256;     // threads per CTA
constexpr int kNwF = kNtF / 32;

// shared-memory layout of one CTA (bytes)
constexpr int kOffS = 0;                                  // double S[2048]
constexpr int kOffSrt = kOffS + 8 * kMaxChan;             // u64 sort keys [2048]
constexpr int kOffFin = kOffSrt + 8 * kMaxChan;           // int finite count [2048]
constexpr int kOffFc = kOffFin + 4 * kMaxChan;            // uint8 Fc [2048]
constexpr int kOffFire = kOffFc + kMaxChan;               // uint8 fire [2048]
constexpr int kOffHist = kOffFire + kMaxChan;             // u32 hist[2][2048]
constexpr int kOffRows = kOffHist + 2 * 2048 * 4;         // per-warp flag words of one row
constexpr int kFixedBytesF = kOffRows;

struct F32Shared {
  double median_f, sigma_f, median_t, sigma_t;
  double tI[kMaxLogWindow + 1];   // threshold_I (time pass)
  float limI[kMaxLogWindow + 1];  // I * threshold_I as float32
  float tIf[kMaxLogWindow + 1];   // threshold_I as float32
  long long n_pool;
  unsigned long long cnt_time, cnt_total, cnt_hist;
  uint32_t prefix[2];
  long long rank[2];
  int n_rank, kmax_t, time_on, nfc, ok, wmiss;
  double red[kNwF];
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullF, v, o);
  return v;
}
// Compensated float32 accumulation (Knuth's TwoSum): hi + lo carries the
// sum of the added values to about 2^-48 relative per lane, in float32
// arithmetic (GB300's binary64 rate is a small fraction of its float32 one).
// The caller checks that hi and lo stay finite (a sum beyond the float32
// range) and then sums in binary64 instead.
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  const float t = __fadd_rn(hi, x);
  const float bp = __fsub_rn(t, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  hi = t;
  lo = __fadd_rn(lo, e);
}
__device__ __forceinline__ bool df_ok(float hi, float lo) { return isfinite(hi) && isfinite(lo); }

__device__ __forceinline__ uint32_t saddr_f(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Adds 1 to the shared counter at byte address base + 4 * t when t < n
// (unsigned), as one predicated reduction.
__device__ __forceinline__ void red_shared_inc_f(uint32_t t, uint32_t n, uint32_t base) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t.reg .u32 a;\n\tsetp.lt.u32 q, %0, %1;\n\t"
      "mad.lo.u32 a, %0, 4, %2;\n\t@q red.shared.add.u32 [a], 1;\n\t}" ::"r"(t),
      "r"(n), "r"(base)
      : "memory");
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullF, v, o);
  return v;
}
__device__ __forceinline__ uint32_t fkey(float x) {  // monotone in x
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_val(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
__device__ __forceinline__ unsigned long long dkey(double x) {  // monotone in x
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  return (u >> 63) ? ~u : (u | (1ull << 63));
}
__device__ __forceinline__ double dkey_val(unsigned long long k) {
  return __longlong_as_double(static_cast<long long>((k >> 63) ? (k & ~(1ull << 63)) : ~k));
}
__device__ __forceinline__ uint32_t dilate32f(uint32_t hi, uint32_t lo, int I) {
  unsigned long long x = (static_cast<unsigned long long>(hi) << 32) | lo;
  for (int s = 1; s < I; s <<= 1) x |= x << s;
  return static_cast<uint32_t>(x >> 32);
}
__device__ void set_error_f(const KParams& kp, int code, int info) {
  if (atomicCAS(kp.err, 0, code) == 0) {
    kp.err_info[0] = info;
    kp.err_info[1] = static_cast<int>(kp.block_seq);
  }
}

// threshold_I = median + sigma * factor_I * sensitivity (Section 2.1), binary64
// in the order of the definition
__device__ __forceinline__ double thr_of(const KParams& kp, double m, double s, int k) {
  return __dadd_rn(m, __dmul_rn(__dmul_rn(s, kp.factor[k]), kp.sensitivity));
}

// Power of a complex float32 sample, in float32 (non-finite if re or im is).
__device__ __forceinline__ float cpw(float re, float im) {
  return __fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im));
}
// Power of sample t of a row: IN = 0 the value itself (Stokes I), IN = 1 the
// |V|^2 of the complex value (re, im interleaved).
template <int IN>
__device__ __forceinline__ float fat(const float* row, int t) {
  if constexpr (IN == 0) return row[t];
  else return cpw(row[2 * t], row[2 * t + 1]);
}
// Powers of 4 samples of a row at x (x a multiple of 4); non-finite and
// past-T samples come back as NaN.
template <int IN>
__device__ __forceinline__ float4 ld4(const float* row, int x, int T, bool vec) {
  if constexpr (IN == 0) {
    if (vec && x + 4 <= T) return __ldg(reinterpret_cast<const float4*>(row + x));
  } else {
    if (vec && x + 4 <= T) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(row + 2 * x));
      const float4 b = __ldg(reinterpret_cast<const float4*>(row + 2 * x + 4));
      return make_float4(cpw(a.x, a.y), cpw(a.z, a.w), cpw(b.x, b.y), cpw(b.z, b.w));
    }
  }
  float a[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) a[j] = x + j < T ? fat<IN>(row, x + j) : __int_as_float(0x7FC00000);
  return make_float4(a[0], a[1], a[2], a[3]);
}
__device__ __forceinline__ float f4at(const float4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// Bitonic sort of n (power of two) u64 keys, ascending.
__device__ void sort64(unsigned long long* a, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += kNtF) {
        const int p = i ^ j;
        if (p > i) {
          const unsigned long long x = a[i], y = a[p];
          if ((x > y) == ((i & k) == 0)) {
            a[i] = y;
            a[p] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Median and sigma of the C doubles in S (Section 4.2 statistics).
__device__ void spectrum_stats(const KParams& kp, const double* S, int C, unsigned long long* srt,
                               F32Shared& f) {
  const int tid = threadIdx.x;
  int n2 = 1;
  while (n2 < C) n2 <<= 1;
  for (int i = tid; i < n2; i += kNtF) srt[i] = i < C ? dkey(S[i]) : ~0ull;
  __syncthreads();
  sort64(srt, n2);
  if (tid == 0) {
    f.median_f = (C & 1) ? dkey_val(srt[C / 2])
                         : __dmul_rn(__dadd_rn(dkey_val(srt[C / 2 - 1]), dkey_val(srt[C / 2])), 0.5);
  }
  __syncthreads();
  const double m = f.median_f;
  for (int i = tid; i < n2; i += kNtF) srt[i] = i < C ? dkey(fabs(__dsub_rn(S[i], m))) : ~0ull;
  __syncthreads();
  sort64(srt, n2);
  if (tid == 0) {
    const double mad = (C & 1) ? dkey_val(srt[C / 2])
                               : __dmul_rn(__dadd_rn(dkey_val(srt[C / 2 - 1]), dkey_val(srt[C / 2])), 0.5);
    double sig;
    if (!kp.sigma_std && mad > 0.0) {
      sig = __dmul_rn(1.482602218505602, mad);
    } else {  // population stddev, two sequential passes
      double s = 0.0;
      for (int i = 0; i < C; ++i) s = __dadd_rn(s, S[i]);
      const double mu = __ddiv_rn(s, static_cast<double>(C));
      double q = 0.0;
      for (int i = 0; i < C; ++i) {
        const double d = __dsub_rn(S[i], mu);
        q = __dadd_rn(q, __dmul_rn(d, d));
      }
      sig = __dsqrt_rn(__ddiv_rn(q, static_cast<double>(C)));
    }
    f.sigma_f = sig;
  }
  __syncthreads();
}

// Section 2.1 over the spectrum: binary64 window sums in index order.
__device__ void spectrum_sum_threshold(const KParams& kp, const double* S, int C, uint8_t* Fc,
                                       uint8_t* fire, const F32Shared& f) {
  const int tid = threadIdx.x;
  const double m = f.median_f, sig = f.sigma_f;
  if (!kp.enable_freq || !(sig > 0.0)) return;
  for (int k = 0; k <= kp.max_log_window; ++k) {
    const int I = 1 << k;
    if (I > C) break;
    const double thr = thr_of(kp, m, sig, k);
    for (int t = tid; t < C; t += kNtF) {
      uint8_t fl = 0;
      if (t + I <= C) {
        double su = 0.0;
        int nf = 0;
        for (int j = t; j < t + I; ++j) {
          if (Fc[j]) ++nf;
          else su = __dadd_rn(su, S[j]);
        }
        fl = su > __dmul_rn(static_cast<double>(I - nf), thr) ? 1 : 0;
      }
      fire[t] = fl;
    }
    __syncthreads();
    for (int c = tid; c < C; c += kNtF) {
      uint8_t any = Fc[c];
      for (int t = max(0, c - I + 1); t <= c && !any; ++t) any = fire[t];
      Fc[c] = any;
    }
    __syncthreads();
  }
}

// Calls fn(v) for each 4-sample vector of the finite-or-not samples of the
// kept rows (Fc clear): the warps take (row, 128-sample chunk) items in turn,
// each warp with the loads of eight items in flight before it counts them.
template <int IN, typename Fn>
__device__ __forceinline__ void for_kept_vectors(const DevUnit& u, const uint8_t* Fc, Fn&& fn) {
  constexpr int NL = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int T = u.T, nchunk = (T + 127) / 128, total = u.C * nchunk;
  const bool vin = (u.flags & kUnitInVec) != 0;
  const float* gin = static_cast<const float*>(u.in);
  // item i = row c, 128-sample chunk q: (c, q) advance by kNwF items a step
  // (chunks < nchunk, kNwF <= nchunk or several wraps), no division per item
  int c = warp / nchunk, q = warp - c * nchunk;
  for (int i0 = warp; i0 < total; i0 += NL * kNwF) {
    float4 v[NL];
    bool ok[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int item = i0 + k * kNwF;
      const int x = q * 128 + lane * 4;
      ok[k] = item < total && !Fc[c] && x < T;
      v[k] = ok[k] ? ld4<IN>(gin + static_cast<int64_t>(c) * u.in_stride * (IN + 1), x, T, vin)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
      q += kNwF;
      while (q >= nchunk) {
        q -= nchunk;
        ++c;
      }
    }
#pragma unroll
    for (int k = 0; k < NL; ++k)
      if (ok[k]) fn(v[k]);
  }
}

// One radix-select pass over the finite samples of the kept rows: histogram
// of the 11 (or 10) key bits below those already fixed, for each open rank.
// MODE 0: keys of x; MODE 1: keys of float(|x - median_t|).
template <int MODE, int IN>
__device__ void select_pass(const DevUnit& u, const uint8_t* Fc, uint32_t* hist, int shift,
                            int nbits, F32Shared& f) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = 1 << nbits;
  for (int i = tid; i < 2 * 2048; i += kNtF) hist[i] = 0u;
  __syncthreads();
  const uint32_t p0 = f.prefix[0], p1 = f.prefix[1];
  const int hs = shift + nbits;  // bits above this digit are fixed
  const bool two = f.n_rank == 2;
  // the two ranks of an even count share their prefix until late: then one
  // histogram serves both
  const bool same = !two || p0 == p1;
  // |x - median| in float32 from the median split into two floats: the
  // error stays within a unit in the last place of the deviation (the keys
  // are float32 anyway), with no binary64 operation per sample
  const float med_hi = __double2float_rn(f.median_t);
  const float med_lo = __double2float_rn(__dsub_rn(f.median_t, static_cast<double>(med_hi)));
  for_kept_vectors<IN>(u, Fc, [&](const float4& v) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float xv = f4at(v, j);
      if (!isfinite(xv)) continue;  // also the NaN past T
      const float kv = MODE == 0 ? xv : fabsf(__fsub_rn(__fsub_rn(xv, med_hi), med_lo));
      const uint32_t key = fkey(kv);
      const uint32_t hi = hs >= 32 ? 0u : (key >> hs);
      const uint32_t dig = (key >> shift) & static_cast<uint32_t>(nb - 1);
      if (hi == p0) atomicAdd(&hist[dig], 1u);
      if (!same && hi == p1) atomicAdd(&hist[2048 + dig], 1u);
    }
  });
  __syncthreads();
  // pick the digit of each open rank (one warp per rank)
  if (warp < f.n_rank) {
    const uint32_t* h = hist + (same ? 0 : 2048 * warp);
    long long rk = f.rank[warp];
    long long base = 0;
    uint32_t digit = 0;
    bool found = false;
    for (int b0 = 0; b0 < nb && !found; b0 += 32) {
      const uint32_t cnt = h[b0 + lane];
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullF, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t tot = __shfl_sync(kFullF, incl, 31);
      if (rk < base + tot) {
        const unsigned hit = __ballot_sync(kFullF, rk < base + static_cast<long long>(incl));
        const int l = __ffs(hit) - 1;
        const uint32_t excl = __shfl_sync(kFullF, incl - cnt, l);
        digit = static_cast<uint32_t>(b0 + l);
        rk -= base + excl;
        found = true;
      } else {
        base += tot;
      }
    }
    if (lane == 0) {
      if (!found) f.ok = 0;
      f.prefix[warp] = (f.prefix[warp] << nbits) | digit;
      f.rank[warp] = rk;
    }
  }
  __syncthreads();
  if (tid == 0 && f.n_rank == 1) {
    f.prefix[1] = f.prefix[0];
    f.rank[1] = f.rank[0];
  }
  __syncthreads();
}

template <int MODE, int IN>
__device__ double select_median(const DevUnit& u, const uint8_t* Fc, uint32_t* hist, F32Shared& f) {
  const long long N = f.n_pool;
  if (threadIdx.x == 0) {
    f.prefix[0] = f.prefix[1] = 0u;
    f.rank[0] = (N & 1) ? N / 2 : N / 2 - 1;
    f.rank[1] = N / 2;
    f.n_rank = (N & 1) ? 1 : 2;
  }
  __syncthreads();
  select_pass<MODE, IN>(u, Fc, hist, 21, 11, f);
  select_pass<MODE, IN>(u, Fc, hist, 10, 11, f);
  select_pass<MODE, IN>(u, Fc, hist, 0, 10, f);
  const double a = static_cast<double>(fkey_val(f.prefix[0]));
  const double b = static_cast<double>(fkey_val(f.prefix[1]));
  return (N & 1) ? a : __dmul_rn(__dadd_rn(a, b), 0.5);
}


// ---- order statistics in a window around the previous block's value
// With a hint h (the unit's median, or MAD, of the previous block) and a
// half-width hw (halved up to four times until it fits), the keys of
// [h - hw, h + hw] form an interval [klo, khi] of at most 2^22 keys (else no
// window).  Pass 1 counts the keys below klo and
// histograms those in the interval in 2048 bins of 2^s keys; the bin of each
// open rank follows from the counts; pass 2 counts key by key inside those
// bins and gives the exact keys.  The result is the same order statistic as
// the three radix passes (select_median); false (nothing decided) when a rank
// falls outside the interval.
template <int MODE, int IN>
__device__ void window_count(const DevUnit& u, const uint8_t* Fc, uint32_t* hist, uint32_t klo, int s,
                             int fine, F32Shared& f, long long* below_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float med_hi = __double2float_rn(f.median_t);
  const float med_lo = __double2float_rn(__dsub_rn(f.median_t, static_cast<double>(med_hi)));
  // fine: bins b0 = f.prefix[0], b1 = f.prefix[1] (coarse bins of the ranks)
  const uint32_t w = 1u << s;
  const uint32_t base0 = klo + (f.prefix[0] << s), base1 = klo + (f.prefix[1] << s);
  const bool two = fine && f.n_rank == 2 && f.prefix[0] != f.prefix[1];
  // Predicated counts, no branch per sample.  A key below klo wraps:
  // key - klo >= 2^32 - klo > 2^23, as klo is the key of a finite value
  // (at most that of FLT_MAX, 0xFF7FFFFF), so (key - klo) >> s >= 4096 for
  // s <= 11 and the bin test alone keeps it out of the counters.
  const uint32_t hsa = saddr_f(hist), hsa1 = hsa + 4u * 2048u;
  const uint32_t wlim = two ? w : 0u;
  uint32_t below = 0u;  // a lane's share: below 2^31 samples
  if (!fine) {
    for_kept_vectors<IN>(u, Fc, [&](const float4& v) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float xv = f4at(v, j);
        const float kv = MODE == 0 ? xv : fabsf(__fsub_rn(__fsub_rn(xv, med_hi), med_lo));
        const uint32_t key = fkey(kv);
        const uint32_t fin = isfinite(xv) ? 1u : 0u;
        below += fin & (key < klo ? 1u : 0u);
        red_shared_inc_f(fin ? (key - klo) >> s : 0xFFFFFFFFu, 2048u, hsa);
      }
    });
  } else {
    for_kept_vectors<IN>(u, Fc, [&](const float4& v) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float xv = f4at(v, j);
        const float kv = MODE == 0 ? xv : fabsf(__fsub_rn(__fsub_rn(xv, med_hi), med_lo));
        const uint32_t key = fkey(kv);
        const bool fin = isfinite(xv);
        red_shared_inc_f(fin ? key - base0 : 0xFFFFFFFFu, w, hsa);
        red_shared_inc_f(fin ? key - base1 : 0xFFFFFFFFu, wlim, hsa1);
      }
    });
  }
  if (!fine) {
    below = static_cast<uint32_t>(warp_sum_ll(static_cast<long long>(below)));
    if (lane == 0) f.red[warp] = static_cast<double>(below);  // exact: counts < 2^53
  }
  __syncthreads();
  if (!fine && tid == 0) {
    long long b = 0;
    for (int q = 0; q < kNwF; ++q) b += static_cast<long long>(f.red[q]);
    *below_out = b;
  }
  __syncthreads();
}

// The bin (or key) of each open rank in hist (nb counters; rank r of rank
// slot q, relative to the counters' start); one warp per rank.  Sets
// f.prefix[q] to the bin and f.rank[q] to the rank inside it; f.ok = 0 if a
// rank lies past the counted values.
__device__ void window_pick(const uint32_t* hist, int nb, bool split, F32Shared& f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < f.n_rank) {
    const uint32_t* h = hist + (split ? 2048 * warp : 0);
    long long rk = f.rank[warp];
    long long base = 0;
    uint32_t digit = 0;
    bool found = false;
    if (rk >= 0) {
      for (int b0 = 0; b0 < nb && !found; b0 += 32) {
        const uint32_t cnt = b0 + lane < nb ? h[b0 + lane] : 0u;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(kFullF, incl, o);
          if (lane >= o) incl += y;
        }
        const uint32_t tw = __shfl_sync(kFullF, incl, 31);
        if (rk < base + tw) {
          const unsigned hit = __ballot_sync(kFullF, rk < base + static_cast<long long>(incl));
          const int l = __ffs(hit) - 1;
          const uint32_t excl = __shfl_sync(kFullF, incl - cnt, l);
          digit = static_cast<uint32_t>(b0 + l);
          rk -= base + excl;
          found = true;
        } else {
          base += tw;
        }
      }
    }
    if (lane == 0) {
      f.prefix[warp] = digit;
      f.rank[warp] = rk;
      if (!found) f.wmiss = 1;
    }
  }
  __syncthreads();
}

template <int MODE, int IN>
__device__ bool window_select(const DevUnit& u, const uint8_t* Fc, uint32_t* hist, F32Shared& f, double h,
                              double hw, double* out) {
  const int tid = threadIdx.x;
  const long long N = f.n_pool;
  if (!(hw > 0.0) || N <= 0) return false;
  // the widest of hw, hw / 2, ..., hw / 16 whose keys fit two passes (2^22)
  uint32_t klo = 0u;
  int s = 12;
  for (int t = 0; t < 5 && s > 11; ++t, hw = __dmul_rn(hw, 0.5)) {
    const float lo_v = __double2float_rd(__dsub_rn(h, hw)), hi_v = __double2float_ru(__dadd_rn(h, hw));
    if (!isfinite(lo_v) || !isfinite(hi_v)) return false;
    const uint32_t a = fkey(lo_v), b = fkey(hi_v);
    if (b < a) return false;
    const unsigned long long span = static_cast<unsigned long long>(b - a) + 1ull;
    s = 0;
    while ((span >> s) > 2048ull) ++s;
    klo = a;
  }
  if (s > 11) return false;
  for (int i = tid; i < 2 * 2048; i += kNtF) hist[i] = 0u;
  if (tid == 0) {
    f.rank[0] = (N & 1) ? N / 2 : N / 2 - 1;
    f.rank[1] = N / 2;
    f.n_rank = (N & 1) ? 1 : 2;
  }
  __shared__ long long s_below;
  __syncthreads();
  window_count<MODE, IN>(u, Fc, hist, klo, s, 0, f, &s_below);
  if (tid == 0) {
    f.rank[0] -= s_below;
    f.rank[1] -= s_below;
    f.wmiss = 0;
  }
  __syncthreads();
  window_pick(hist, 2048, false, f);
  const bool miss1 = f.wmiss != 0;
  __syncthreads();
  if (miss1) return false;
  // pass 2: key by key inside the ranks' bins
  for (int i = tid; i < 2 * 2048; i += kNtF) hist[i] = 0u;
  __syncthreads();
  const uint32_t bin0 = f.prefix[0], bin1 = f.n_rank == 2 ? f.prefix[1] : f.prefix[0];
  if (tid == 0 && f.n_rank == 1) f.prefix[1] = f.prefix[0];
  __syncthreads();
  window_count<MODE, IN>(u, Fc, hist, klo, s, 1, f, &s_below);
  const bool split = f.n_rank == 2 && bin0 != bin1;
  window_pick(hist, 1 << s, split, f);
  const bool miss2 = f.wmiss != 0;
  __syncthreads();
  if (miss2) {  // cannot happen when pass 1 placed the ranks (same counts)
    if (tid == 0) f.ok = 0;
    return false;
  }
  const uint32_t k0 = klo + (bin0 << s) + f.prefix[0];
  const uint32_t k1 = klo + (bin1 << s) + (f.n_rank == 2 ? f.prefix[1] : f.prefix[0]);
  const double a = static_cast<double>(fkey_val(k0)), b = static_cast<double>(fkey_val(k1));
  *out = (N & 1) ? a : __dmul_rn(__dadd_rn(a, b), 0.5);
  __syncthreads();
  return true;
}

// The previous block's median and MAD of a unit with a history slot (the
// statistics hints, stored as binary64), if any.
__device__ __forceinline__ bool f32_hints(const KParams& kp, const DevUnit& u, double* m, double* d) {
  if (!kp.hist.hint || u.hist_slot < 0) return false;
  const unsigned long long a = kp.hist.hint[2 * u.hist_slot], b = kp.hist.hint[2 * u.hist_slot + 1];
  if (a == ~0ull || b == ~0ull) return false;
  *m = __longlong_as_double(static_cast<long long>(a));
  *d = __longlong_as_double(static_cast<long long>(b));
  return isfinite(*m) && isfinite(*d) && *d > 0.0;
}

// population stddev of the pooled finite samples (binary64, two passes)
template <int IN>
__device__ double pooled_std(const DevUnit& u, const uint8_t* Fc, F32Shared& f) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* gin = static_cast<const float*>(u.in);
  const int T = u.T;
  double acc[2] = {0.0, 0.0};
  double mu = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    double s = 0.0;
    for (int c = warp; c < u.C; c += kNwF) {
      if (Fc[c]) continue;
      const float* row = gin + static_cast<int64_t>(c) * u.in_stride * (IN + 1);
      for (int t = lane; t < T; t += 32) {
        const float xv = fat<IN>(row, t);
        if (!isfinite(xv)) continue;
        const double d = pass == 0 ? static_cast<double>(xv) : __dsub_rn(static_cast<double>(xv), mu);
        s = pass == 0 ? __dadd_rn(s, d) : __dadd_rn(s, __dmul_rn(d, d));
      }
    }
    s = warp_sum_d(s);
    if (lane == 0) f.red[warp] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kNwF; ++w) t = __dadd_rn(t, f.red[w]);
      f.red[0] = t;
    }
    __syncthreads();
    acc[pass] = f.red[0];
    __syncthreads();
    if (pass == 0) mu = __ddiv_rn(acc[0], static_cast<double>(f.n_pool));
  }
  return __dsqrt_rn(__ddiv_rn(acc[1], static_cast<double>(f.n_pool)));
}

// ---- Stokes I units in a thread-block cluster (F32, Section 3's
// beamformed placement)
// One cluster of CL CTAs (CL = 16 where the device allows clusters that
// large, else 8) flags one unit: CTA r holds rows [r R, r R + R) of it in
// shared memory (R = ceil(C / CL)), read from global memory once.  The
// steps and their arithmetic are those of f32_unit; what the CTAs share goes
// through distributed shared memory:
//   * the row sums S[c] and finite counts (every CTA writes its rows into
//     every CTA), so each CTA runs the frequency pass on the whole spectrum;
//   * each radix-select pass: every CTA histograms its rows, CTA r adds up
//     bins [r B / CL, (r + 1) B / CL) of all CTAs and writes the sums into
//     every CTA, each CTA then picks the same digit;
//   * the binary64 sums of the std estimator (per CTA, added in rank order);
//   * the flag counts, added into CTA 0, which reports the unit's statistics.
// Row sums, window sums, order statistics and the history test are computed
// exactly as in f32_unit (same per-row summation order), so both kernels
// give the same flags; only the std estimator's binary64 sums may round
// differently (their order follows the CTAs).
namespace cg = cooperative_groups;

constexpr int kCMaxCl = 256;                 // channels of a unit in the cluster path
constexpr int kClMaxSeg = 48;                // row segments (1024-sample spans) of one row

// shared-memory layout of one cluster CTA (bytes), for R rows of T samples
constexpr int kOffClS = 0;                                // double S[256]
constexpr int kOffClSrt = kOffClS + 8 * kCMaxCl;          // u64 sort keys [256]
constexpr int kOffClFin = kOffClSrt + 8 * kCMaxCl;        // int finite count [256]
constexpr int kOffClFc = kOffClFin + 4 * kCMaxCl;         // uint8 Fc [256]
constexpr int kOffClFire = kOffClFc + kCMaxCl;            // uint8 fire [256]
constexpr int kOffClHist = kOffClFire + kCMaxCl;          // u32 local hist[2][2048]
constexpr int kOffClTot = kOffClHist + 2 * 2048 * 4;      // u32 cluster hist[2][2048]
constexpr int kOffClRed = kOffClTot + 2 * 2048 * 4;       // double red[16], u64 cnt[4]
constexpr int kOffClRows = kOffClRed + 16 * 8 + 4 * 8;    // per-row: segment sums, counts
constexpr int kClRowBytes = kClMaxSeg * 8 + 4 * 4;        //   double su[48]; int nflag, nentry, fh, pad
__host__ __device__ constexpr int cl_words(int T) { return (T + 31) / 32; }
__host__ __device__ constexpr int cl_pitch(int T) { return (T + 3) & ~3; }  // floats per stored row
__host__ __device__ inline int cl_off_mrow(int R) { return (kOffClRows + R * kClRowBytes + 15) & ~15; }
__host__ __device__ inline int cl_off_data(int R, int T) {
  return (cl_off_mrow(R) + R * cl_words(T) * 4 + 15) & ~15;
}
__host__ __device__ inline int cl_smem(int R, int T) { return cl_off_data(R, T) + R * cl_pitch(T) * 4; }

// 4 samples of a stored row at x (x a multiple of 4); past T: NaN
__device__ __forceinline__ float4 ld4s(const float* srow, int x, int T) {
  if (x + 4 <= T) return *reinterpret_cast<const float4*>(srow + x);
  float a[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) a[j] = x + j < T ? srow[x + j] : __int_as_float(0x7FC00000);
  return make_float4(a[0], a[1], a[2], a[3]);
}

// Adds the CTAs' histograms (nbins words) and leaves the sums in every CTA's
// tot (reduce-scatter then all-gather over distributed shared memory).
__device__ void cl_allreduce_hist(cg::cluster_group& cl, uint32_t* hist, uint32_t* tot, int nbins) {
  const int CL = static_cast<int>(cl.num_blocks()), r = static_cast<int>(cl.block_rank());
  cl.sync();  // every CTA's histogram complete
  const int per = (nbins + CL - 1) / CL, b0 = r * per, b1 = min(nbins, b0 + per);
  for (int b = b0 + static_cast<int>(threadIdx.x); b < b1; b += kNtF) {
    uint32_t s = 0u;
    for (int q = 0; q < CL; ++q) s += cl.map_shared_rank(hist, q)[b];
    for (int q = 0; q < CL; ++q) cl.map_shared_rank(tot, q)[b] = s;
  }
  cl.sync();  // every sum in place; no CTA reads hist any more
}

// ---- time pass of one row segment by one warp (float32 window sums)
struct WfRow {
  float v[kNplF];  // the sample (0 where non-finite)
  uint32_t M;      // flag bits
};

template <int I>
__device__ __forceinline__ uint32_t wf_fire(const WfRow& R, int lane, float tI, float lim) {
  float W[kNplF];
#pragma unroll
  for (int j = 0; j < kNplF; ++j) W[j] = ((R.M >> j) & 1u) ? tI : R.v[j];
#pragma unroll
  for (int s = 1; s < I; s <<= 1) {
    float nx[kNplF];
#pragma unroll
    for (int j = 0; j < kNplF; ++j) {
      if (j + s >= kNplF) {
        const int q = (j + s) / kNplF;
        float y = __shfl_down_sync(kFullF, W[j + s - q * kNplF], q);
        nx[j] = lane + q < 32 ? y : 0.0f;
      }
    }
#pragma unroll
    for (int j = 0; j < kNplF; ++j) W[j] = __fadd_rn(W[j], j + s < kNplF ? W[j + s] : nx[j]);
  }
  uint32_t f = 0u;
#pragma unroll
  for (int j = kNplF - 1; j >= 0; --j) f = __funnelshift_l(__float_as_uint(__fsub_rn(lim, W[j])), f, 1);
  return f;
}

// Segments of a row of T samples: a segment that does not reach T ends its
// interior D = (SPAN - halo) & ~31 after its start (a multiple of 32), and
// the next starts STEP = (D - halo) & ~31 later.
__device__ __forceinline__ int wf_seg_count(int T) {
  constexpr int SPAN = 32 * kNplF, D = (SPAN - kHaloF) & ~31, STEP = (D - kHaloF) & ~31;
  return T <= SPAN ? 1 : (T - SPAN + STEP - 1) / STEP + 1;
}

// Flags of segment sg of one row (rows past 1024 samples overlap by a halo of
// 120 samples); interior flag words go to Mrow, returns the interior's number
// of flagged samples, entry-flagged samples and unflagged sum.
template <int IN, bool SM = false>
__device__ void wf_segment(const float* row, int T, int sg, bool vin, const F32Shared& f,
                           uint32_t* Mrow, int& nflag, int& nentry, double& su) {
  constexpr int SPAN = 32 * kNplF;
  const int lane = threadIdx.x & 31;
  // starts are multiples of 32, so the steps are constant (wf_seg_count)
  constexpr int D = (SPAN - kHaloF) & ~31, STEP = (D - kHaloF) & ~31;
  const int s0 = sg * STEP, oa = sg == 0 ? 0 : s0 - STEP + D, ob = s0 + SPAN >= T ? T : s0 + D;
  const int vend = min(T, s0 + SPAN);
  const int xl = s0 + lane * kNplF;
  WfRow R;
  R.M = 0u;
#pragma unroll
  for (int q = 0; q < kNplF / 4; ++q) {
    const int x = xl + 4 * q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x < T) {
      if constexpr (SM) v = ld4s(row, x, T);  // a row stored in shared memory (IN = 0)
      else v = ld4<IN>(row, x, T, vin);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float xv = f4at(v, j);
      const bool bad = x + j < T && !isfinite(xv);
      R.v[4 * q + j] = (x + j < T && !bad) ? xv : 0.0f;
      if (bad) R.M |= 1u << (4 * q + j);
    }
  }
  if constexpr (!SM) {
    // the next segment's samples toward L2 while this one is computed
    if (ob < T) {
      const int s0n = (ob - kHaloF) & ~31;
      const float* pn = row + static_cast<int64_t>(s0n + lane * kNplF) * (IN + 1);
      if (s0n + lane * kNplF < T) {
#pragma unroll
        for (int q = 0; q <= IN; ++q) asm volatile("prefetch.global.L2 [%0];" ::"l"(pn + 32 * q));
      }
    }
  }
  const uint32_t entry = R.M;
#pragma unroll 1
  for (int k = 0; k <= f.kmax_t; ++k) {
    const int I = 1 << k;
    const float tI = f.tIf[k], lim = f.limI[k];
    uint32_t F;
    switch (k) {
      case 0: F = wf_fire<1>(R, lane, tI, lim); break;
      case 1: F = wf_fire<2>(R, lane, tI, lim); break;
      case 2: F = wf_fire<4>(R, lane, tI, lim); break;
      case 3: F = wf_fire<8>(R, lane, tI, lim); break;
      case 4: F = wf_fire<16>(R, lane, tI, lim); break;
      case 5: F = wf_fire<32>(R, lane, tI, lim); break;
      default: F = wf_fire<64>(R, lane, tI, lim); break;
    }
    const int nv = vend - I + 1 - xl;
    F &= nv >= 32 ? kFullF : (nv <= 0 ? 0u : ((1u << nv) - 1u));
    uint32_t p1 = __shfl_up_sync(kFullF, F, 1), p2 = __shfl_up_sync(kFullF, F, 2);
    if (lane < 1) p1 = 0u;
    if (lane < 2) p2 = 0u;
    const uint32_t D = I <= 32 ? dilate32f(F, p1, I) : (dilate32f(F, p1, 32) | dilate32f(p1, p2, 32));
    R.M |= D;
  }
  int nf = 0, ne = 0;
  double s = 0.0;
  if (xl >= oa && xl < ob) {
    Mrow[xl >> 5] = R.M;
    nf = __popc(R.M);
    ne = __popc(entry);
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int j = 0; j < kNplF; ++j)
      if (!((R.M >> j) & 1u)) df_add(hi, lo, R.v[j]);
    s = __dadd_rn(static_cast<double>(hi), static_cast<double>(lo));
    if (!df_ok(hi, lo)) {  // beyond the float32 range
      s = 0.0;
#pragma unroll
      for (int j = 0; j < kNplF; ++j)
        if (!((R.M >> j) & 1u)) s = __dadd_rn(s, static_cast<double>(R.v[j]));
    }
  }
  nflag = __reduce_add_sync(kFullF, nf);
  nentry = __reduce_add_sync(kFullF, ne);
  su = warp_sum_d(s);
}

// Entry flags (non-finite samples) of a row without a time pass.
template <int IN>
__device__ void wf_entry_only(const float* row, int T, uint32_t* Mrow, int& nflag, double& su) {
  const int lane = threadIdx.x & 31;
  int nf = 0;
  double s = 0.0;
  for (int w = lane; w < (T + 31) / 32; w += 32) {
    uint32_t m = 0u;
    for (int j = 0; j < 32 && 32 * w + j < T; ++j) {
      const float xv = fat<IN>(row, 32 * w + j);
      if (!isfinite(xv)) m |= 1u << j;
      else s = __dadd_rn(s, static_cast<double>(xv));
    }
    Mrow[w] = m;
    nf += __popc(m);
  }
  nflag = __reduce_add_sync(kFullF, nf);
  su = warp_sum_d(s);
}

// ---- one unit
template <int IN>
__device__ void f32_unit(const KParams& kp, const DevUnit& u, uint8_t* smem, F32Shared& f) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int C = u.C, T = u.T;
  double* S = reinterpret_cast<double*>(smem + kOffS);
  unsigned long long* srt = reinterpret_cast<unsigned long long*>(smem + kOffSrt);
  int* fin = reinterpret_cast<int*>(smem + kOffFin);
  uint8_t* Fc = smem + kOffFc;
  uint8_t* fire = smem + kOffFire;
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + kOffHist);
  const int nwr = (T + 31) / 32;
  uint32_t* Mrow = reinterpret_cast<uint32_t*>(smem + kOffRows) + warp * nwr;
  const bool vin = (u.flags & kUnitInVec) != 0;
  const float* gin = static_cast<const float*>(u.in);
  if (tid == 0) {
    f.cnt_time = f.cnt_total = f.cnt_hist = 0;
    f.ok = 1;
  }
  // a2: row sums of the finite samples (binary64)
  for (int c = warp; c < C; c += kNwF) {
    const float* row = gin + static_cast<int64_t>(c) * u.in_stride * (IN + 1);
    float hi = 0.f, lo = 0.f;
    int nfin = 0;
    for (int x0 = lane * 4; x0 < T; x0 += 4 * 128) {  // four loads in flight, then the sums in order
      float4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        v[k] = x0 + 128 * k < T ? ld4<IN>(row, x0 + 128 * k, T, vin) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = x0 + 128 * k;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float xv = f4at(v[k], j);
          if (x + j < T && isfinite(xv)) {
            df_add(hi, lo, xv);
            ++nfin;
          }
        }
      }
    }
    double s = __dadd_rn(static_cast<double>(hi), static_cast<double>(lo));
    if (__any_sync(kFullF, !df_ok(hi, lo))) {  // beyond the float32 range: binary64, same lanes and order
      s = 0.0;
      for (int x = lane * 4; x < T; x += 128) {
        const float4 v = ld4<IN>(row, x, T, vin);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float xv = f4at(v, j);
          if (x + j < T && isfinite(xv)) s = __dadd_rn(s, static_cast<double>(xv));
        }
      }
    }
    s = warp_sum_d(s);
    nfin = __reduce_add_sync(kFullF, nfin);
    if (lane == 0) {
      S[c] = s;
      fin[c] = nfin;
      Fc[c] = 0;
    }
  }
  __syncthreads();
  // a3, a4
  spectrum_stats(kp, S, C, srt, f);
  spectrum_sum_threshold(kp, S, C, Fc, fire, f);
  // a5
  long long np = 0;
  int nfc = 0;
  for (int c = tid; c < C; c += kNtF) {
    if (!Fc[c]) np += fin[c];
    nfc += Fc[c];
  }
  np = warp_sum_ll(np);
  nfc = __reduce_add_sync(kFullF, nfc);
  if (lane == 0) {
    srt[warp] = static_cast<unsigned long long>(np);
    fire[warp] = 0;
    reinterpret_cast<int*>(hist)[warp] = nfc;
  }
  __syncthreads();
  if (tid == 0) {
    long long t = 0;
    int tc = 0;
    for (int w = 0; w < kNwF; ++w) {
      t += static_cast<long long>(srt[w]);
      tc += reinterpret_cast<int*>(hist)[w];
    }
    f.n_pool = t;
    f.nfc = tc;
  }
  __syncthreads();
  double med = 0.0, sig = 0.0;
  if (f.n_pool > 0) {
    // two window passes around the previous block's median and MAD where
    // they hold the ranks, else the three radix passes
    double hm = 0.0, hd = 0.0;
    const bool hinted = f32_hints(kp, u, &hm, &hd);
    if (!(hinted && window_select<0, IN>(u, Fc, hist, f, hm, __dmul_rn(0.25, hd), &med)))
      med = select_median<0, IN>(u, Fc, hist, f);
    if (tid == 0) f.median_t = med;
    __syncthreads();
    double mad = 0.0;
    if (!kp.sigma_std) {
      if (!(hinted && window_select<1, IN>(u, Fc, hist, f, hd, __dmul_rn(0.25, hd), &mad)))
        mad = select_median<1, IN>(u, Fc, hist, f);
      if (tid == 0 && kp.hist.hint && u.hist_slot >= 0) {
        kp.hist.hint[2 * u.hist_slot] = static_cast<unsigned long long>(__double_as_longlong(med));
        kp.hist.hint[2 * u.hist_slot + 1] = static_cast<unsigned long long>(__double_as_longlong(mad));
      }
    }
    if (!kp.sigma_std && mad > 0.0) sig = __dmul_rn(1.482602218505602, mad);
    else sig = pooled_std<IN>(u, Fc, f);
  }
  if (tid == 0) {
    if (!f.ok) set_error_f(kp, kErrSelect, 700);
    f.median_t = med;
    f.sigma_t = sig;
    int kmax = 0;
    while (kmax < kp.max_log_window && (2 << kmax) <= T) ++kmax;
    f.kmax_t = kmax;
    f.time_on = (kp.enable_time && f.n_pool > 0 && sig > 0.0) ? 1 : 0;
    for (int k = 0; k <= kmax; ++k) {
      const double t = thr_of(kp, med, sig, k);
      f.tI[k] = t;
      f.tIf[k] = __double2float_rn(t);
      f.limI[k] = __double2float_rn(__dmul_rn(static_cast<double>(1 << k), t));
    }
  }
  __syncthreads();
  // a6 - a8, one warp per row
  const int nsg = wf_seg_count(T);
  const bool mask_vec = (u.flags & kUnitMaskVec) != 0;
  const bool vout = (u.flags & kUnitOutVec) != 0;
  const bool inplace = (u.flags & kUnitInPlace) != 0;
  for (int c = warp; c < C; c += kNwF) {
    const float* row = gin + static_cast<int64_t>(c) * u.in_stride * (IN + 1);
    const long long h = u.hist_slot >= 0 ? u.hist_slot + c : -1;
    bool full = Fc[c] != 0;
    int nflag = 0;
    if (!full) {
      int nentry = 0;
      double su = 0.0;
      if (f.time_on) {
        for (int sg = 0; sg < nsg; ++sg) {
          int a, b;
          double s;
          wf_segment<IN>(row, T, sg, vin, f, Mrow, a, b, s);
          nflag += a;
          nentry += b;
          su = __dadd_rn(su, s);
        }
      } else {
        wf_entry_only<IN>(row, T, Mrow, nflag, su);
        nentry = nflag;
      }
      __syncwarp();
      // a7: history (Section 4.1)
      const int n = T - nflag;
      bool fh = false;
      if (lane == 0) {
        if (n > 0) {
          const double cur = __ddiv_rn(su, static_cast<double>(n));
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
        atomicAdd(&f.cnt_time, static_cast<unsigned long long>(nflag - nentry));
        if (fh) atomicAdd(&f.cnt_hist, 1ull);
        atomicAdd(&f.cnt_total, fh ? static_cast<unsigned long long>(T)
                                   : static_cast<unsigned long long>(nflag));
      }
      full = __shfl_sync(kFullF, fh ? 1 : 0, 0) != 0;
    } else {
      if (lane == 0) {
        if (h >= 0) kp.hist.pend_flag[h] = 0;
        atomicAdd(&f.cnt_total, static_cast<unsigned long long>(T));
      }
    }
    // a8: mask and masked data (the input vectors of four chunks loaded ahead)
    const int64_t gi = c;
    const bool pf = IN == 0 && u.out && !inplace && vin && vout;
    for (int x0 = lane * 4; x0 < T; x0 += 4 * 128) {
    float4 pre[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (pf && x0 + 128 * k + 4 <= T && !full) pre[k] = __ldg(reinterpret_cast<const float4*>(row + x0 + 128 * k));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int x = x0 + 128 * k;
      if (x >= T) break;
      const int nv = min(4, T - x);
      const uint32_t valid = nv >= 4 ? 0xFu : ((1u << nv) - 1u);
      const uint32_t bits = full ? valid : ((Mrow[x >> 5] >> (x & 31)) & valid);
      if (u.mask) {
        uint8_t* mr = u.mask + gi * u.mask_stride;
        if (mask_vec && nv == 4) *reinterpret_cast<uint32_t*>(mr + x) = (bits * 0x00204081u) & 0x01010101u;
        else for (int j = 0; j < nv; ++j) mr[x + j] = static_cast<uint8_t>((bits >> j) & 1u);
      }
      if (u.out && IN == 1) {
        // complex samples: both floats of a flagged sample zeroed
        float* orow = static_cast<float*>(u.out) + gi * u.out_stride * 2;
        if (inplace) {
          for (int j = 0; j < nv; ++j)
            if ((bits >> j) & 1u) orow[2 * (x + j)] = orow[2 * (x + j) + 1] = 0.0f;
        } else if (vin && vout && nv == 4) {
          float4 a = __ldg(reinterpret_cast<const float4*>(row + 2 * x));
          float4 b = __ldg(reinterpret_cast<const float4*>(row + 2 * x + 4));
          if (bits & 1u) a.x = a.y = 0.0f;
          if (bits & 2u) a.z = a.w = 0.0f;
          if (bits & 4u) b.x = b.y = 0.0f;
          if (bits & 8u) b.z = b.w = 0.0f;
          __stcs(reinterpret_cast<float4*>(orow + 2 * x), a);
          __stcs(reinterpret_cast<float4*>(orow + 2 * x + 4), b);
        } else {
          for (int j = 0; j < nv; ++j) {
            const bool fl = (bits >> j) & 1u;
            orow[2 * (x + j)] = fl ? 0.0f : row[2 * (x + j)];
            orow[2 * (x + j) + 1] = fl ? 0.0f : row[2 * (x + j) + 1];
          }
        }
      } else if (u.out) {
        float* orow = static_cast<float*>(u.out) + gi * u.out_stride;
        if (inplace) {
          for (int j = 0; j < nv; ++j)
            if ((bits >> j) & 1u) orow[x + j] = 0.0f;
        } else if (vin && vout && nv == 4) {
          float4 w = full ? make_float4(0.f, 0.f, 0.f, 0.f) : pre[k];
          if (bits & 1u) w.x = 0.0f;
          if (bits & 2u) w.y = 0.0f;
          if (bits & 4u) w.z = 0.0f;
          if (bits & 8u) w.w = 0.0f;
          __stcs(reinterpret_cast<float4*>(orow + x), w);
        } else {
          for (int j = 0; j < nv; ++j) orow[x + j] = ((bits >> j) & 1u) ? 0.0f : row[x + j];
        }
      }
    }
    }
    __syncwarp();
  }
  __syncthreads();
  if (tid == 0 && u.stats) {
    u.stats->median_f = f.median_f;
    u.stats->sigma_f = f.sigma_f;
    u.stats->median_t = f.median_t;
    u.stats->sigma_t = f.sigma_t;
    u.stats->n_chan_freq = f.nfc;
    u.stats->n_flag_time = static_cast<long long>(f.cnt_time);
    u.stats->n_chan_hist = static_cast<long long>(f.cnt_hist);
    u.stats->n_flag_total = static_cast<long long>(f.cnt_total);
  }
  __syncthreads();
}

template <int IN>
__global__ void __launch_bounds__(kNtF, 2) lof_f32_kernel(const KParams kp) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ F32Shared f;
  for (int ui = blockIdx.x; ui < kp.n_units; ui += gridDim.x) {
    const DevUnit u = kp.units[ui];
    f32_unit<IN>(kp, u, smem, f);
  }
}


// One radix-select pass of the cluster (see select_pass): histograms of the
// CTA's own kept rows from shared memory, added over the cluster, then the
// digit of each open rank, picked identically in every CTA.
template <int MODE>
__device__ void cl_select_pass(cg::cluster_group& cl, const DevUnit& u, int r0, int R, const float* data,
                               const uint8_t* Fc, uint32_t* hist, uint32_t* tot, int shift, int nbits,
                               F32Shared& f) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = u.T, nb = 1 << nbits, P = cl_pitch(T);
  for (int i = tid; i < 2 * 2048; i += kNtF) hist[i] = 0u;
  __syncthreads();
  const uint32_t p0 = f.prefix[0], p1 = f.prefix[1];
  const int hs = shift + nbits;
  const bool two = f.n_rank == 2;
  const bool same = !two || p0 == p1;
  const float med_hi = __double2float_rn(f.median_t);
  const float med_lo = __double2float_rn(__dsub_rn(f.median_t, static_cast<double>(med_hi)));
  const int nchunk = (T + 127) / 128;
  for (int item = warp; item < R * nchunk; item += kNwF) {
    const int i = item / nchunk, s = item - i * nchunk;
    if (r0 + i >= u.C || Fc[r0 + i]) continue;
    const int x = s * 128 + lane * 4;
    if (x >= T) continue;
    const float4 v = ld4s(data + static_cast<size_t>(i) * P, x, T);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float xv = f4at(v, j);
      if (!isfinite(xv)) continue;
      const float kv = MODE == 0 ? xv : fabsf(__fsub_rn(__fsub_rn(xv, med_hi), med_lo));
      const uint32_t key = fkey(kv);
      const uint32_t hi = hs >= 32 ? 0u : (key >> hs);
      const uint32_t dig = (key >> shift) & static_cast<uint32_t>(nb - 1);
      if (hi == p0) atomicAdd(&hist[dig], 1u);
      if (!same && hi == p1) atomicAdd(&hist[2048 + dig], 1u);
    }
  }
  __syncthreads();
  cl_allreduce_hist(cl, hist, tot, same ? nb : 2048 + nb);
  if (warp < f.n_rank) {
    const uint32_t* h = tot + (same ? 0 : 2048 * warp);
    long long rk = f.rank[warp];
    long long base = 0;
    uint32_t digit = 0;
    bool found = false;
    for (int b0 = 0; b0 < nb && !found; b0 += 32) {
      const uint32_t cnt = h[b0 + lane];
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullF, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t tot_w = __shfl_sync(kFullF, incl, 31);
      if (rk < base + tot_w) {
        const unsigned hit = __ballot_sync(kFullF, rk < base + static_cast<long long>(incl));
        const int l = __ffs(hit) - 1;
        const uint32_t excl = __shfl_sync(kFullF, incl - cnt, l);
        digit = static_cast<uint32_t>(b0 + l);
        rk -= base + excl;
        found = true;
      } else {
        base += tot_w;
      }
    }
    if (lane == 0) {
      if (!found) f.ok = 0;
      f.prefix[warp] = (f.prefix[warp] << nbits) | digit;
      f.rank[warp] = rk;
    }
  }
  __syncthreads();
  if (tid == 0 && f.n_rank == 1) {
    f.prefix[1] = f.prefix[0];
    f.rank[1] = f.rank[0];
  }
  __syncthreads();
}

template <int MODE>
__device__ double cl_select_median(cg::cluster_group& cl, const DevUnit& u, int r0, int R, const float* data,
                                   const uint8_t* Fc, uint32_t* hist, uint32_t* tot, F32Shared& f) {
  const long long N = f.n_pool;
  if (threadIdx.x == 0) {
    f.prefix[0] = f.prefix[1] = 0u;
    f.rank[0] = (N & 1) ? N / 2 : N / 2 - 1;
    f.rank[1] = N / 2;
    f.n_rank = (N & 1) ? 1 : 2;
  }
  __syncthreads();
  cl_select_pass<MODE>(cl, u, r0, R, data, Fc, hist, tot, 21, 11, f);
  cl_select_pass<MODE>(cl, u, r0, R, data, Fc, hist, tot, 10, 11, f);
  cl_select_pass<MODE>(cl, u, r0, R, data, Fc, hist, tot, 0, 10, f);
  const double a = static_cast<double>(fkey_val(f.prefix[0]));
  const double b = static_cast<double>(fkey_val(f.prefix[1]));
  return (N & 1) ? a : __dmul_rn(__dadd_rn(a, b), 0.5);
}

// population stddev of the pooled finite samples: per CTA binary64 sums of
// its rows, added over the CTAs in rank order (two passes)
__device__ double cl_pooled_std(cg::cluster_group& cl, const DevUnit& u, int r0, int R, const float* data,
                                const uint8_t* Fc, double* red, F32Shared& f) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int CL = static_cast<int>(cl.num_blocks()), rank = static_cast<int>(cl.block_rank());
  const int T = u.T, P = cl_pitch(T);
  double acc[2] = {0.0, 0.0};
  double mu = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    double s = 0.0;
    for (int i = warp; i < R; i += kNwF) {
      if (r0 + i >= u.C || Fc[r0 + i]) continue;
      const float* row = data + static_cast<size_t>(i) * P;
      for (int t = lane; t < T; t += 32) {
        const float xv = row[t];
        if (!isfinite(xv)) continue;
        const double d = pass == 0 ? static_cast<double>(xv) : __dsub_rn(static_cast<double>(xv), mu);
        s = pass == 0 ? __dadd_rn(s, d) : __dadd_rn(s, __dmul_rn(d, d));
      }
    }
    s = warp_sum_d(s);
    if (lane == 0) f.red[warp] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kNwF; ++w) t = __dadd_rn(t, f.red[w]);
      for (int q = 0; q < CL; ++q) cl.map_shared_rank(red, q)[rank] = t;
    }
    cl.sync();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < CL; ++q) t = __dadd_rn(t, red[q]);
      f.red[0] = t;
    }
    __syncthreads();
    acc[pass] = f.red[0];
    cl.sync();  // red is reused by the next pass
    if (pass == 0) mu = __ddiv_rn(acc[0], static_cast<double>(f.n_pool));
  }
  return __dsqrt_rn(__ddiv_rn(acc[1], static_cast<double>(f.n_pool)));
}

// One unit per cluster; grid = units x CL CTAs, cluster dimension CL.
__global__ void __launch_bounds__(kNtF, 2) lof_f32c_kernel(const KParams kp) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ F32Shared f;
  cg::cluster_group cl = cg::this_cluster();
  const int CL = static_cast<int>(cl.num_blocks()), rank = static_cast<int>(cl.block_rank());
  const int ui = static_cast<int>(blockIdx.x) / CL;  // the same for every CTA of the cluster
  if (ui >= kp.n_units) return;
  const DevUnit u = kp.units[ui];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int C = u.C, T = u.T, P = cl_pitch(T), nwr = cl_words(T);
  const int R = (C + CL - 1) / CL, r0 = rank * R, nr = max(0, min(R, C - r0));
  double* S = reinterpret_cast<double*>(smem + kOffClS);
  unsigned long long* srt = reinterpret_cast<unsigned long long*>(smem + kOffClSrt);
  int* fin = reinterpret_cast<int*>(smem + kOffClFin);
  uint8_t* Fc = smem + kOffClFc;
  uint8_t* fire = smem + kOffClFire;
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + kOffClHist);
  uint32_t* tot = reinterpret_cast<uint32_t*>(smem + kOffClTot);
  double* red = reinterpret_cast<double*>(smem + kOffClRed);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smem + kOffClRed + 16 * 8);
  uint8_t* rinfo = smem + kOffClRows;
  uint32_t* Mrows = reinterpret_cast<uint32_t*>(smem + cl_off_mrow(R));
  float* data = reinterpret_cast<float*>(smem + cl_off_data(R, T));
  const bool vin = (u.flags & kUnitInVec) != 0;
  const float* gin = static_cast<const float*>(u.in);
  auto row_su = [&](int i) { return reinterpret_cast<double*>(rinfo + i * kClRowBytes); };
  auto row_int = [&](int i) { return reinterpret_cast<int*>(rinfo + i * kClRowBytes + kClMaxSeg * 8); };
  if (tid == 0) {
    f.cnt_time = f.cnt_total = f.cnt_hist = 0;
    f.ok = 1;
  }
  if (tid < 4) cnt[tid] = 0ull;
  // a1: the CTA's rows into shared memory, each sample read from global once
  for (int i = 0; i < nr; ++i) {
    const float* row = gin + static_cast<int64_t>(r0 + i) * u.in_stride;
    float* srow = data + static_cast<size_t>(i) * P;
    for (int x = tid * 4; x < T; x += kNtF * 4) {
      const float4 v = ld4<0>(row, x, T, vin);
      if (x + 4 <= T) {
        *reinterpret_cast<float4*>(srow + x) = v;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (x + j < T) srow[x + j] = f4at(v, j);
      }
    }
  }
  for (int i = tid; i < R * 4; i += kNtF) row_int(i >> 2)[i & 3] = 0;
  __syncthreads();
  // a2: row sums (binary64, one warp per row in f32_unit's order), written
  // into every CTA of the cluster
  for (int i = warp; i < nr; i += kNwF) {
    const float* srow = data + static_cast<size_t>(i) * P;
    float hi = 0.f, lo = 0.f;
    int nfin = 0;
    for (int x = lane * 4; x < T; x += 128) {
      const float4 v = ld4s(srow, x, T);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float xv = f4at(v, j);
        if (x + j < T && isfinite(xv)) {
          df_add(hi, lo, xv);
          ++nfin;
        }
      }
    }
    double s = __dadd_rn(static_cast<double>(hi), static_cast<double>(lo));
    if (__any_sync(kFullF, !df_ok(hi, lo))) {  // beyond the float32 range: binary64, same lanes and order
      s = 0.0;
      for (int x = lane * 4; x < T; x += 128) {
        const float4 v = ld4s(srow, x, T);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float xv = f4at(v, j);
          if (x + j < T && isfinite(xv)) s = __dadd_rn(s, static_cast<double>(xv));
        }
      }
    }
    s = warp_sum_d(s);
    nfin = __reduce_add_sync(kFullF, nfin);
    if (lane < CL) {
      cl.map_shared_rank(S, lane)[r0 + i] = s;
      cl.map_shared_rank(fin, lane)[r0 + i] = nfin;
    }
  }
  for (int c = tid; c < C; c += kNtF) Fc[c] = 0;
  cl.sync();
  // a3, a4 on the whole spectrum, alike in every CTA
  spectrum_stats(kp, S, C, srt, f);
  spectrum_sum_threshold(kp, S, C, Fc, fire, f);
  {
    long long np = 0;
    int nfc = 0;
    for (int c = tid; c < C; c += kNtF) {
      if (!Fc[c]) np += fin[c];
      nfc += Fc[c];
    }
    np = warp_sum_ll(np);
    nfc = __reduce_add_sync(kFullF, nfc);
    if (lane == 0) {
      srt[warp] = static_cast<unsigned long long>(np);
      srt[kNwF + warp] = static_cast<unsigned long long>(nfc);
    }
    __syncthreads();
    if (tid == 0) {
      long long t = 0, tc = 0;
      for (int w = 0; w < kNwF; ++w) {
        t += static_cast<long long>(srt[w]);
        tc += static_cast<long long>(srt[kNwF + w]);
      }
      f.n_pool = t;
      f.nfc = static_cast<int>(tc);
    }
    __syncthreads();
  }
  // a5
  double med = 0.0, sig = 0.0;
  if (f.n_pool > 0) {
    med = cl_select_median<0>(cl, u, r0, nr, data, Fc, hist, tot, f);
    if (tid == 0) f.median_t = med;
    __syncthreads();
    double mad = 0.0;
    if (!kp.sigma_std) mad = cl_select_median<1>(cl, u, r0, nr, data, Fc, hist, tot, f);
    if (!kp.sigma_std && mad > 0.0) sig = __dmul_rn(1.482602218505602, mad);
    else sig = cl_pooled_std(cl, u, r0, nr, data, Fc, red, f);
  }
  if (tid == 0) {
    if (!f.ok) set_error_f(kp, kErrSelect, 701);
    f.median_t = med;
    f.sigma_t = sig;
    int kmax = 0;
    while (kmax < kp.max_log_window && (2 << kmax) <= T) ++kmax;
    f.kmax_t = kmax;
    f.time_on = (kp.enable_time && f.n_pool > 0 && sig > 0.0) ? 1 : 0;
    for (int k = 0; k <= kmax; ++k) {
      const double t = thr_of(kp, med, sig, k);
      f.tI[k] = t;
      f.tIf[k] = __double2float_rn(t);
      f.limI[k] = __double2float_rn(__dmul_rn(static_cast<double>(1 << k), t));
    }
  }
  __syncthreads();
  // a6: time pass, warps over (own row, segment)
  const int nsg = wf_seg_count(T);
  if (f.time_on) {
    for (int item = warp; item < nr * nsg; item += kNwF) {
      const int i = item / nsg, sg = item - i * nsg;
      if (Fc[r0 + i]) continue;
      int a, b;
      double s;
      wf_segment<0, true>(data + static_cast<size_t>(i) * P, T, sg, true, f, Mrows + i * nwr, a, b, s);
      if (lane == 0) {
        row_su(i)[sg] = s;
        atomicAdd(&row_int(i)[0], a);
        atomicAdd(&row_int(i)[1], b);
      }
    }
  } else {
    for (int i = warp; i < nr; i += kNwF) {
      if (Fc[r0 + i]) continue;
      int nflag;
      double su;
      wf_entry_only<0>(data + static_cast<size_t>(i) * P, T, Mrows + i * nwr, nflag, su);
      if (lane == 0) {
        row_su(i)[0] = su;
        row_int(i)[0] = nflag;
        row_int(i)[1] = nflag;
      }
    }
  }
  __syncthreads();
  // a7: history (Section 4.1), one thread per own row
  if (tid < nr) {
    const int i = tid, c = r0 + i;
    const long long h = u.hist_slot >= 0 ? u.hist_slot + c : -1;
    int fh = 0;
    if (!Fc[c]) {
      const int nflag = row_int(i)[0], nentry = row_int(i)[1];
      double su = 0.0;
      for (int sg = 0; sg < (f.time_on ? nsg : 1); ++sg) su = __dadd_rn(su, row_su(i)[sg]);
      const int n = T - nflag;
      if (n > 0) {
        const double cur = __ddiv_rn(su, static_cast<double>(n));
        double staged = cur;
        if (kp.enable_history && h >= 0) {
          const int hc = kp.hist.count[h];
          if (hc >= kp.history_min && hc > 0) {
            const double thr = kp.hist.thr[h];
            if (!(cur < thr)) {
              fh = 1;
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
      atomicAdd(&f.cnt_time, static_cast<unsigned long long>(nflag - nentry));
      if (fh) atomicAdd(&f.cnt_hist, 1ull);
      atomicAdd(&f.cnt_total, fh ? static_cast<unsigned long long>(T) : static_cast<unsigned long long>(nflag));
    } else {
      if (h >= 0) kp.hist.pend_flag[h] = 0;
      atomicAdd(&f.cnt_total, static_cast<unsigned long long>(T));
      fh = 1;
    }
    row_int(i)[2] = fh;
  }
  __syncthreads();
  // a8: mask bytes and masked data of the own rows, the data from shared memory
  {
    const bool mask_vec = (u.flags & kUnitMaskVec) != 0;
    const bool vout = (u.flags & kUnitOutVec) != 0;
    const bool inplace = (u.flags & kUnitInPlace) != 0;
    const int nx = (T + 3) / 4;
    for (int item = tid; item < nr * nx; item += kNtF) {
      const int i = item / nx, x = (item - i * nx) * 4, c = r0 + i;
      const bool full = row_int(i)[2] != 0;
      const int nv = min(4, T - x);
      const uint32_t valid = nv >= 4 ? 0xFu : ((1u << nv) - 1u);
      const uint32_t bits = full ? valid : ((Mrows[i * nwr + (x >> 5)] >> (x & 31)) & valid);
      if (u.mask) {
        uint8_t* mr = u.mask + static_cast<int64_t>(c) * u.mask_stride;
        if (mask_vec && nv == 4) *reinterpret_cast<uint32_t*>(mr + x) = (bits * 0x00204081u) & 0x01010101u;
        else for (int j = 0; j < nv; ++j) mr[x + j] = static_cast<uint8_t>((bits >> j) & 1u);
      }
      if (u.out) {
        float* orow = static_cast<float*>(u.out) + static_cast<int64_t>(c) * u.out_stride;
        const float* srow = data + static_cast<size_t>(i) * P;
        if (inplace) {
          for (int j = 0; j < nv; ++j)
            if ((bits >> j) & 1u) orow[x + j] = 0.0f;
        } else if (vout && nv == 4) {
          float4 w = *reinterpret_cast<const float4*>(srow + x);
          if (bits & 1u) w.x = 0.0f;
          if (bits & 2u) w.y = 0.0f;
          if (bits & 4u) w.z = 0.0f;
          if (bits & 8u) w.w = 0.0f;
          __stcs(reinterpret_cast<float4*>(orow + x), w);
        } else {
          for (int j = 0; j < nv; ++j) orow[x + j] = ((bits >> j) & 1u) ? 0.0f : srow[x + j];
        }
      }
    }
  }
  // the unit's counts, added into CTA 0, which reports the statistics
  if (tid == 0) {
    unsigned long long* c0 = cl.map_shared_rank(cnt, 0);
    atomicAdd(c0 + 0, f.cnt_time);
    atomicAdd(c0 + 1, f.cnt_hist);
    atomicAdd(c0 + 2, f.cnt_total);
  }
  cl.sync();
  if (rank == 0 && tid == 0 && u.stats) {
    if (!f.ok) set_error_f(kp, kErrSelect, 702);
    u.stats->median_f = f.median_f;
    u.stats->sigma_f = f.sigma_f;
    u.stats->median_t = f.median_t;
    u.stats->sigma_t = f.sigma_t;
    u.stats->n_chan_freq = f.nfc;
    u.stats->n_flag_time = static_cast<long long>(cnt[0]);
    u.stats->n_chan_hist = static_cast<long long>(cnt[1]);
    u.stats->n_flag_total = static_cast<long long>(cnt[2]);
  }
}

}  // namespace
}  // namespace lofk

// Shared-memory bytes for units of up to n_time samples per row.
extern "C" int lofk_f32_smem(int max_T) {
  return lofk::kFixedBytesF + lofk::kNwF * ((max_T + 31) / 32) * 4;
}

// Float units: cplx = 0 Stokes I power, 1 complex float32 visibilities.
extern "C" int lofk_launch_f32x(const lofk::KParams* kp, int n_units, int n_sm, int smem_bytes,
                                void* stream, int cplx) {
  using namespace lofk;
  if (n_units <= 0) return 0;
  const void* k = cplx ? reinterpret_cast<const void*>(&lof_f32_kernel<1>)
                       : reinterpret_cast<const void*>(&lof_f32_kernel<0>);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) != cudaSuccess)
    return -2;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kNtF, smem_bytes) != cudaSuccess || occ < 1)
    return -3;
  const int grid = n_units < n_sm * occ ? n_units : n_sm * occ;
  void* args[] = {const_cast<KParams*>(kp)};
  const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(kNtF), args, static_cast<size_t>(smem_bytes),
                                         static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? 0 : static_cast<int>(e);
}

extern "C" int lofk_launch_f32(const lofk::KParams* kp, int n_units, int n_sm, int smem_bytes,
                               void* stream) {
  return lofk_launch_f32x(kp, n_units, n_sm, smem_bytes, stream, 0);
}

// Stokes I units in thread-block clusters (lof_f32c_kernel): 0 launched, 1
// not possible for these units on this device (the caller takes the one-CTA
// kernel), else a CUDA error code.  max_C, max_T: the largest unit.
extern "C" int lofk_launch_f32c(const lofk::KParams* kp, int n_units, int max_C, int max_T, void* stream) {
  using namespace lofk;
  if (n_units <= 0) return 0;
  if (max_C > kCMaxCl || max_C < 1) return 1;
  {
    int n = 1, ob = (32 * kNplF - kHaloF) & ~31;
    while (ob < max_T) {
      const int s0 = (ob - kHaloF) & ~31;
      ob = s0 + 32 * kNplF >= max_T ? max_T : ((s0 + 32 * kNplF - kHaloF) & ~31);
      ++n;
    }
    if (n > kClMaxSeg) return 1;
  }
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const void* k = reinterpret_cast<const void*>(&lof_f32c_kernel);
  for (int CL : {16, 8}) {
    const int R = (max_C + CL - 1) / CL;
    const int smem = cl_smem(R, max_T);
    if (smem + static_cast<int>(sizeof(F32Shared)) + 1024 > optin) continue;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        (CL > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(n_units * CL));
    cfg.blockDim = dim3(kNtF);
    cfg.dynamicSmemBytes = static_cast<size_t>(smem);
    cfg.stream = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = static_cast<unsigned>(CL);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k, &cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      continue;
    }
    const cudaError_t e = cudaLaunchKernelEx(&cfg, lof_f32c_kernel, *kp);
    return e == cudaSuccess ? 0 : static_cast<int>(e);
  }
  return 1;
}
