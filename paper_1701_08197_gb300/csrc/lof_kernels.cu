// lof_kernels.cu -- sm_103a kernels of the LOFAR Online Flagger hot path.
//
// One persistent, cooperatively launched kernel flags every unit of a block
// (one unit = one station/polarisation/subband: C channels x T samples).
// Each CTA repeatedly takes an "item" (a run of whole rows of one unit) from a
// device queue, stages the rows in shared memory with cp.async.bulk and keeps
// them there for the whole pipeline, so every input byte crosses HBM once.
// The unit-wide steps are resolved by the CTAs of a unit through bounded
// group barriers; the last CTA to arrive at a round does the unit-wide work:
//   round 1   row power sums -> spectrum S[c] -> median / MAD of S ->
//             SumThreshold over S (Section 4: frequency flagging first)
//   round 2   coarse histogram of the pooled powers of the kept channels
//   round 3+  exact counts inside the few bins holding the median and the MAD
//             end points, until both are exact (Section 4.2: O(N), no sort)
// Then every CTA runs SumThreshold along time on its rows (Section 2.1, all
// window sizes over a shared-memory prefix array), the history test
// (Section 4.1), and writes the mask and the masked data.
//
// Integer inputs are exact end to end: powers and (window) sums are integers,
// and each threshold is the binary64 formula of Section 2.1 turned into an
// integer table K[n] = floor((I - n) * threshold_I) for n flagged samples.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "lof_internal.h"

// The task bodies of the complex-int8 kernel are separate functions: its
// wider unpacking of 16-byte vectors otherwise exhausts the register budget
// of the inlined whole (spills); the int16 kernel inlines them.
#if defined(LOF_KERNEL_DT) && LOF_KERNEL_DT == 1
#define LOFK_TASK_FN __noinline__
#else
#define LOFK_TASK_FN __forceinline__
#endif

namespace lofk {
namespace {

constexpr int kWarp = 32;

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(b))
      : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(saddr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------------------ sample types
// Power of one complex sample (Section 4: amplitudes first).  re^2 + im^2 of
// int8/int16 components is exact in 32 bits (at most 2^31).

template <int DT>
struct Traits;

template <>
struct Traits<LOF_CI16> {
  static constexpr int kBytes = 4;
  static constexpr int kVec = 4;  // samples per 16-byte vector
  __device__ static __forceinline__ uint32_t pw(uint32_t w) {
    const int re = static_cast<int>(static_cast<int16_t>(w & 0xFFFFu));
    const int im = static_cast<int>(static_cast<int16_t>(w >> 16));
    return static_cast<uint32_t>(re * re) + static_cast<uint32_t>(im * im);
  }
  __device__ static __forceinline__ uint32_t at(const uint8_t* row, int t) {
    return pw(reinterpret_cast<const uint32_t*>(row)[t]);
  }
  __device__ static __forceinline__ void vec(const uint8_t* row, int x, uint32_t (&v)[kVec]) {
    const uint4 w = *reinterpret_cast<const uint4*>(row + static_cast<size_t>(x) * kBytes);
    v[0] = pw(w.x);
    v[1] = pw(w.y);
    v[2] = pw(w.z);
    v[3] = pw(w.w);
  }
  __device__ static __forceinline__ void zero(uint8_t* row, int t) {
    reinterpret_cast<uint32_t*>(row)[t] = 0u;
  }
  __device__ static __forceinline__ void copy(uint8_t* dst, const uint8_t* src) {
    *reinterpret_cast<uint32_t*>(dst) = *reinterpret_cast<const uint32_t*>(src);
  }
};

template <>
struct Traits<LOF_CI8> {
  static constexpr int kBytes = 2;
  static constexpr int kVec = 8;
  __device__ static __forceinline__ uint32_t pw(uint32_t h) {
    // re^2 + im^2 as one signed byte-wise dot product (upper bytes zero)
    const int b = static_cast<int>(h & 0xFFFFu);
    return static_cast<uint32_t>(__dp4a(b, b, 0));
  }
  __device__ static __forceinline__ uint32_t at(const uint8_t* row, int t) {
    return pw(reinterpret_cast<const uint16_t*>(row)[t]);
  }
  __device__ static __forceinline__ void vec(const uint8_t* row, int x, uint32_t (&v)[kVec]) {
    const uint4 w = *reinterpret_cast<const uint4*>(row + static_cast<size_t>(x) * kBytes);
    v[0] = pw(w.x);
    v[1] = pw(w.x >> 16);
    v[2] = pw(w.y);
    v[3] = pw(w.y >> 16);
    v[4] = pw(w.z);
    v[5] = pw(w.z >> 16);
    v[6] = pw(w.w);
    v[7] = pw(w.w >> 16);
  }
  __device__ static __forceinline__ void zero(uint8_t* row, int t) {
    reinterpret_cast<uint16_t*>(row)[t] = 0;
  }
  __device__ static __forceinline__ void copy(uint8_t* dst, const uint8_t* src) {
    *reinterpret_cast<uint16_t*>(dst) = *reinterpret_cast<const uint16_t*>(src);
  }
};

// Powers of samples [x, x + kVec) of a staged row; zero at or beyond T.
template <int DT>
__device__ __forceinline__ void load_vec(const uint8_t* row, int x, int T,
                                         uint32_t (&v)[Traits<DT>::kVec]) {
  if (x + Traits<DT>::kVec <= T) {
    Traits<DT>::vec(row, x, v);
  } else {
#pragma unroll
    for (int j = 0; j < Traits<DT>::kVec; ++j)
      v[j] = (x + j < T) ? Traits<DT>::at(row, x + j) : 0u;
  }
}

// ------------------------------------------------------------------ small helpers

// Coarse key of a 32-bit value: the top bits of its binary32 value rounded
// toward zero (exponent and 5 mantissa bits), i.e. 32 bins per octave and
// one bin per integer below 64.  Key 0 holds the value 0; keys 1..31 are
// empty; the largest key is 1055.
constexpr int kKeyBias = 4032;  // (127 - 1) << 5
__device__ __forceinline__ uint32_t coarse_key(uint32_t v) {
  const int k = static_cast<int>(__float_as_uint(__uint2float_rz(v)) >> 18) - kKeyBias;
  return static_cast<uint32_t>(max(k, 0));
}
// Smallest integer v with coarse_key(v) >= k (k >= 1); 2^32 for k = 1056.
__device__ __forceinline__ unsigned long long key_floor(uint32_t k) {
  const float fv = __uint_as_float((k + static_cast<uint32_t>(kKeyBias)) << 18);
  return static_cast<unsigned long long>(ceil(static_cast<double>(fv)));
}
// Integer range [lo, hi] of key k; false when the key holds no integer.
__device__ __forceinline__ bool key_range(uint32_t k, uint32_t* lo, uint32_t* hi) {
  const unsigned long long a = (k == 0) ? 0ull : key_floor(k);
  const unsigned long long b = key_floor(k + 1);
  if (a >= b) return false;
  *lo = static_cast<uint32_t>(a);
  *hi = static_cast<uint32_t>(b - 1ull);
  return true;
}

// Index of prefix entry x in the padded prefix layout (4 spare words after
// every 32): threads reading consecutive 32-word chunks hit distinct banks.
__device__ __forceinline__ int pidx(int x) { return x + ((x >> 5) << 2); }

__device__ __forceinline__ int round_up(int x, int m) { return (x + m - 1) / m * m; }

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}
__device__ __forceinline__ uint32_t warp_max32(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}
__device__ __forceinline__ uint32_t warp_sum32(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}
// exclusive warp scan (u32, wrapping); *total = sum over the warp
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, int lane, uint32_t* total) {
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  *total = __shfl_sync(0xFFFFFFFFu, x, 31);
  return x - v;
}

// u128 -> binary64, round to nearest even.
__device__ __forceinline__ double u128_to_double(unsigned __int128 m) {
  const unsigned long long hi = static_cast<unsigned long long>(m >> 64);
  const unsigned long long lo = static_cast<unsigned long long>(m);
  if (hi == 0) return __ull2double_rn(lo);
  const int s = __clzll(static_cast<long long>(hi));
  unsigned long long top = s ? ((hi << s) | (lo >> (64 - s))) : hi;
  const unsigned long long rest = s ? (lo << s) : lo;
  top |= (rest != 0ull) ? 1ull : 0ull;
  return ldexp(__ull2double_rn(top), 64 - s);
}

// Population stddev from exact moments: sqrt((N*S2 - S1^2) / N^2).
__device__ double moments_std(long long n, unsigned __int128 s1, unsigned __int128 s2) {
  if (n <= 0) return 0.0;
  const unsigned __int128 M = static_cast<unsigned __int128>(n) * s2 - s1 * s1;
  const double nn = __dmul_rn(static_cast<double>(n), static_cast<double>(n));
  return __dsqrt_rn(__ddiv_rn(u128_to_double(M), nn));
}

__device__ __forceinline__ int koffset(int k) { return (1 << k) + k - 1; }  // sum_{j<k}(2^j+1)

// Section 2.1: threshold_I = median + stddev * factor_I * sensitivity and its
// integer table K[n] = floor((I - n) * threshold_I), n = 0..I, for I = 2^k,
// k <= kmax; one entry per thread of the calling CTA (no barrier inside).
template <int NT>
__device__ void fill_ktable(const KParams& kp, double median, double sigma, int kmax,
                            long long* K) {
  const int total = koffset(kmax + 1);
  for (int e = threadIdx.x; e < total; e += NT) {
    int k = 0;
    while (koffset(k + 1) <= e) ++k;
    const int I = 1 << k, n = e - koffset(k);
    const double thr =
        __dadd_rn(median, __dmul_rn(__dmul_rn(sigma, kp.factor[k]), kp.sensitivity));
    const double lim = __dmul_rn(static_cast<double>(I - n), thr);
    long long q;
    if (!(lim == lim)) q = (1ll << 62);  // NaN threshold: never fires
    else if (lim >= 4.0e18) q = (1ll << 62);
    else if (lim <= -4.0e18) q = -(1ll << 62);
    else q = __double2ll_rd(lim);
    K[e] = q;
  }
}


__device__ void set_error(const KParams& kp, int code, int info) {
  if (atomicCAS(kp.err, 0, code) == 0) {
    kp.err_info[0] = info;
    kp.err_info[1] = static_cast<int>(blockIdx.x);
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until *p >= v (another CTA of this launch releases it).  Gives
// up after kp.spin_limit nanoseconds, or as soon as another CTA reported an
// error, and records a timeout.
__device__ bool wait_geq(const KParams& kp, const int* p, int v, int code_info) {
  const unsigned long long t0 = global_ns();
  while (ld_acquire(p) < v) {
    if (*reinterpret_cast<volatile int*>(kp.err) != 0) return false;
    if (global_ns() - t0 > static_cast<unsigned long long>(kp.spin_limit)) {
      set_error(kp, kErrTimeout, code_info);
      return false;
    }
    __nanosleep(128);
  }
  return true;
}

// Bitonic sort of n (power of two) u64 values in shared memory, ascending.
template <int NT>
__device__ void block_sort64(unsigned long long* a, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += NT) {
        const int p = i ^ j;
        if (p > i) {
          const unsigned long long x = a[i], y = a[p];
          const bool asc = (i & k) == 0;
          if ((x > y) == asc) {
            a[i] = y;
            a[p] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// 128-bit add into a pair of 64-bit words (lo, hi) in global memory.
__device__ __forceinline__ void atomic_add_u128(unsigned long long* lohi, unsigned __int128 v) {
  const unsigned long long vl = static_cast<unsigned long long>(v);
  const unsigned long long vh = static_cast<unsigned long long>(v >> 64);
  const unsigned long long old = atomicAdd(lohi, vl);
  const unsigned long long carry = (old + vl < old) ? 1ull : 0ull;
  if (vh + carry) atomicAdd(lohi + 1, vh + carry);
}

// Offset-map entry of a coarse key that holds no target: val + kNoTarget >=
// 2^31 - 1 for every power (at most 2^31), beyond any spec index.
constexpr uint32_t kNoTarget = 0x7FFFFFFFu;

__device__ __forceinline__ Target ld_target(const Target* p) {
  const uint4 v = __ldcg(reinterpret_cast<const uint4*>(p));
  return Target{v.x, v.y, v.z, v.w};
}

// Coarse bins around the previous block's median and MAD end points, to be
// counted value by value while the stats tasks run.  For each point p of
// m - d, m, m + d (d = MAD) the bins overlapping [p - w, p + w] with
// w = max(2, d / 4, p / 32), at most kSpecHalf: between blocks the pooled
// median and MAD move by a fraction of d (a burst that covers a few percent
// of a unit's samples shifts them by about a tenth of d), so the order
// statistics normally land inside these bins and round 1 resolves them.
// Bins in increasing order, none twice; the list stops where kMaxSpec
// counters or kMaxTargets bins are used.  Deterministic in (m2, mad4): every
// task of a unit derives the same list.  One whole warp; returns the number
// of bins in every lane.
__device__ int spec_targets(unsigned long long m2, unsigned long long mad4, Target* tg) {
  const int lane = threadIdx.x & 31;
  if (m2 == ~0ull) return 0;
  const long long m = static_cast<long long>(m2 >> 1), d = static_cast<long long>(mad4 >> 2);
  const long long P[3] = {m - d, m, m + d};
  int nt = 0;
  uint32_t base = 0;
  long long last_hi = -1;  // highest value covered so far
  for (int i = 0; i < 3; ++i) {
    const long long p = P[i] < 0 ? 0 : P[i];
    if (p > 0xFFFFFFFFll) break;
    long long del = max(2ll, max(d / 4, p / 32));
    if (del > kSpecHalf) del = kSpecHalf;
    const long long a = p - del < 0 ? 0 : p - del;
    const long long b = p + del > 0xFFFFFFFFll ? 0xFFFFFFFFll : p + del;
    const uint32_t k0 = coarse_key(static_cast<uint32_t>(a)), k1 = coarse_key(static_cast<uint32_t>(b));
    for (uint32_t kb = k0; kb <= k1; kb += kWarp) {
      const uint32_t k = kb + lane;
      uint32_t lo = 0, hi = 0;
      const bool ok = k <= k1 && key_range(k, &lo, &hi) && static_cast<long long>(lo) > last_hi;
      const uint32_t w = ok ? hi - lo + 1u : 0u;
      uint32_t tot;
      const uint32_t ex = warp_excl_scan(w, lane, &tot);
      const unsigned okb = __ballot_sync(0xFFFFFFFFu, ok);
      const int rank = __popc(okb & ((1u << lane) - 1u));
      // the ok lanes in order: a prefix of them fits (widths are positive)
      const bool fits = ok && base + ex + w <= static_cast<uint32_t>(kMaxSpec) && nt + rank < kMaxTargets;
      if (fits) tg[nt + rank] = Target{lo, hi, 0u, base + ex};
      const unsigned fb = __ballot_sync(0xFFFFFFFFu, fits);
      const int nfit = __popc(fb);
      if (nfit > 0) {
        const int top = 31 - __clz(static_cast<int>(fb));
        last_hi = static_cast<long long>(__shfl_sync(0xFFFFFFFFu, hi, top));
        base += __shfl_sync(0xFFFFFFFFu, ex + w, top);
      }
      nt += nfit;
      if (nfit < __popc(okb)) return nt;  // full
    }
  }
  return nt;
}

// Value window of a unit (statistics counted value by value): the kWinVals
// values around the previous block's median m (hint 2m, 4d), starting at 1 or
// later and ending at 2^31 or earlier, chosen when m - d and m + d lie inside
// it with a margin of max(64, d / 2) on each side -- between blocks the
// pooled median and MAD move by a small fraction of d.
// Deterministic in the hint, so every task of a unit and its round 1 agree.
constexpr uint32_t kWinVals = kMaxSpec;
__device__ __forceinline__ bool hint_window(unsigned long long m2, unsigned long long mad4, uint32_t* lo) {
  if (m2 == ~0ull) return false;
  const long long m = static_cast<long long>(m2 >> 1), d = static_cast<long long>(mad4 >> 2);
  const long long margin = d / 2 > 64 ? d / 2 : 64;
  if (2 * (d + margin) > static_cast<long long>(kWinVals)) return false;
  long long a = m - static_cast<long long>(kWinVals / 2);
  const long long top = 0x80000000ll - static_cast<long long>(kWinVals);
  if (a < 1) a = 1;  // the value 0, if any, counts as below the window
  if (a > top) return false;
  *lo = static_cast<uint32_t>(a);
  return true;
}

// ------------------------------------------------------------------ shared state

template <int NT>
struct Fixed {
  uint64_t mbar;
  int item, ok, last, state, n_keep, n_tgt, q_done, n_def, rows_done;
  int row_next;  // flag task: next (kept row, segment) item to hand out (warps claim items as they go)
  int def[9];  // parked tasks whose unit was not ready
  unsigned int red_u32[NT / kWarp];
  unsigned long long red_a[NT / kWarp], red_b[NT / kWarp], red_c[NT / kWarp];
  unsigned long long cnt_time, cnt_total, cnt_hist;
  unsigned long long mo1, mo2lo, mo2hi;  // moments of this CTA's rows
  unsigned long long rowS[kMaxRowsPerTask];
  unsigned long long rowFlagSum[kMaxRowsPerTask];  // flagged sum (general path), unflagged (packed)
  int rowNFlag[kMaxRowsPerTask];
  uint8_t rowFc[kMaxRowsPerTask];
  uint8_t rowFh[kMaxRowsPerTask];
  uint8_t rowHon[kMaxRowsPerTask];   // the row's history threshold applies (count >= history_min)
  double rowThr[kMaxRowsPerTask];    // that threshold (mean + k * stddev of the ring)
  int keep[kMaxRowsPerTask];
  long long K[kKTable];
  double median_t, sigma_t;
  int time_on, kmax_t;
  Target tgt[kMaxTargets];
  // last-arriver scratch
  long long m2lo, m2hi, da[2], db[2];
  int mb[2], resolved, tb[kMaxTargets], nnz[kMaxTargets];
  int wmode;                  // value-window statistics for this unit
  uint32_t wlo;               // first value of the window
  long long wbelow;           // kept samples below the window
  unsigned long long sd, md4;
  unsigned long long sel1, sel2;  // order statistics of the spectrum (rank selection)
  double sig;
  int kmax_f;
};

// ------------------------------------------------------------------ round 1
// Order statistics r1 <= r2 of n <= 2 NT values (whole CTA): each value's
// rank is counted against all n (ties by index), and the values of ranks r1
// and r2 are written to *o1, *o2.
template <int NT>
__device__ void rank_select2(const unsigned long long* v, int n, int r1, int r2, unsigned long long* o1,
                             unsigned long long* o2) {
  for (int i = threadIdx.x; i < n; i += NT) {
    const unsigned long long x = v[i];
    int rk = 0;
#pragma unroll 8
    for (int j = 0; j < n; ++j) {
      const unsigned long long y = v[j];
      rk += (y < x || (y == x && j < i)) ? 1 : 0;
    }
    if (rk == r1) *o1 = x;
    if (rk == r2) *o2 = x;
  }
  __syncthreads();
}

// Frequency pass, run by the CTA that completes round 1 of a unit: median and
// robust sigma of the spectrum and SumThreshold over it (Section 4).
// Needs 36 KB of shared workspace.
template <int NT>
__device__ void frequency_pass(const KParams& kp, const DevUnit& u, UnitState* slot, uint8_t* ws,
                               Fixed<NT>& f) {
  const int tid = threadIdx.x;
  const int C = u.C;
  int n2 = 1;
  while (n2 < C) n2 <<= 1;
  unsigned long long* srt = reinterpret_cast<unsigned long long*>(ws);  // kMaxChan
  unsigned long long* Sv = srt + kMaxChan;                               // kMaxChan
  // fire flags [32K, 34K); Fc [34K, 36K) is kept for round 1
  uint8_t* Fc = reinterpret_cast<uint8_t*>(Sv + kMaxChan) + kMaxChan;
  const unsigned long long* gS = kp.chan_S + u.chan_off;
  for (int i = tid; i < n2; i += NT) {
    unsigned long long v = ~0ull;
    if (i < C) {
      v = __ldcg(gS + i);
      Sv[i] = v;
      Fc[i] = 0;
    }
    srt[i] = v;
  }
  __syncthreads();
  // the middle order statistics: counted ranks for up to 2 NT channels, else a sort
  const bool ranks = C <= 2 * NT;
  if (ranks) {
    rank_select2<NT>(Sv, C, (C - 1) / 2, C / 2, &f.sel1, &f.sel2);
    if (tid == 0) f.sd = (C & 1) ? 2ull * f.sel2 : f.sel1 + f.sel2;
  } else {
    block_sort64<NT>(srt, n2);
    if (tid == 0) f.sd = (C & 1) ? 2ull * srt[C / 2] : srt[C / 2 - 1] + srt[C / 2];
  }
  __syncthreads();
  const unsigned long long M2 = f.sd;  // twice the median of S
  for (int i = tid; i < n2; i += NT) {
    unsigned long long d = ~0ull;
    if (i < C) {
      const unsigned long long x2 = 2ull * Sv[i];
      d = x2 > M2 ? x2 - M2 : M2 - x2;
    }
    srt[i] = d;
  }
  __syncthreads();
  if (ranks) rank_select2<NT>(srt, C, (C - 1) / 2, C / 2, &f.sel1, &f.sel2);
  else block_sort64<NT>(srt, n2);
  if (tid == 0) {
    // 4 x MAD: the median of |2S - M2| counted twice
    f.md4 = ranks ? ((C & 1) ? 2ull * f.sel2 : f.sel1 + f.sel2)
                  : ((C & 1) ? 2ull * srt[C / 2] : srt[C / 2 - 1] + srt[C / 2]);
    const double med = __dmul_rn(__ull2double_rn(M2), 0.5);
    const double mad = __dmul_rn(__ull2double_rn(f.md4), 0.25);
    double sig;
    if (!kp.sigma_std && mad > 0.0) {
      sig = __dmul_rn(1.482602218505602, mad);
    } else {
      unsigned __int128 s1 = 0, s2 = 0;
      for (int i = 0; i < C; ++i) {
        s1 += Sv[i];
        s2 += static_cast<unsigned __int128>(Sv[i]) * Sv[i];
      }
      sig = moments_std(C, s1, s2);
    }
    f.sig = sig;
    slot->median_f = med;
    slot->sigma_f = sig;
    int kmax = 0;
    while (kmax < kp.max_log_window && (2 << kmax) <= C) ++kmax;
    f.kmax_f = kmax;
  }
  __syncthreads();
  fill_ktable<NT>(kp, __dmul_rn(__ull2double_rn(M2), 0.5), f.sig, f.kmax_f, f.K);
  __syncthreads();
  const double sig = f.sig;
  const int kmax = f.kmax_f;
  // Section 2.1 over the spectrum: direct window sums (C <= 2048 values)
  if (kp.enable_freq && sig > 0.0) {
    uint8_t* fire = Fc - kMaxChan;  // [32K, 34K)
    for (int k = 0; k <= kmax; ++k) {
      const int I = 1 << k;
      const long long* Kt = f.K + koffset(k);
      for (int t = tid; t < C; t += NT) {
        uint8_t fl = 0;
        if (t + I <= C) {
          unsigned long long su = 0;
          int nf = 0;
          for (int j = t; j < t + I; ++j) {
            if (Fc[j]) ++nf;
            else su += Sv[j];
          }
          fl = static_cast<long long>(su) > Kt[nf] ? 1 : 0;
        }
        fire[t] = fl;
      }
      __syncthreads();
      for (int c = tid; c < C; c += NT) {
        uint8_t any = Fc[c];
        const int lo = c - I + 1 < 0 ? 0 : c - I + 1;
        for (int t = lo; t <= c && !any; ++t) any = fire[t];
        Fc[c] = any;
      }
      __syncthreads();
    }
  }
  int nfc = 0;
  for (int c = tid; c < C; c += NT) {
    kp.chan_Fc[u.chan_off + c] = Fc[c];
    nfc += Fc[c];
  }
  nfc = __reduce_add_sync(0xFFFFFFFFu, nfc);
  if ((tid & 31) == 0) f.red_u32[tid >> 5] = static_cast<unsigned>(nfc);
  for (int i = tid; i < kMaxFine; i += NT) slot->fine[i] = 0;
  __syncthreads();
  if (tid == 0) {
    int tot = 0;
    for (int w = 0; w < NT / kWarp; ++w) tot += static_cast<int>(f.red_u32[w]);
    slot->n_chan_freq = tot;
    slot->n_pool = static_cast<long long>(C - tot) * u.T;
    slot->mom_ready = 0;
    slot->round = 1;
    slot->n_bins = 0;
    slot->n_targets = 0;
    slot->n_fine = 0;
    slot->median_t = 0.0;
    slot->sigma_t = 0.0;
    slot->time_on = 0;
    slot->state = slot->n_pool > 0 ? kStateCoarse : kStateDone;
    if (u.stats) {
      u.stats->median_f = slot->median_f;
      u.stats->sigma_f = slot->sigma_f;
      u.stats->median_t = 0.0;
      u.stats->sigma_t = 0.0;
      u.stats->n_chan_freq = tot;
      u.stats->n_flag_time = 0;
      u.stats->n_chan_hist = 0;
      u.stats->n_flag_total = 0;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ exact selection
// The pooled values are described by a sorted list of disjoint non-empty bins
// [lo, hi] with counts.  An order statistic is exact once its bin has width 1.
// The MAD is the r-th smallest |2x - M2| (M2 = twice the median); for a
// distance d, c(d) = #{x : ceil((M2-d)/2) <= x <= floor((M2+d)/2)} is bounded
// from both sides by the bins, which brackets d* = min{d : c(d) >= r+1}.

struct BinList {
  const uint32_t* lo;
  const uint32_t* hi;
  const uint32_t* cum;  // n + 1 entries, cum[0] = 0
  int n;
};

// values in bins with lo <= y (an upper bound of #{x <= y})
__device__ __forceinline__ long long cnt_upper(const BinList& B, long long y) {
  if (y < 0) return 0;
  int a = 0, b = B.n;
  while (a < b) {
    const int m = (a + b) >> 1;
    if (static_cast<long long>(B.lo[m]) <= y) a = m + 1;
    else b = m;
  }
  return B.cum[a];
}
// values in bins with hi <= y (a lower bound of #{x <= y})
__device__ __forceinline__ long long cnt_lower(const BinList& B, long long y) {
  if (y < 0) return 0;
  int a = 0, b = B.n;
  while (a < b) {
    const int m = (a + b) >> 1;
    if (static_cast<long long>(B.hi[m]) <= y) a = m + 1;
    else b = m;
  }
  return B.cum[a];
}
__device__ __forceinline__ long long endA(long long M2, long long d) {
  const long long t = M2 - d;
  return t <= 0 ? 0 : (t + 1) >> 1;
}
__device__ __forceinline__ long long endB(long long M2, long long d) {
  const long long t = (M2 + d) >> 1;
  return t > 0xFFFFFFFFll ? 0xFFFFFFFFll : t;
}
__device__ __forceinline__ long long c_hi(const BinList& B, long long m2lo, long long m2hi,
                                          long long d) {
  return cnt_upper(B, endB(m2hi, d)) - cnt_lower(B, endA(m2lo, d) - 1);
}
__device__ __forceinline__ long long c_lo(const BinList& B, long long m2lo, long long m2hi,
                                          long long d) {
  const long long a = endA(m2hi, d), b = endB(m2lo, d);
  if (a > b) return 0;
  const long long v = cnt_lower(B, b) - cnt_upper(B, a - 1);
  return v < 0 ? 0 : v;
}
// warp-wide 33-ary search: smallest d in [0, 2^34] with F(d) >= target (F monotone)
template <bool HI>
__device__ long long warp_search(const BinList& B, long long m2lo, long long m2hi,
                                 long long target, int lane) {
  long long lo = -1, hi = (1ll << 34);
  while (hi - lo > 1) {
    const long long span = hi - lo;
    const long long d = lo + (span * (lane + 1)) / 33;
    bool ok = false;
    if (d > lo && d < hi) {
      const long long cd = HI ? c_hi(B, m2lo, m2hi, d) : c_lo(B, m2lo, m2hi, d);
      ok = cd >= target;
    } else if (d >= hi) {
      ok = true;
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, ok);
    if (bal == 0u) {
      lo = __shfl_sync(0xFFFFFFFFu, d, 31);
    } else {
      const int j = __ffs(bal) - 1;
      const long long dj = __shfl_sync(0xFFFFFFFFu, d, j);
      const long long dp = __shfl_sync(0xFFFFFFFFu, d, j > 0 ? j - 1 : 0);
      if (dj < hi) hi = dj;
      if (j > 0 && dp > lo) lo = dp;
    }
  }
  return hi;
}

// Copies the slot's bin list to shared memory and forms cumulative counts.
template <int NT>
__device__ BinList load_bins(const UnitState* slot, uint8_t* ws, int n) {
  uint32_t* lo = reinterpret_cast<uint32_t*>(ws);
  uint32_t* hi = lo + kSelCap;
  uint32_t* cum = hi + kSelCap;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += NT) {
    lo[i] = __ldcg(slot->blo + i);
    hi[i] = __ldcg(slot->bhi + i);
    cum[i + 1] = __ldcg(slot->bcnt + i);
  }
  if (tid == 0) cum[0] = 0;
  __syncthreads();
  if (tid < kWarp) {
    uint32_t carry = 0;
    for (int base = 0; base < n; base += kWarp) {
      const int i = base + tid;
      const uint32_t v = i < n ? cum[i + 1] : 0u;
      uint32_t tot;
      const uint32_t ex = warp_excl_scan(v, tid, &tot);
      if (i < n) cum[i + 1] = carry + ex + v;
      carry += tot;
    }
  }
  __syncthreads();
  return BinList{lo, hi, cum, n};
}

__device__ __forceinline__ int bin_of_rank(const BinList& B, long long r) {
  int a = 0, b = B.n;  // last index with cum[i] <= r
  while (b - a > 1) {
    const int m = (a + b) >> 1;
    if (static_cast<long long>(B.cum[m]) <= r) a = m;
    else b = m;
  }
  return a;
}

// Statistics are final: thresholds of the time pass (Section 2.1).
template <int NT>
__device__ void finalize_stats(const KParams& kp, const DevUnit& u, UnitState* slot, double median,
                               double sigma) {
  int kmax = 0;
  while (kmax < kp.max_log_window && (2 << kmax) <= u.T) ++kmax;
  fill_ktable<NT>(kp, median, sigma, kmax, slot->K);
  if (threadIdx.x == 0) {
    slot->median_t = median;
    slot->sigma_t = sigma;
    slot->time_on = (kp.enable_time && sigma > 0.0) ? 1 : 0;
    slot->state = kStateDone;
    if (u.stats) {
      u.stats->median_t = median;
      u.stats->sigma_t = sigma;
    }
  }
  __syncthreads();
}

// Exact twice-median M2 and four-times-MAD mad4 of a unit's pool of N
// values: remembered as the next block's hint, then the time-pass thresholds
// (sigma = 1.4826 MAD, Section 2.1), or the moments for the std estimator /
// a zero MAD.  Whole CTA.
template <int NT>
__device__ void finish_selected(const KParams& kp, const DevUnit& u, UnitState* slot, long long M2,
                                long long mad4, long long N) {
  const int tid = threadIdx.x;
  if (tid == 0 && kp.hist.hint && u.hist_slot >= 0) {
    kp.hist.hint[2 * u.hist_slot] = static_cast<unsigned long long>(M2);
    kp.hist.hint[2 * u.hist_slot + 1] = static_cast<unsigned long long>(mad4);
  }
  const double med = __dmul_rn(static_cast<double>(M2), 0.5);
  const double mad = __dmul_rn(static_cast<double>(mad4), 0.25);
  if (!kp.sigma_std && mad > 0.0) {
    finalize_stats<NT>(kp, u, slot, med, __dmul_rn(1.482602218505602, mad));
  } else if (kp.sigma_std) {
    // moments were accumulated with the coarse histogram
    const unsigned __int128 s1 =
        (static_cast<unsigned __int128>(__ldcg(slot->mom + 1)) << 64) | __ldcg(slot->mom + 0);
    const unsigned __int128 s2 =
        (static_cast<unsigned __int128>(__ldcg(slot->mom + 3)) << 64) | __ldcg(slot->mom + 2);
    finalize_stats<NT>(kp, u, slot, med, moments_std(N, s1, s2));
  } else {
    if (tid == 0) {
      slot->median_t = med;
      slot->mom[0] = slot->mom[1] = slot->mom[2] = slot->mom[3] = 0;
      slot->state = kStateMoments;
    }
    __syncthreads();
  }
}

// Plan the next refinement round, or finish.  Whole CTA of the last arriver;
// the bin list is in shared memory.
template <int NT>
__device__ void select_plan(const KParams& kp, const DevUnit& u, UnitState* slot, const BinList& B,
                            Fixed<NT>& f) {
  const int tid = threadIdx.x, lane = tid & 31;
  const long long N = B.cum[B.n];
  if (tid == 0) {
    if (N != slot->n_pool) set_error(kp, kErrInternal, 10);
    const long long r1 = (N & 1) ? (N - 1) / 2 : N / 2 - 1;
    const long long r2 = (N & 1) ? r1 : N / 2;
    const int b1 = bin_of_rank(B, r1), b2 = bin_of_rank(B, r2);
    f.mb[0] = b1;
    f.mb[1] = b2;
    if (N & 1) {
      f.m2lo = 2ll * B.lo[b1];
      f.m2hi = 2ll * B.hi[b1];
    } else {
      f.m2lo = static_cast<long long>(B.lo[b1]) + B.lo[b2];
      f.m2hi = static_cast<long long>(B.hi[b1]) + B.hi[b2];
    }
  }
  __syncthreads();
  const long long m2lo = f.m2lo, m2hi = f.m2hi;
  {
    // warps 0..3: lower / upper bracket of the MAD rank(s), one search each
    const int warp = tid >> 5;
    const int nr = (N & 1) ? 1 : 2;
    if (warp < 2 * nr) {
      const int q = warp >> 1;
      const long long r = (N & 1) ? (N - 1) / 2 : N / 2 - 1 + q;
      const long long d = (warp & 1) ? warp_search<false>(B, m2lo, m2hi, r + 1, lane)
                                     : warp_search<true>(B, m2lo, m2hi, r + 1, lane);
      if (lane == 0) {
        if (warp & 1) f.db[q] = d;
        else f.da[q] = d;
      }
    }
    __syncthreads();
    if (tid == 0 && nr == 1) {
      f.da[1] = f.da[0];
      f.db[1] = f.db[0];
    }
  }
  __syncthreads();
  if (tid == 0) {
    int nt = 0;
    auto add = [&](int b) {
      if (b < 0 || b >= B.n || B.hi[b] == B.lo[b]) return;
      for (int i = 0; i < nt; ++i)
        if (f.tb[i] == b) return;
      if (nt < kMaxTargets) f.tb[nt++] = b;
    };
    auto add_range = [&](long long ylo, long long yhi) {
      if (ylo < 0) ylo = 0;
      if (yhi > 0xFFFFFFFFll) yhi = 0xFFFFFFFFll;
      if (ylo > yhi) return;
      int a = 0, b = B.n;  // first bin with hi >= ylo
      while (a < b) {
        const int m = (a + b) >> 1;
        if (static_cast<long long>(B.hi[m]) < ylo) a = m + 1;
        else b = m;
      }
      for (int i = a; i < B.n && static_cast<long long>(B.lo[i]) <= yhi; ++i) add(i);
    };
    add(f.mb[0]);
    add(f.mb[1]);
    const bool med_exact = (m2lo == m2hi);
    bool mad_exact = med_exact;
    for (int q = 0; q < 2; ++q) {
      const long long da = f.da[q], db = f.db[q];
      if (da != db || !med_exact) {
        mad_exact = false;
        add_range(endA(m2lo, db) - 1, endA(m2hi, da));
        add_range(endB(m2lo, da) - 1, endB(m2hi, db) + 1);
      }
    }
    f.resolved = (med_exact && mad_exact) ? 1 : 0;
    for (int i = 1; i < nt; ++i)
      for (int j = i; j > 0 && f.tb[j - 1] > f.tb[j]; --j) {
        const int t = f.tb[j];
        f.tb[j] = f.tb[j - 1];
        f.tb[j - 1] = t;
      }
    if (!f.resolved && nt == 0) {
      set_error(kp, kErrSelect, 1);
      f.resolved = 2;
    }
    if (f.resolved == 0) {
      int per = kp.fine_bins / nt;
      int p2 = 1;
      while (p2 * 2 <= per) p2 *= 2;
      int base = 0;
      for (int i = 0; i < nt; ++i) {
        const uint32_t lo = B.lo[f.tb[i]], hi = B.hi[f.tb[i]];
        const unsigned long long W = static_cast<unsigned long long>(hi - lo) + 1ull;
        uint32_t sh = 0;
        while (((W - 1ull) >> sh) + 1ull > static_cast<unsigned long long>(p2)) ++sh;
        const int nsub = static_cast<int>(((W - 1ull) >> sh) + 1ull);
        slot->tgt[i] = Target{lo, hi, sh, static_cast<uint32_t>(base)};
        slot->tgt_bin[i] = f.tb[i];
        base += nsub;
      }
      slot->n_targets = nt;
      slot->n_fine = base;
      slot->round += 1;
      if (slot->round > kMaxRounds) {
        set_error(kp, kErrSelect, 2);
        f.resolved = 2;
      } else {
        slot->state = kStateFine;
      }
    }
  }
  __syncthreads();
  if (f.resolved == 0) {
    for (int i = tid; i < kMaxFine; i += NT) slot->fine[i] = 0;
    __syncthreads();
    return;
  }
  if (f.resolved == 2) {  // give up: no time pass for this unit
    finalize_stats<NT>(kp, u, slot, 0.0, 0.0);
    return;
  }
  finish_selected<NT>(kp, u, slot, m2lo, f.da[0] + f.da[1], N);  // odd N: 2 d*, even N: d*(a) + d*(b)
}

// Builds the initial bin list from a coarse histogram in shared memory (warp
// 0): non-empty keys in order, straight into the shared-memory list (lo, hi,
// cumulative counts) and into the slot for later refinement rounds.
template <int NT>
__device__ BinList build_coarse_list(const KParams& kp, UnitState* slot, const uint32_t* hist,
                                     uint8_t* ws) {
  uint32_t* lo = reinterpret_cast<uint32_t*>(ws);
  uint32_t* hi = lo + kSelCap;
  uint32_t* cum = hi + kSelCap;
  const int tid = threadIdx.x;
  __shared__ int s_n;
  if (tid < kWarp) {
    int n = 0;
    uint32_t carry = 0;
    if (tid == 0) cum[0] = 0;
    for (int base = 0; base < kCoarseBins; base += kWarp) {
      const int k = base + tid;
      const uint32_t c = k < kCoarseBins ? hist[k] : 0u;
      uint32_t a = 0, b = 0;
      const bool ok = c != 0u && key_range(static_cast<uint32_t>(k), &a, &b);
      if (c != 0u && !ok) set_error(kp, kErrInternal, 40);
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, ok);
      uint32_t tot;
      const uint32_t ex = warp_excl_scan(ok ? c : 0u, tid, &tot);
      if (ok) {
        const int pos = n + __popc(bal & ((1u << tid) - 1u));
        lo[pos] = a;
        hi[pos] = b;
        cum[pos + 1] = carry + ex + c;
        slot->blo[pos] = a;
        slot->bhi[pos] = b;
        slot->bcnt[pos] = c;
      }
      n += __popc(bal);
      carry += tot;
    }
    if (tid == 0) {
      slot->n_bins = n;
      s_n = n;
    }
  }
  __syncthreads();
  return BinList{lo, hi, cum, s_n};
}

// Replaces every refined bin by its non-empty sub-bins.
template <int NT>
__device__ void merge_fine(const KParams& kp, UnitState* slot, uint8_t* ws, Fixed<NT>& f) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = __ldcg(&slot->n_bins);
  const int nt = __ldcg(&slot->n_targets);
  uint32_t* lo = reinterpret_cast<uint32_t*>(ws);
  uint32_t* hi = lo + kSelCap;
  uint32_t* cnt = hi + kSelCap;
  for (int i = tid; i < n; i += NT) {
    lo[i] = __ldcg(slot->blo + i);
    hi[i] = __ldcg(slot->bhi + i);
    cnt[i] = __ldcg(slot->bcnt + i);
  }
  if (tid < kMaxTargets) {
    if (tid < nt) {
      f.tgt[tid] = ld_target(slot->tgt + tid);
      f.tb[tid] = __ldcg(slot->tgt_bin + tid);
    }
  }
  __syncthreads();
  for (int t = warp; t < nt; t += NT / kWarp) {
    const Target g = f.tgt[t];
    const int nsub = static_cast<int>((static_cast<unsigned long long>(g.hi - g.lo) >> g.shift) + 1ull);
    int nz = 0;
    unsigned long long sum = 0;
    for (int j = lane; j < nsub; j += kWarp) {
      const uint32_t c = __ldcg(slot->fine + g.base + j);
      nz += c != 0u;
      sum += c;
    }
    nz = __reduce_add_sync(0xFFFFFFFFu, nz);
    sum = warp_sum64(sum);
    if (lane == 0) {
      f.nnz[t] = nz;
      if (sum != cnt[f.tb[t]]) set_error(kp, kErrInternal, 20);
    }
  }
  __syncthreads();
  int grow = 0;
  for (int t = 0; t < nt; ++t) grow += f.nnz[t] - 1;
  const int nn = n + grow;
  if (nn > kSelCap) {
    if (tid == 0) set_error(kp, kErrSelect, 3);
    __syncthreads();
    return;
  }
  for (int i = tid; i < n; i += NT) {
    int shift = 0;
    bool is_t = false;
    for (int t = 0; t < nt; ++t) {
      if (f.tb[t] < i) shift += f.nnz[t] - 1;
      if (f.tb[t] == i) is_t = true;
    }
    if (!is_t) {
      slot->blo[i + shift] = lo[i];
      slot->bhi[i + shift] = hi[i];
      slot->bcnt[i + shift] = cnt[i];
    }
  }
  for (int t = warp; t < nt; t += NT / kWarp) {
    const Target g = f.tgt[t];
    int pos = f.tb[t];
    for (int q = 0; q < t; ++q) pos += f.nnz[q] - 1;
    const int nsub = static_cast<int>((static_cast<unsigned long long>(g.hi - g.lo) >> g.shift) + 1ull);
    for (int base = 0; base < nsub; base += kWarp) {
      const int j = base + lane;
      const uint32_t c = j < nsub ? __ldcg(slot->fine + g.base + j) : 0u;
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, c != 0u);
      if (c) {
        const int p = pos + __popc(bal & ((1u << lane) - 1u));
        const unsigned long long a = static_cast<unsigned long long>(g.lo) +
                                     (static_cast<unsigned long long>(j) << g.shift);
        unsigned long long b = a + (1ull << g.shift) - 1ull;
        if (b > g.hi) b = g.hi;
        slot->blo[p] = static_cast<uint32_t>(a);
        slot->bhi[p] = static_cast<uint32_t>(b);
        slot->bcnt[p] = c;
      }
      pos += __popc(bal);
    }
  }
  __threadfence_block();
  __syncthreads();
  if (tid == 0) slot->n_bins = nn;
  __syncthreads();
}

// ------------------------------------------------------------------ time pass helpers
//
// Packed values (integer units whose I = 1 threshold is below 2^20): after
// the I = 1 pass every unflagged power is at most floor(threshold_1), so a
// window of up to 64 unflagged values sums to less than Z = 2^26.  Flagged
// samples are stored as u = Z: the difference of two prefix entries is then
// S = n_flagged * Z + sum_unflagged with both parts recoverable, and the
// window fires exactly when S > Kp[n] = n * Z + floor((I - n) * threshold_I).
// These rows run one warp per row with the row in registers (wr_passes), in
// the equivalent low-bit form (kLowShift).
//
// Any other unit takes the general path: rows in a shared-memory prefix
// buffer, exact 64-bit sums of the unflagged values.  Layout of one batch of
// rows in that buffer (32-bit words per row):
//   Pl: (nch + 3) chunks x 36 words -- exclusive prefix, inside each 32-sample
//       chunk, of the values u (padded layout, see pidx); three zero chunks
//       follow the row so windows may look ahead by up to 64 samples
//   Pb: nch + 4 words -- exclusive prefix of the chunk totals (chunk bases)
//   Tc: nch + 4 words -- chunk totals
// so that the prefix of u at x is Pb[x >> 5] + Pl[pidx(x)] (mod 2^32).

constexpr uint32_t kZ = 1u << 26;
// The warp-row pass keeps its values in the low-bit form: unflagged
// u = power << 6, flagged u = 1, so that the sum of a window of I <= 32
// values is S = 64 * sum_unflagged + n_flagged (n < 64, S < 2^31 while
// threshold_1 < 2^20) and its low five bits index the register table by
// shuffle.  The window fires exactly when S > 64 * floor((I - n) *
// threshold_I) + 63.  The 64-sample window works on block sums converted
// back to n * Z + sum_unflagged.
constexpr uint32_t kLowShift = 6;
// s_Kp holds the kKTable thresholds (entry 0: floor(threshold_1); windows
// 2..32 in the low-bit form above; window 64 as n * Z + Kt[n]), then (c,
// Cb - 1) of each window size 2^k at kKbOff + 2k (k >= 3).
constexpr int kKbOff = kKTable;

struct StLayout {
  int PLW, PBW, per_row;
};
__device__ __forceinline__ StLayout st_layout(int nch) {
  StLayout L;
  L.PLW = (nch + 3) * 36;
  L.PBW = nch + 4;
  L.per_row = (L.PLW + 2 * L.PBW + 3) & ~3;  // rows start on 16-byte boundaries
  return L;
}

__device__ __forceinline__ uint32_t bit_at(const uint32_t* M, int j) {
  return (M[j >> 5] >> (j & 31)) & 1u;
}
__device__ __forceinline__ uint32_t pre_at(const uint32_t* pl, const uint32_t* pb, int x) {
  return pb[x >> 5] + pl[pidx(x)];
}

// General path (any integer magnitudes): exact 64-bit sums of the unflagged
// values of each window, sliding across the chunk; fires when
// sum_unflagged > K[n_flagged].  Values are single prefix differences,
// exact modulo 2^32.
__device__ uint32_t general_fire(const uint32_t* pl, const uint32_t* pb, const uint32_t* M,
                                 int t0, int I, int T, const long long* Kt) {
  const int tl = min(t0 + 31, T - I);
  unsigned long long su = 0;
  int nf = 0;
  uint32_t prev = pre_at(pl, pb, t0);
  for (int j = t0; j < t0 + I; ++j) {
    const uint32_t nx = pre_at(pl, pb, j + 1);
    if (bit_at(M, j)) ++nf;
    else su += nx - prev;
    prev = nx;
  }
  uint32_t fire = 0;
  for (int t = t0;; ++t) {
    if (static_cast<long long>(su) > Kt[nf]) fire |= 1u << (t - t0);
    if (t >= tl) break;
    if (bit_at(M, t)) --nf;
    else su -= pre_at(pl, pb, t + 1) - pre_at(pl, pb, t);
    if (bit_at(M, t + I)) ++nf;
    else su += pre_at(pl, pb, t + I + 1) - pre_at(pl, pb, t + I);
  }
  return fire;
}

// Flag bits covered by windows of I samples that start at a fired bit: bits
// of word w from fire words w (hi) and w-1 (lo), for I <= 32.
__device__ __forceinline__ uint32_t dilate32(uint32_t hi, uint32_t lo, int I) {
  unsigned long long x = (static_cast<unsigned long long>(hi) << 32) | lo;
  for (int s = 1; s < I; s <<= 1) x |= x << s;
  return static_cast<uint32_t>(x >> 32);
}

// Chunk bases Pb = exclusive prefix of the chunk totals (warp per row);
// only rows with dirty[rb] set (all rows when dirty == nullptr).
template <int NT>
__device__ void st_bases(uint32_t* region, const StLayout& L, int nch, int nbb, int* dirty) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int rb = warp; rb < nbb; rb += NT / kWarp) {
    if (dirty && !dirty[rb]) continue;
    uint32_t* pb = region + rb * L.per_row + L.PLW;
    const uint32_t* tc = pb + L.PBW;
    uint32_t carry = 0;
    for (int base = 0; base < L.PBW; base += kWarp) {
      const int c = base + lane;
      const uint32_t v = c < nch ? tc[c] : 0u;
      uint32_t tot;
      const uint32_t ex = warp_excl_scan(v, lane, &tot);
      if (c < L.PBW) pb[c] = carry + ex;
      carry += tot;
    }
    if (dirty && lane == 0) dirty[rb] = 0;
  }
}

// ------------------------------------------------------------------ global row access

template <int DT>
__device__ __forceinline__ void gload_vec(const uint8_t* grow, int x, int T, bool vec,
                                          uint32_t (&v)[Traits<DT>::kVec]) {
  using TR = Traits<DT>;
  if (vec && x + TR::kVec <= T) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(grow + static_cast<size_t>(x) * TR::kBytes));
    if constexpr (DT == LOF_CI16) {
      v[0] = TR::pw(w.x);
      v[1] = TR::pw(w.y);
      v[2] = TR::pw(w.z);
      v[3] = TR::pw(w.w);
    } else {
      v[0] = TR::pw(w.x);
      v[1] = TR::pw(w.x >> 16);
      v[2] = TR::pw(w.y);
      v[3] = TR::pw(w.y >> 16);
      v[4] = TR::pw(w.z);
      v[5] = TR::pw(w.z >> 16);
      v[6] = TR::pw(w.w);
      v[7] = TR::pw(w.w >> 16);
    }
  } else {
#pragma unroll
    for (int j = 0; j < TR::kVec; ++j) v[j] = (x + j < T) ? TR::at(grow, x + j) : 0u;
  }
}

__device__ __forceinline__ void warp_sum_u128(unsigned long long& lo, unsigned long long& hi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long l2 = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
    const unsigned long long h2 = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
    const unsigned long long nl = lo + l2;
    hi = hi + h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
}

// Chunk-local prefixes of u for the task's kept rows, read straight from the
// input in global memory (each warp reads 512 contiguous bytes per load).  In
// the packed path this is also the I = 1 pass: samples above K1 are flagged
// and stored as Z.
template <int DT, int NT>
__device__ void st_build(const DevUnit& u, int row0, int T, int nch, const int* rows, int nbb,
                         uint32_t* region, const StLayout& L, uint32_t* smbits, int MW,
                         bool packed, uint32_t K1) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, LPC = 32 / VS, NQ = 16 / VS, SEG = 32 * NQ * VS, NW = NT / kWarp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lp = lane & (LPC - 1);
  const int nseg = (T + SEG - 1) / SEG;
  const bool vin = (u.flags & kUnitInVec) != 0;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  for (int task = warp; task < nbb * nseg; task += NW) {
    const int rb = task / nseg, s = task - rb * nseg;
    const int r = rows[rb];
    const uint8_t* grow = gin + static_cast<int64_t>(row0 + r) * u.in_stride * TR::kBytes;
    uint32_t* pl = region + rb * L.per_row;
    uint32_t* tc = pl + L.PLW + L.PBW;
    uint32_t* mrow = smbits + r * MW + 2;
    uint32_t v[NQ][VS];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int x = s * SEG + q * 32 * VS + lane * VS;
      if (x < T) {
        gload_vec<DT>(grow, x, T, vin, v[q]);
      } else {
#pragma unroll
        for (int j = 0; j < VS; ++j) v[q][j] = 0u;
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int x = s * SEG + q * 32 * VS + lane * VS;
      uint32_t e[VS], acc = 0, fb = 0;
#pragma unroll
      for (int j = 0; j < VS; ++j) {
        uint32_t uu = v[q][j];
        if (packed && uu > K1) {
          fb |= 1u << j;
          uu = kZ;
        }
        e[j] = acc;
        acc += uu;
      }
      uint32_t incl = acc;
#pragma unroll
      for (int o = 1; o < LPC; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lp >= o) incl += y;
      }
      const uint32_t off = incl - acc;
      uint32_t fw = fb << (VS * lp);
#pragma unroll
      for (int o = 1; o < LPC; o <<= 1) fw |= __shfl_xor_sync(0xFFFFFFFFu, fw, o);
      const int c = x >> 5;
      if (c < nch + 3) {
#pragma unroll
        for (int j = 0; j < VS; j += 4) {
          uint4 w4;
          w4.x = off + e[j + 0];
          w4.y = off + e[j + 1];
          w4.z = off + e[j + 2];
          w4.w = off + e[j + 3];
          *reinterpret_cast<uint4*>(pl + pidx(x + j)) = w4;
        }
        if (lp == LPC - 1) tc[c] = incl;
        if (lp == 0 && packed && c < nch) mrow[c] = fw;
      }
    }
  }
  // zero chunks after the row (look-ahead of the last windows)
  for (int i = threadIdx.x; i < nbb * 3 * 32; i += NT) {
    const int rb = i / 96, j = i - rb * 96;
    const int x = nch * 32 + j;
    uint32_t* pl = region + rb * L.per_row;
    pl[pidx(x)] = 0u;
    if ((j & 31) == 0) pl[L.PLW + L.PBW + (x >> 5)] = 0u;
  }
}

// L2 eviction policies: the input of a unit is read by its statistics
// tasks and again by its flag tasks shortly after, so those reads mark it
// evict_last; the last read (the output copy) marks it evict_first.
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_drop() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint4 ldg_policy(const void* ptr, uint64_t pol) {
  uint4 v;
  asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(ptr), "l"(pol));
  return v;
}
// Streaming (evict-first) stores of the mask bytes.
__device__ __forceinline__ void st_stream_u32(void* p, uint32_t v) {
  asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_stream_u64(void* p, uint32_t lo, uint32_t hi) {
  asm volatile("st.global.cs.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(lo), "r"(hi) : "memory");
}

// Raw 16-byte vector of samples [x, x + kVec) of a row, zero at or past T.
template <int DT>
__device__ __forceinline__ uint4 gload_raw(const uint8_t* grow, int x, int T, bool vec,
                                           uint64_t pol) {
  using TR = Traits<DT>;
  if (vec && x + TR::kVec <= T)
    return ldg_policy(grow + static_cast<size_t>(x) * TR::kBytes, pol);
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  for (int j = 0; j < TR::kVec && x + j < T; ++j) {
    if constexpr (DT == LOF_CI16) {
      w[j] = reinterpret_cast<const uint32_t*>(grow)[x + j];
    } else {
      const uint32_t h = reinterpret_cast<const uint16_t*>(grow)[x + j];
      w[j >> 1] |= h << (16 * (j & 1));
    }
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Power of sample j (static) of a raw vector.
template <int DT>
__device__ __forceinline__ uint32_t raw_pw(const uint4& w, int j) {
  if constexpr (DT == LOF_CI16) {
    const uint32_t c = j == 0 ? w.x : j == 1 ? w.y : j == 2 ? w.z : w.w;
    return Traits<DT>::pw(c);
  } else {
    const int k = j >> 1;
    const uint32_t c = k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
    return Traits<DT>::pw((j & 1) ? (c >> 16) : c);
  }
}

// ------------------------------------------------------------------ warp-row time pass
// SumThreshold along time (Section 2.1) over one row segment by one warp,
// every value in registers.  Lane L holds the NPL consecutive samples
// s0 + L*NPL + [0, NPL) as packed values u[] (unflagged: the power, at most
// K1 < 2^20 after the I = 1 pass; flagged: Z = 2^26) and their flag bits
// M[].  The packed sum of a window is S = n * Z + sum_unflagged, and the
// window fires exactly when S > Kp[n] = n * Z + floor((I - n) * threshold_I)
// (n = S >> 26).  The sums slide along the lane, one three-input add per
// window, taking the values past the lane's end from the next lanes by
// shuffle; each decision is the sign bit of Kp[n] - S (|.| < 2^26), shifted
// into the lane's fire words with a funnel shift.  New flags replace their
// values by Z.
//
// Rows longer than 32 * NPL are cut into segments that overlap by a halo of
// sum_I (I - 1) = 120 samples on each side: a flag decision at x depends
// only on samples within I - 1 of x at each window size, so the flags of a
// segment's interior equal those of the whole row.

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWrHalo = 120;  // 0 + 1 + 3 + 7 + 15 + 31 + 63

template <int NPL>
struct WrRow {
  static constexpr int NW = NPL / 32;
  uint32_t u[NPL];  // packed values
  uint32_t M[NW];   // flag bits of the lane's samples
};

// u at lane-relative position x >= 0 (x < 3 * NPL), from the next lanes by
// shuffle.  Past lane 31 (past the segment's span) the shuffle returns the
// lane's own value: another valid packed value, read only by windows that
// run past the span, whose fire bits wr_apply masks off.  The slide stays
// exact for the others (every value it adds it later subtracts).
template <int NPL>
__device__ __forceinline__ uint32_t wr_uat(const WrRow<NPL>& R, int lane, int x) {
  (void)lane;
  if (x < NPL) return R.u[x];
  const int q = x / NPL;
  return __shfl_down_sync(kFull, R.u[x - q * NPL], q);
}

// Fire words F[w] (bit b: the window of size I at j = 32w + b fires), by a
// descending slide of the packed window sums.
template <int NPL, int I>
__device__ __forceinline__ void wr_fire(const WrRow<NPL>& R, int lane, const uint32_t* Kp,
                                        uint32_t (&F)[NPL / 32]) {
  constexpr int NW = NPL / 32, m = I - 1;
  // packed sum of the m values after the lane's last one
  uint32_t hs;
  {
    constexpr int a = m < NPL ? m : NPL;
    uint32_t A = 0u;
#pragma unroll
    for (int k = 0; k < a; ++k) A += R.u[k];
    hs = __shfl_down_sync(kFull, A, 1);
    if constexpr (m > NPL) {
      uint32_t B = 0u;
#pragma unroll
      for (int k = 0; k < m - NPL; ++k) B += R.u[k];
      uint32_t hb = __shfl_down_sync(kFull, B, 2);
      hs += hb;
    }
  }
  static_assert(I <= 32, "low-bit window sums");
  uint32_t S = R.u[NPL - 1] + hs;
  // the table sits in registers, lane n holding Kp[n], and is read by
  // shuffle with the sum itself as the index (its low five bits are n; n = 32
  // wraps to Kp[0] > S: a window of 32 flagged samples, which would flag
  // nothing new anyway)
  const uint32_t Kreg = Kp[lane < I ? lane : I];
#pragma unroll
  for (int w = NW - 1; w >= 0; --w) {
    uint32_t f = 0u;
#pragma unroll
    for (int b = 31; b >= 0; --b) {
      const int j = 32 * w + b;
      f = __funnelshift_l(__shfl_sync(kFull, Kreg, S) - S, f, 1);
      if (j > 0) S = S + R.u[j - 1] - wr_uat<NPL>(R, lane, j - 1 + I);
    }
    F[w] = f;
  }
}

// Q of block b (lane-relative), blocks past the lane's last from the next
// lanes by shuffle (past lane 31: another valid packed sum; only windows that
// the caller masks off read those).
template <int NB>
__device__ __forceinline__ uint32_t wr_qat(const uint32_t (&Q)[NB], int b) {
  if (b < NB) return Q[b];
  const int q = b / NB;
  return __shfl_down_sync(kFull, Q[b - q * NB], q);
}

// Fire words for windows of I >= 8 samples, with an exact prefilter.  The
// lane's samples form blocks of four; the windows that start in block b lie
// in its union [4b, 4b + I + 4), whose n_U flagged samples and unflagged sum
// s_U bound every such window (n <= n_U, s <= s_U).  With
// c = Kt[I - 1] + 1 >= threshold_I and Cb = min_n (Kt[n] + 1 + n * c), a window
// can fire (s > Kt[n]) only if s_U + n_U * c >= Cb, so blocks whose union
// stays below Cb hold no firing window.  Only the block slots where some lane
// has a candidate run the exact test (warp-uniform, so shuffles stay valid);
// every other fire bit is zero, as the exact test would give.  Cb1 = Cb - 1.
template <int NPL, int I>
__device__ __forceinline__ void wr_fire_pf(const WrRow<NPL>& R, int lane, const uint32_t* Kp,
                                           uint32_t c, uint32_t Cb1, bool bound, uint32_t (&F)[NPL / 32]) {
  static_assert(NPL == 32 && I >= 8 && I <= 64, "one flag word per lane, blocks of four");
  constexpr int NB = NPL / 4, D = I / 4;
  uint32_t Q[NB], X[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    // low-bit block sum 64 * s + n (n <= 4), then s + n * c (< 2^24)
    Q[b] = R.u[4 * b] + R.u[4 * b + 1] + R.u[4 * b + 2] + R.u[4 * b + 3];
    X[b] = (Q[b] >> kLowShift) + (Q[b] & 63u) * c;
  }
  // V = sum of X over blocks b .. b + D, descending from b = NB - 1
  uint32_t hs;
  {
    constexpr int a = D < NB ? D : NB;
    uint32_t A = 0u;
#pragma unroll
    for (int k = 0; k < a; ++k) A += X[k];
    hs = __shfl_down_sync(kFull, A, 1);
    if constexpr (D > NB) hs += __shfl_down_sync(kFull, A, 2);
  }
  uint32_t V = X[NB - 1] + hs, cand = 0u;
#pragma unroll
  for (int b = NB - 1; b >= 0; --b) {
    cand = __funnelshift_l(Cb1 - V, cand, 1);
    if (b > 0) V = V + X[b - 1] - wr_qat<NB>(X, b + D);
  }
  // without the bound (schedule) every block slot takes the exact test
  const uint32_t any = bound ? __reduce_or_sync(kFull, cand) : ((1u << NB) - 1u);
  uint32_t f = 0u;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (!((any >> b) & 1u)) continue;
    // window sum at 4b as n * Z + s: blocks b .. b + D - 1
    uint32_t S = 0u;
    {
      auto zq = [](uint32_t q) { return (q >> kLowShift) + (q & 63u) * kZ; };
      uint32_t own = 0u, p1 = 0u, p2 = 0u;
#pragma unroll
      for (int i = b; i < b + D && i < NB; ++i) own += zq(Q[i]);
      if (b + D > NB) {
#pragma unroll
        for (int i = 0; i < b + D - NB && i < NB; ++i) p1 += zq(Q[i]);
        p1 = __shfl_down_sync(kFull, p1, 1);
      }
      if (b + D > 2 * NB) {
#pragma unroll
        for (int i = 0; i < b + D - 2 * NB; ++i) p2 += zq(Q[i]);
        p2 = __shfl_down_sync(kFull, p2, 2);
      }
      S = own + p1 + p2;
    }
    auto zu = [](uint32_t v) { return (v >> kLowShift) + (v & 1u) * kZ; };
    uint32_t bits = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      bits |= ((Kp[S >> 26] - S) >> 31) << i;
      if (i < 3) S = S - zu(R.u[4 * b + i]) + zu(wr_uat<NPL>(R, lane, 4 * b + i + I));
    }
    f |= bits << (4 * b);
  }
  F[0] = f;
}

// Dilate the fire bits (a fired window flags its I samples), add the new
// flags to M and store them as flagged (u = 1).  I is a run-time value here
// so that one copy of this code serves every window size.
template <int NPL>
__device__ __forceinline__ void wr_apply(WrRow<NPL>& R, int lane, int nvalid, int I,
                                         uint32_t (&F)[NPL / 32]) {
  constexpr int NW = NPL / 32;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const int nv = nvalid - 32 * w;
    const uint32_t vm = nv >= 32 ? kFull : (nv <= 0 ? 0u : ((1u << nv) - 1u));
    F[w] &= vm;
  }
  {
    uint32_t anyf = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) anyf |= F[w];
    if (!__any_sync(kFull, anyf != 0u)) return;  // no window of this size fired
  }
  // the two fire words just before the lane's first word
  uint32_t p1, p2;
  if constexpr (NW == 1) {
    p1 = __shfl_up_sync(kFull, F[0], 1);
    p2 = __shfl_up_sync(kFull, F[0], 2);
  } else {
    p1 = __shfl_up_sync(kFull, F[NW - 1], 1);
    p2 = __shfl_up_sync(kFull, F[NW - 2], 1);
  }
  if (lane < 1) p1 = 0u;
  if (lane < (NW == 1 ? 2 : 1)) p2 = 0u;
  uint32_t nw[NW];
  uint32_t anyw = 0u;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t f0 = F[w];
    const uint32_t f1 = w >= 1 ? F[w - 1] : p1;
    const uint32_t f2 = w >= 2 ? F[w - 2] : (w == 1 ? p1 : p2);
    const uint32_t Dw = (I <= 32) ? dilate32(f0, f1, I) : (dilate32(f0, f1, 32) | dilate32(f1, f2, 32));
    nw[w] = Dw & ~R.M[w];
    anyw |= nw[w];
  }
#pragma unroll
  for (int w = 0; w < NW; ++w) R.M[w] |= nw[w];
  if (!__any_sync(kFull, anyw != 0u)) return;
#pragma unroll
  for (int j = 0; j < NPL; ++j)
    if ((nw[j >> 5] >> (j & 31)) & 1u) R.u[j] = 1u;
}

// ---- staged segment I/O of the warp-row pass
// Each warp owns two staging buffers in shared memory.  Lane L's NPL samples
// of a segment fill row L of a buffer in sample order; rows are padded by 16
// bytes so that the 16-byte shared loads of a quarter warp hit distinct
// banks.  A segment is staged by cp.async (no registers) while the previous
// one is computed; the build reads it from shared memory, and the output
// zeroes its flagged samples there and stores the lane's interior samples
// with one bulk copy.
template <int DT, int NPL>
struct WrStage {
  static constexpr int kRowBytes = NPL * Traits<DT>::kBytes + 16;
  static constexpr int kBufBytes = 32 * kRowBytes;
};

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Stages the lane's samples [x, x + NPL) of a row (zeros at or past T) into
// its buffer row srow as one cp.async group: 16-byte asynchronous copies
// where the row is 16-byte aligned and the piece lies inside the row, plain
// loads and shared stores elsewhere.
template <int DT, int NPL>
__device__ __forceinline__ void wr_stage(uint8_t* srow, const uint8_t* grow, int x, int T, bool vin,
                                         uint64_t pol) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, NV = NPL / VS;
  const uint32_t sa = saddr(srow);
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int xs = x + q * VS;
    if (vin && xs + VS <= T) {
      asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(sa + 16 * q),
                   "l"(grow + static_cast<size_t>(xs) * TR::kBytes), "l"(pol)
                   : "memory");
    } else {
      const uint4 v = xs < T ? gload_raw<DT>(grow, xs, T, false, pol) : make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(srow + 16 * q) = v;
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Loads the lane's staged samples as powers, flags those above K1 (the I = 1
// pass) and stores them as flagged (u = 1), the others as power << 6.
template <int DT, int NPL>
__device__ __forceinline__ void wr_build(WrRow<NPL>& R, const uint8_t* srow, uint32_t K1) {
  constexpr int VS = Traits<DT>::kVec, NV = NPL / VS;
  uint4 v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = *reinterpret_cast<const uint4*>(srow + 16 * q);
#pragma unroll
  for (int w = 0; w < NPL / 32; ++w) R.M[w] = 0u;
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const uint32_t uu = raw_pw<DT>(v[j / VS], j % VS);
    const bool fl = uu > K1;
    R.u[j] = fl ? 1u : (uu << kLowShift);
    if (fl) R.M[j >> 5] |= 1u << (j & 31);
  }
}

// Segments of a row: the first starts at 0, each later one at least
// kWrHalo samples (rounded to whole 32-sample words) before the end of the
// previous interior; a segment's interior ends kWrHalo samples (rounded down
// to a word) before its span, except at the end of the row.
// With every start a multiple of 32, the steps are constant: a segment that
// does not reach T ends its interior D = (SPAN - halo) & ~31 after its start,
// and the next one starts STEP = (D - halo) & ~31 later, so segment sg spans
// [sg * STEP, sg * STEP + SPAN) with interior [(sg - 1) * STEP + D, sg * STEP + D)
// (from 0 for the first, to T for the last).
template <int NPL>
__device__ __forceinline__ void wr_seg_bounds(int T, int sg, int& s0, int& oa, int& ob) {
  constexpr int SPAN = 32 * NPL, D = (SPAN - kWrHalo) & ~31, STEP = (D - kWrHalo) & ~31;
  s0 = sg * STEP;
  oa = sg == 0 ? 0 : s0 - STEP + D;
  ob = s0 + SPAN >= T ? T : s0 + D;
}
template <int NPL>
__device__ __forceinline__ int wr_seg_count(int T) {
  constexpr int SPAN = 32 * NPL, D = (SPAN - kWrHalo) & ~31, STEP = (D - kWrHalo) & ~31;
  return T <= SPAN ? 1 : (T - SPAN + STEP - 1) / STEP + 1;
}

// Output of one row for the fused writer of the warp-row pass.
struct WrOut {
  uint8_t* out;   // masked data row (NULL: none)
  uint8_t* mask;  // mask row (NULL: none)
  bool enabled, inplace, vout, mask_vec, vin;
};

// Mask bytes and masked data of the 32 samples [x, x + 32) of one row, from
// their flag word m (one lane; bits past T are zero) and the lane's staged
// samples srow.  In-place rows get no data here: their flagged samples are
// zeroed once the whole row is final, as a later segment's halo re-reads
// this segment's samples.
template <int DT>
__device__ __forceinline__ void wr_write_word(const WrOut& o, uint8_t* srow, int x, int T, uint32_t m) {
  using TR = Traits<DT>;
  const int nv = min(32, T - x);
  if (o.mask) {
    if (o.mask_vec && nv == 32) {
      uint32_t w[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) w[q] = (((m >> (4 * q)) & 0xFu) * 0x00204081u) & 0x01010101u;
      st_stream_u64(o.mask + x, w[0], w[1]);
      st_stream_u64(o.mask + x + 8, w[2], w[3]);
      st_stream_u64(o.mask + x + 16, w[4], w[5]);
      st_stream_u64(o.mask + x + 24, w[6], w[7]);
    } else {
      for (int j = 0; j < nv; ++j) o.mask[x + j] = static_cast<uint8_t>((m >> j) & 1u);
    }
  }
  if (!o.out || o.inplace) return;
  uint32_t mm = m;
  while (mm) {
    const int j = __ffs(mm) - 1;
    mm &= mm - 1u;
    TR::zero(srow, j);
  }
  const int bytes = nv * TR::kBytes;
  if (o.vout && (bytes & 15) == 0) {
    fence_async_smem();  // the staged samples and the zeroes above: generic-proxy writes
    bulk_store(o.out + static_cast<size_t>(x) * TR::kBytes, srow, static_cast<uint32_t>(bytes));
    bulk_commit();
  } else {
    for (int j = 0; j < nv; ++j)
      TR::copy(o.out + static_cast<size_t>(x + j) * TR::kBytes, srow + j * TR::kBytes);
  }
}

// One segment of a row as seen by the lane: its span's start s0, interior
// [oa, ob), end of valid samples vend and the lane's first sample xl.
struct WrSeg {
  int s0, oa, ob, vend, xl;
};
template <int NPL>
__device__ __forceinline__ WrSeg wr_seg(int T, int sg) {
  WrSeg g;
  wr_seg_bounds<NPL>(T, sg, g.s0, g.oa, g.ob);
  g.vend = min(T, g.s0 + 32 * NPL);
  g.xl = g.s0 + (threadIdx.x & 31) * NPL;
  return g;
}

// Masked data of a segment's interior [oa, ob) with coalesced 16-byte
// stores (whole warp): in round r lane L writes the (32 r + L)-th 16-byte
// chunk of the span, read from the staged row of lane (32 r + L) / CPL
// (CPL = chunks per lane) with the flagged samples zeroed from that lane's
// flag word, and, when mask_row is given, the chunk's mask bytes (four or
// eight, one store).  Only whole chunks inside [oa, min(ob, T)) are stored
// in the rounds; a row's last chunk, when the row ends inside it, goes
// sample by sample from lane 0.  (Measured against one bulk copy per lane
// from the staged rows: 0.26 against 0.42 ms for the data of a full-station
// block.)  Staged rows are padded by 16 bytes, so the 16-byte shared loads of
// a quarter warp still fall on distinct banks.
template <int DT, int NPL>
__device__ __forceinline__ void wr_store_coalesced(const uint8_t* stage, uint32_t M, const WrSeg& g, int T,
                                                   uint8_t* out_row, uint8_t* mask_row) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, CPL = NPL / VS, LPR = 32 / CPL, RB = WrStage<DT, NPL>::kRowBytes;
  static_assert(32 % CPL == 0, "whole staged rows per round");
  const int lane = threadIdx.x & 31;
  const int xe = min(g.ob, T);
  const int k_lo = (g.oa - g.s0) / VS, k_hi = (xe - g.s0) / VS;  // whole chunks [k_lo, k_hi)
  const int q = lane % CPL, sh = VS * q;
  const uint8_t* const sp = stage + (lane / CPL) * RB + 16 * q;
  uint8_t* const op = out_row + static_cast<size_t>(g.s0 + lane * VS) * TR::kBytes;
  uint8_t* const mp = mask_row ? mask_row + g.s0 + lane * VS : nullptr;
  __syncwarp();  // every lane's staged samples (its own cp.async group) visible to the warp
#pragma unroll
  for (int r = 0; r < CPL; ++r) {
    const uint32_t m = __shfl_sync(kFull, M, r * LPR + lane / CPL);
    if (static_cast<unsigned>(32 * r + lane - k_lo) < static_cast<unsigned>(k_hi - k_lo)) {
      uint4 w = *reinterpret_cast<const uint4*>(sp + r * LPR * RB);
      const uint32_t bits = (m >> sh) & ((1u << VS) - 1u);
      if (bits) {
        uint32_t wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < VS; ++j) {
          if ((bits >> j) & 1u) {
            if constexpr (VS == 4) wd[j] = 0u;
            else wd[j >> 1] &= (j & 1) ? 0x0000FFFFu : 0xFFFF0000u;
          }
        }
        w = make_uint4(wd[0], wd[1], wd[2], wd[3]);
      }
      __stcs(reinterpret_cast<uint4*>(op + r * 32 * 16), w);
      if (mp) {
        if constexpr (VS == 4) {
          __stcs(reinterpret_cast<unsigned int*>(mp + r * 32 * VS), (bits * 0x00204081u) & 0x01010101u);
        } else {
          __stcs(reinterpret_cast<uint2*>(mp + r * 32 * VS),
                 make_uint2(((bits & 0xFu) * 0x00204081u) & 0x01010101u, ((bits >> 4) * 0x00204081u) & 0x01010101u));
        }
      }
    }
  }
  // the row's last, partial chunk (warp-uniform condition)
  const int xp = g.s0 + k_hi * VS;
  if (xe == T && xp < T && xp >= g.oa) {
    const uint32_t m = __shfl_sync(kFull, M, k_hi / CPL);
    if (lane == 0) {
      const uint8_t* spp = stage + (k_hi / CPL) * RB + 16 * (k_hi % CPL);
      const int sb = VS * (k_hi % CPL);
      for (int j = 0; j < T - xp; ++j) {
        const uint32_t fl = (m >> (sb + j)) & 1u;
        if (fl) TR::zero(out_row, xp + j);
        else TR::copy(out_row + static_cast<size_t>(xp + j) * TR::kBytes, spp + j * TR::kBytes);
        if (mask_row) mask_row[xp + j] = static_cast<uint8_t>(fl);
      }
    }
  }
}

// Window sizes 2^k, k0 <= k <= k1, of the time pass over a segment held in R.
template <int NPL>
__device__ __forceinline__ void wr_passes(WrRow<NPL>& R, const WrSeg& g, int k0, int k1,
                                          const uint32_t* s_Kp, bool bound64) {
  static_assert(NPL == 32, "one flag word per lane");
  constexpr int NW = NPL / 32;
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int k = k0; k <= k1; ++k) {
    const int I = 1 << k;
    const uint32_t* Kp = s_Kp + koffset(k);
    uint32_t F[NW];
    // the prefilter pays off for the largest window only (fewest candidate
    // blocks, most shuffles in the exact loop)
    const uint32_t c = s_Kp[kKbOff + 2 * k], Cb1 = s_Kp[kKbOff + 2 * k + 1];
    switch (k) {
      case 1: wr_fire<NPL, 2>(R, lane, Kp, F); break;
      case 2: wr_fire<NPL, 4>(R, lane, Kp, F); break;
      case 3: wr_fire<NPL, 8>(R, lane, Kp, F); break;
      case 4: wr_fire<NPL, 16>(R, lane, Kp, F); break;
      case 5: wr_fire<NPL, 32>(R, lane, Kp, F); break;
      default: wr_fire_pf<NPL, 64>(R, lane, Kp, c, Cb1, bound64, F); break;
    }
    wr_apply<NPL>(R, lane, g.vend - I + 1 - g.xl, I, F);
  }
}

// Interior words [oa, ob) of a segment: flag words to M_out (the row's
// words), mask and masked data, and the interior's number of flagged samples
// and sum of unflagged powers (returned in every lane).
template <int DT, int NPL>
__device__ __forceinline__ void wr_finish(const WrRow<NPL>& R, const WrSeg& g, int T, uint8_t* srow,
                                          uint32_t* M_out, const WrOut& o, int& n_flag,
                                          unsigned long long& sum_unflagged) {
  constexpr int NW = NPL / 32;
  int nfl = 0;
  unsigned long long su = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const int x = g.xl + 32 * w;
    if (x >= g.oa && x < g.ob) {
      M_out[x >> 5] = R.M[w];
      nfl += __popc(R.M[w]);
      uint32_t s = 0u;  // low-bit form: 64 * sum_unflagged + n, n <= 32
#pragma unroll
      for (int b = 0; b < 32; ++b) s += R.u[32 * w + b];
      su += s >> kLowShift;
      if (o.enabled) wr_write_word<DT>(o, srow + 32 * w * Traits<DT>::kBytes, x, T, R.M[w]);
    }
  }
  n_flag = __reduce_add_sync(kFull, nfl);
  sum_unflagged = warp_sum64(su);
}

// Samples per lane of the warp-row pass (rows longer than 32 * kWrNpl are
// cut into overlapping segments).
constexpr int kWrNpl = 32;

// ------------------------------------------------------------------ fine counts

// Exact counts of the pooled values inside the refinement targets, for rows
// [ra, rb) of the unit whose frequency flag is clear; added to us->fine.
template <int DT, int NT>
__device__ void count_fine_rows(const KParams& kp, const DevUnit& u, UnitState* us, int ra,
                                int rb_end, uint8_t* ws, Fixed<NT>& f) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, SEG = 64 * VS, NW = NT / kWarp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = u.T, nseg = (T + SEG - 1) / SEG;
  const bool vin = (u.flags & kUnitInVec) != 0;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  uint32_t* fine = reinterpret_cast<uint32_t*>(ws);
  uint8_t* map = ws + 4 * kMaxFine;
  uint8_t* fc = map + kCoarseBins;
  const int nt = __ldcg(&us->n_targets);
  const int nf = __ldcg(&us->n_fine);
  if (tid < nt) f.tgt[tid] = ld_target(us->tgt + tid);
  for (int i = tid; i < nf; i += NT) fine[i] = 0u;
  for (int r = ra + tid; r < rb_end; r += NT) fc[r - ra] = __ldcg(kp.chan_Fc + u.chan_off + r);
  __syncthreads();
  for (int k = tid; k < kCoarseBins; k += NT) {
    uint32_t lo, hi;
    uint8_t mk = 0xFFu;
    if (key_range(static_cast<uint32_t>(k), &lo, &hi)) {
      int t = 0;
      while (t < nt && f.tgt[t].hi < lo) ++t;
      if (t < nt && f.tgt[t].lo <= hi) mk = static_cast<uint8_t>(t);
    }
    map[k] = mk;
  }
  __syncthreads();
  for (int task = warp; task < (rb_end - ra) * nseg; task += NW) {
    const int rr = task / nseg, s = task - rr * nseg;
    if (fc[rr]) continue;
    const uint8_t* grow = gin + static_cast<int64_t>(ra + rr) * u.in_stride * TR::kBytes;
    uint32_t v[2][VS];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int x = s * SEG + q * 32 * VS + lane * VS;
      if (x < T) gload_vec<DT>(grow, x, T, vin, v[q]);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int x = s * SEG + q * 32 * VS + lane * VS;
      if (x < T) {
#pragma unroll
        for (int j = 0; j < VS; ++j) {
          if (x + j < T) {
            const uint32_t val = v[q][j];
            int t = map[coarse_key(val)];
            if (t != 0xFF) {
              for (; t < nt && val >= f.tgt[t].lo; ++t) {
                if (val <= f.tgt[t].hi) {
                  atomicAdd(&fine[f.tgt[t].base + ((val - f.tgt[t].lo) >> f.tgt[t].shift)], 1u);
                  break;
                }
              }
            }
          }
        }
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < nf; i += NT) {
    const uint32_t h = fine[i];
    if (h) atomicAdd(us->fine + i, h);
  }
  __syncthreads();
}

// Exact moments of every kept sample of the unit (std estimator fallback when
// the MAD is zero), then the final statistics.
template <int DT, int NT>
__device__ void unit_moments(const KParams& kp, const DevUnit& u, UnitState* us, uint8_t* ws,
                             Fixed<NT>& f) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, SEG = 64 * VS, NW = NT / kWarp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = u.T, nseg = (T + SEG - 1) / SEG;
  const bool vin = (u.flags & kUnitInVec) != 0;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  unsigned long long s1 = 0;
  unsigned __int128 s2 = 0;
  for (int task = warp; task < u.C * nseg; task += NW) {
    const int r = task / nseg, s = task - r * nseg;
    if (__ldcg(kp.chan_Fc + u.chan_off + r)) continue;
    const uint8_t* grow = gin + static_cast<int64_t>(r) * u.in_stride * TR::kBytes;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int x = s * SEG + q * 32 * VS + lane * VS;
      if (x < T) {
        uint32_t v[VS];
        gload_vec<DT>(grow, x, T, vin, v);
#pragma unroll
        for (int j = 0; j < VS; ++j) {
          s1 += v[j];
          s2 += static_cast<unsigned long long>(v[j]) * v[j];
        }
      }
    }
  }
  s1 = warp_sum64(s1);
  unsigned long long lo = static_cast<unsigned long long>(s2);
  unsigned long long hi = static_cast<unsigned long long>(s2 >> 64);
  warp_sum_u128(lo, hi);
  if (lane == 0) {
    f.red_a[warp] = s1;
    f.red_b[warp] = lo;
    f.red_c[warp] = hi;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned __int128 t1 = 0, t2 = 0;
    for (int w = 0; w < NW; ++w) {
      t1 += f.red_a[w];
      t2 += (static_cast<unsigned __int128>(f.red_c[w]) << 64) | f.red_b[w];
    }
    f.sig = moments_std(__ldcg(&us->n_pool), t1, t2);
  }
  __syncthreads();
  finalize_stats<NT>(kp, u, us, __ldcg(&us->median_t), f.sig);
}

// Coarse histogram uh of every kept row of a unit, by one CTA: round 1 of a
// unit whose block left its value window starts over from it.
template <int DT, int NT>
__device__ void count_coarse_rows(const DevUnit& u, const uint8_t* Fc, uint32_t* uh) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, SEG = 64 * VS, NW = NT / kWarp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = u.T, nseg = (T + SEG - 1) / SEG;
  const bool vin = (u.flags & kUnitInVec) != 0;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  for (int k = tid; k < kCoarseBins; k += NT) uh[k] = 0u;
  __syncthreads();
  for (int task = warp; task < u.C * nseg; task += NW) {
    const int r = task / nseg, s = task - r * nseg;
    if (Fc[r]) continue;
    const uint8_t* grow = gin + static_cast<int64_t>(r) * u.in_stride * TR::kBytes;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int x = s * SEG + q * 32 * VS + lane * VS;
      if (x < T) {
        uint32_t v[VS];
        gload_vec<DT>(grow, x, T, vin, v);
#pragma unroll
        for (int j = 0; j < VS; ++j)
          if (x + j < T) atomicAdd(&uh[coarse_key(v[j])], 1u);
      }
    }
  }
  __syncthreads();
}

// Round 1 of a unit counted in its value window (after the frequency pass):
// takes the rows the frequency pass flagged out of the counts, then finds the
// exact median and MAD of the pooled powers -- the same order statistics as
// the bin-list selection -- from the window counts, provided they and every
// count they rest on lie inside the window.  With the cumulative counts
// cle(y) = #{x <= y}, exact for wlo - 1 <= y < wlo + kWinVals: the r-th
// smallest value is the least y with cle(y) >= r + 1, and the r-th smallest
// distance |2x - M2| is the least d with c(d) = cle(endB(d)) -
// cle(endA(d) - 1) >= r + 1 (c grows with d, and so does the range it reads,
// so the search stops at the first d that either reaches r + 1 or reads past
// the window).  Returns false, having written nothing, when they do not.
template <int DT, int NT>
__device__ bool window_resolve(const KParams& kp, const DevUnit& u, UnitState* us, uint8_t* ws,
                               Fixed<NT>& f) {
  using TR = Traits<DT>;
  constexpr int NW = NT / kWarp, PER = static_cast<int>(kWinVals) / NT;
  static_assert(PER * NT == static_cast<int>(kWinVals), "whole counters per thread");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = u.T;
  const uint32_t wlo = f.wlo;
  // Workspace: flagged-row list [0, 8K), Fc [34K, 36K) from the frequency
  // pass, the window counts [36K, 52K)
  const uint8_t* Fc = ws + 2 * kMaxChan * sizeof(unsigned long long) + kMaxChan;
  int* frows = reinterpret_cast<int*>(ws);
  uint32_t* sp = reinterpret_cast<uint32_t*>(ws + 36 * 1024);
  for (int k = tid; k < static_cast<int>(kWinVals); k += NT) sp[k] = __ldcg(us->spec + k);
  if (warp == 0) {
    int n = 0;
    for (int base = 0; base < u.C; base += kWarp) {
      const int c = base + lane;
      const bool fl = c < u.C && Fc[c];
      const unsigned bal = __ballot_sync(kFull, fl);
      if (fl) frows[n + __popc(bal & ((1u << lane) - 1u))] = c;
      n += __popc(bal);
    }
    if (lane == 0) f.n_keep = n;
  }
  __syncthreads();
  // the stats tasks counted every row: take out the flagged ones
  const int nfr = f.n_keep;
  uint32_t nb = 0;
  if (nfr > 0) {
    // warps over (flagged row, segment of 32 * NQ vectors): the NQ loads of a
    // segment are in flight together
    constexpr int VS = TR::kVec, NQ = 32 / VS, SEG = 32 * NQ * VS;
    const int nseg = (T + SEG - 1) / SEG;
    const bool vin = (u.flags & kUnitInVec) != 0;
    const uint8_t* gin = static_cast<const uint8_t*>(u.in);
    const uint64_t pol = l2_policy_drop();
    for (int task = warp; task < nfr * nseg; task += NW) {
      const int i = task / nseg, s = task - i * nseg;
      const uint8_t* grow = gin + static_cast<int64_t>(frows[i]) * u.in_stride * TR::kBytes;
      uint4 v[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int x = s * SEG + q * 32 * VS + lane * VS;
        v[q] = x < T ? gload_raw<DT>(grow, x, T, vin, pol) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int x = s * SEG + q * 32 * VS + lane * VS;
#pragma unroll
        for (int j = 0; j < VS; ++j) {
          if (x + j < T) {
            const uint32_t val = raw_pw<DT>(v[q], j), t = val - wlo;
            if (t < kWinVals) atomicSub(&sp[t], 1u);
            else nb += val < wlo ? 1u : 0u;
          }
        }
      }
    }
  }
  nb = warp_sum32(nb);
  if (lane == 0) f.red_u32[warp] = nb;
  __syncthreads();
  if (tid == 0) {
    long long b = __ldcg(&us->win_below);
    for (int w = 0; w < NW; ++w) b -= f.red_u32[w];
    f.wbelow = b;
  }
  // inclusive prefix of the window counts, PER consecutive counters a thread
  uint32_t loc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) loc[k] = sp[tid * PER + k];
#pragma unroll
  for (int k = 1; k < PER; ++k) loc[k] += loc[k - 1];
  uint32_t wt;
  const uint32_t ex = warp_excl_scan(loc[PER - 1], lane, &wt);
  __syncthreads();
  if (lane == 0) f.red_u32[warp] = wt;
  __syncthreads();
  uint32_t off = ex;
  for (int w = 0; w < warp; ++w) off += f.red_u32[w];
#pragma unroll
  for (int k = 0; k < PER; ++k) sp[tid * PER + k] = off + loc[k];
  __syncthreads();
  if (warp == 0) {
    // warp 0: 32-ary searches (each step probes 32 points of the range)
    const long long N = __ldcg(&us->n_pool), below = f.wbelow, inw = sp[kWinVals - 1];
    bool ok = below >= 0 && below + inw <= N;
    if (!ok && lane == 0) set_error(kp, kErrInternal, 50);
    // least x in [a, b] with pred(x), pred monotone and true at b (whole warp)
    auto first_true = [&](long long a, long long b, auto pred) -> long long {
      while (a < b) {
        const long long step = (b - a + 31) / 32;
        const long long x = a + lane * step;
        const unsigned bal = __ballot_sync(kFull, x >= b || pred(x));
        if (bal == 0u) {  // every probe below the answer: it lies in (x_31, b]
          a = a + 31 * step + 1;
          continue;
        }
        const int fl = __ffs(bal) - 1;
        const long long xf = a + fl * step;
        if (xf < b) b = xf;
        if (fl > 0) a = a + (fl - 1) * step + 1;
      }
      return a;
    };
    // the r-th smallest value (0-based)
    auto vrank = [&](long long r, long long* y) -> bool {
      const long long q = r + 1 - below;
      if (q < 1 || q > inw) return false;
      *y = static_cast<long long>(wlo) +
           first_true(0, kWinVals - 1, [&](long long i) { return static_cast<long long>(sp[i]) >= q; });
      return true;
    };
    auto cle = [&](long long y, bool* exact) -> long long {
      if (y < static_cast<long long>(wlo)) {  // y = wlo - 1 (-1 when wlo = 0): the count below
        if (y + 1 < static_cast<long long>(wlo)) *exact = false;
        return below;
      }
      if (y >= static_cast<long long>(wlo) + kWinVals) {
        *exact = false;
        return below + inw;
      }
      return below + sp[y - wlo];
    };
    const long long r1 = (N & 1) ? (N - 1) / 2 : N / 2 - 1, r2 = (N & 1) ? r1 : N / 2;
    long long v1 = 0, v2 = 0;
    ok = ok && N > 0 && vrank(r1, &v1) && vrank(r2, &v2);
    const long long M2 = v1 + v2;
    // the r-th smallest distance: least d in [0, 2 kWinVals + 2] (beyond it
    // endB leaves the window) with c(d) >= r + 1 or an inexact c(d)
    auto dist = [&](long long r, long long* D) -> bool {
      const long long a = first_true(0, 2ll * kWinVals + 2, [&](long long m) {
        bool e = true;
        const long long c = cle(endB(M2, m), &e) - cle(endA(M2, m) - 1, &e);
        return !e || c >= r + 1;
      });
      bool e = true;
      const long long c = cle(endB(M2, a), &e) - cle(endA(M2, a) - 1, &e);
      *D = a;
      return e && c >= r + 1;
    };
    long long d1 = 0, d2 = 0;
    ok = ok && dist(r1, &d1) && ((N & 1) ? (d2 = d1, true) : dist(r2, &d2));
    if (lane == 0) {
      f.resolved = ok ? 1 : 0;
      f.m2lo = M2;
      f.da[0] = d1 + d2;
    }
  }
  __syncthreads();
  if (!f.resolved) return false;
  finish_selected<NT>(kp, u, us, f.m2lo, f.da[0], __ldcg(&us->n_pool));
  return true;
}

// ------------------------------------------------------------------ unit-wide steps

// After the last stats task of a unit: frequency pass, pooled coarse
// histogram of the kept channels and the selection plan.  Releases the unit
// with ready = 1 (fine counts needed) or 2 (statistics final).
template <int DT, int NT>
__device__ LOFK_TASK_FN void unit_round1(const KParams& kp, const DevUnit& u, UnitState* us, uint8_t* ws,
                            Fixed<NT>& f) {
  using TR = Traits<DT>;
  constexpr int NW = NT / kWarp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = u.T;
  frequency_pass<NT>(kp, u, us, ws, f);
  bool recounted = false;
  if (__ldcg(&us->state) != kStateDone && f.wmode) {
    if (!window_resolve<DT, NT>(kp, u, us, ws, f)) {
      // the block left its value window: count its kept rows in full
      if (tid == 0 && kp.counters) atomicAdd(kp.counters + 1, 1);
      count_coarse_rows<DT, NT>(u, ws + 2 * kMaxChan * sizeof(unsigned long long) + kMaxChan,
                                reinterpret_cast<uint32_t*>(ws + 24 * 1024));
      recounted = true;
    } else if (__ldcg(&us->state) == kStateMoments) {
      unit_moments<DT, NT>(kp, u, us, ws, f);
    }
  }
  if (__ldcg(&us->state) != kStateDone && (!f.wmode || recounted)) {
    // Workspace (bytes): the bin list lo [0, 8K), hi [8K, 16K), cum [16K,
    // 24K) once the flagged rows are out; before that the key -> offset map
    // [0, 4.2K) and the flagged-row list [4.5K, 6.25K); histogram [24K,
    // 28.2K); Fc [34K, 36K) (from the frequency pass); spec counts [36K, 52K).
    const uint8_t* Fc = ws + 2 * kMaxChan * sizeof(unsigned long long) + kMaxChan;
    uint32_t* uh = reinterpret_cast<uint32_t*>(ws + 24 * 1024);
    uint32_t* sp = reinterpret_cast<uint32_t*>(ws + 36 * 1024);
    if (recounted) {
      if (tid == 0) f.n_tgt = 0;
      __syncthreads();
    } else {
    if (tid < kWarp) {
      int nt = 0;
      if (kp.hist.hint && u.hist_slot >= 0)
        nt = spec_targets(__ldcg(kp.hist.hint + 2 * u.hist_slot),
                          __ldcg(kp.hist.hint + 2 * u.hist_slot + 1), f.tgt);
      if (tid == 0) f.n_tgt = nt;
    }
    for (int k = tid; k < kCoarseBins; k += NT) uh[k] = __ldcg(us->coarse + k);
    for (int k = tid; k < kMaxSpec; k += NT) sp[k] = __ldcg(us->spec + k);
    __syncthreads();
    const int nspec_t = f.n_tgt;
    // the stats tasks histogrammed every row: take out the flagged ones
    // (warps over (flagged row, segment) pairs, loads one segment ahead)
    constexpr int VS = TR::kVec, NQ = 4, SEG = 32 * NQ * VS;
    const int nseg = (T + SEG - 1) / SEG;
    const bool vin = (u.flags & kUnitInVec) != 0;
    const uint8_t* gin = static_cast<const uint8_t*>(u.in);
    int* frows = reinterpret_cast<int*>(ws + 4 * 1024 + 512);  // [4.5K, 6.25K): up to 448 rows
    uint32_t* moff = reinterpret_cast<uint32_t*>(ws);           // [0, 4.2K): key -> offset
    for (int i = tid; i < kCoarseBins; i += NT) moff[i] = kNoTarget;
    __syncthreads();
    if (tid < nspec_t) moff[coarse_key(f.tgt[tid].lo)] = f.tgt[tid].base - f.tgt[tid].lo;
    const uint32_t nsc = nspec_t ? f.tgt[nspec_t - 1].base + (f.tgt[nspec_t - 1].hi - f.tgt[nspec_t - 1].lo) + 1u : 0u;
    if (tid == 0) {
      int nf = 0;
      for (int c = 0; c < u.C; ++c)
        if (Fc[c]) {
          if (nf < 448) frows[nf] = c;
          ++nf;
        }
      f.n_keep = nf;
    }
    __syncthreads();
    const int nfr = f.n_keep;
    unsigned long long s1 = 0;
    unsigned __int128 s2 = 0;
    for (int fb = 0; fb < nfr; fb += 448) {
      if (fb > 0) {
        __syncthreads();
        if (tid == 0) {
          int nf = 0, seen = 0;
          for (int c = 0; c < u.C && nf < 448; ++c)
            if (Fc[c] && seen++ >= fb) frows[nf++] = c;
        }
        __syncthreads();
      }
      const int nfb = min(448, nfr - fb);
      const int nsegs = nfb * nseg;
      const uint64_t pol = l2_policy_drop();
      uint4 cur[NQ], nxt[NQ];
      auto load_seg = [&](int task, uint4 (&v)[NQ]) {
        const int i = task / nseg, s = task - i * nseg;
        const uint8_t* grow = gin + static_cast<int64_t>(frows[min(i, nfb - 1)]) * u.in_stride * TR::kBytes;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int x = s * SEG + q * 32 * VS + lane * VS;
          v[q] = (task < nsegs && x < T) ? gload_raw<DT>(grow, x, T, vin, pol) : make_uint4(0u, 0u, 0u, 0u);
        }
      };
      load_seg(warp, cur);
      for (int task = warp; task < nsegs; task += NW) {
        load_seg(task + NW, nxt);
        const int s = task % nseg;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int x = s * SEG + q * 32 * VS + lane * VS;
#pragma unroll
          for (int j = 0; j < VS; ++j) {
            if (x + j >= T) continue;
            const uint32_t val = raw_pw<DT>(cur[q], j);
            const uint32_t key = coarse_key(val);
            atomicSub(&uh[key], 1u);
            const uint32_t si = val + moff[key];
            if (si < nsc) atomicSub(&sp[si], 1u);
            if (kp.sigma_std) {
              s1 += val;
              s2 += static_cast<unsigned long long>(val) * val;
            }
          }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) cur[q] = nxt[q];
      }
    }
    if (kp.sigma_std) {
      s1 = warp_sum64(s1);
      unsigned long long lo = static_cast<unsigned long long>(s2);
      unsigned long long hi = static_cast<unsigned long long>(s2 >> 64);
      warp_sum_u128(lo, hi);
      if (lane == 0) {
        f.red_a[warp] = s1;
        f.red_b[warp] = lo;
        f.red_c[warp] = hi;
      }
    }
    __syncthreads();
    if (tid == 0 && kp.sigma_std) {
      unsigned __int128 t1 = (static_cast<unsigned __int128>(__ldcg(us->mom + 1)) << 64) |
                             __ldcg(us->mom + 0);
      unsigned __int128 t2 = (static_cast<unsigned __int128>(__ldcg(us->mom + 3)) << 64) |
                             __ldcg(us->mom + 2);
      for (int w = 0; w < NW; ++w) {
        t1 -= f.red_a[w];
        t2 -= (static_cast<unsigned __int128>(f.red_c[w]) << 64) | f.red_b[w];
      }
      us->mom[0] = static_cast<unsigned long long>(t1);
      us->mom[1] = static_cast<unsigned long long>(t1 >> 64);
      us->mom[2] = static_cast<unsigned long long>(t2);
      us->mom[3] = static_cast<unsigned long long>(t2 >> 64);
      us->mom_ready = 1;
    }
    __syncthreads();
    }  // counts of the stats tasks
    const int nspec_t = f.n_tgt;
    const BinList B0 = build_coarse_list<NT>(kp, us, uh, ws);
    // merge the value-by-value counts of the hinted bins (as a fine round)
    if (tid == 0) {
      int nt = 0, nsc = 0;
      for (int t = 0; t < nspec_t; ++t) {
        int a = 0, b = B0.n;  // bin with lo == target lo
        while (a < b) {
          const int mid = (a + b) >> 1;
          if (B0.lo[mid] < f.tgt[t].lo) a = mid + 1;
          else b = mid;
        }
        if (a < B0.n && B0.lo[a] == f.tgt[t].lo && B0.hi[a] == f.tgt[t].hi) {
          us->tgt[nt] = f.tgt[t];
          us->tgt_bin[nt] = a;
          ++nt;
        }
        nsc = static_cast<int>(f.tgt[t].base + (f.tgt[t].hi - f.tgt[t].lo) + 1u);
      }
      us->n_targets = nt;
      us->n_fine = nsc;
      f.n_tgt = nt;
      f.state = nsc;
    }
    __syncthreads();
    if (f.n_tgt > 0) {
      for (int i = tid; i < f.state; i += NT) us->fine[i] = sp[i];
      __syncthreads();
      merge_fine<NT>(kp, us, ws, f);
      const BinList B = load_bins<NT>(us, ws, __ldcg(&us->n_bins));
      select_plan<NT>(kp, u, us, B, f);
    } else {
      select_plan<NT>(kp, u, us, B0, f);
    }
    if (__ldcg(&us->state) == kStateMoments) unit_moments<DT, NT>(kp, u, us, ws, f);
  }
  __syncthreads();
  if (tid == 0) {
    const bool fine = __ldcg(&us->state) == kStateFine;
    if ((fine || recounted) && kp.counters) atomicAdd(kp.counters, 1);
    // a unit that needs refinement rounds is finished by the same CTA
    // (task_stats), which releases it then
    if (!fine) {
      __threadfence();
      st_release(&us->ready, 2);
    }
  }
}

// After the last fine task of a unit: merge the counts, plan again; further
// rounds (rare) are counted here over every kept row of the unit.
template <int DT, int NT>
__device__ LOFK_TASK_FN void unit_round2(const KParams& kp, const DevUnit& u, UnitState* us, uint8_t* ws,
                            Fixed<NT>& f) {
  for (int guard = 0;; ++guard) {
    merge_fine<NT>(kp, us, ws, f);
    const BinList B = load_bins<NT>(us, ws, __ldcg(&us->n_bins));
    select_plan<NT>(kp, u, us, B, f);
    if (__ldcg(&us->state) != kStateFine || guard > kMaxRounds) break;
    if (threadIdx.x == 0 && kp.counters) atomicAdd(kp.counters + 1, 1);
    count_fine_rows<DT, NT>(kp, u, us, 0, u.C, ws, f);
  }
  if (__ldcg(&us->state) == kStateMoments) unit_moments<DT, NT>(kp, u, us, ws, f);
  if (__ldcg(&us->state) != kStateDone) {  // did not converge: no time pass
    finalize_stats<NT>(kp, u, us, 0.0, 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(&us->ready, 2);
  }
}

// ------------------------------------------------------------------ tasks

// One shared-memory count, by a reduction without return value; predicated:
// only when p holds.
__device__ __forceinline__ void red_shared_inc(uint32_t addr) {
  asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
}
// Adds 1 to the shared counter at byte address base + 4 * t when t < n
// (unsigned): the comparison and the reduction in one predicated pair.
__device__ __forceinline__ void red_shared_inc_below(uint32_t t, uint32_t n, uint32_t base) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t.reg .u32 a;\n\tsetp.lt.u32 q, %0, %1;\n\t"
      "mad.lo.u32 a, %0, 4, %2;\n\t@q red.shared.add.u32 [a], 1;\n\t}" ::"r"(t),
      "r"(n), "r"(base)
      : "memory");
}

// Row power sums (spectrum) of rows [row0, row0 + R) of a unit into f.rowS,
// and one count per sample: WIN, its value's counter in the value window
// [wlo, wlo + kWinVals) (win), values below the window in the returned
// per-thread total and those above it nowhere; otherwise its value's counter
// inside a target bin (win = the spec counters, via the key -> offset map
// moff), else its coarse bin (hist).  Warp w owns rows w, w + NW, ... and
// walks their segments in order, the loads of its next segment in flight
// while it counts the current one; a row's sum is reduced once, when the
// warp leaves the row.  WIN needs
// 1 <= wlo <= 2^31 - kWinVals, so that val - wlo is exact as a signed value
// for every power (at most 2^31).
template <int DT, int NT, bool WIN>
__device__ __forceinline__ uint32_t stats_rows(const DevUnit& u, int row0, int R, uint32_t* hist,
                                               uint32_t* win, const uint32_t* moff, uint32_t nsc,
                                               uint32_t wlo, Fixed<NT>& f) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, NQ = 32 / VS, SEG = 32 * NQ * VS, NW = NT / kWarp;
  // per-lane row sums: 32 bits hold a lane's share of a ci8 row (powers at
  // most 2^15, a lane's share at most 2^17 of them for any admissible row)
  using Acc = std::conditional_t<DT == LOF_CI8, uint32_t, unsigned long long>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int T = u.T, nseg = (T + SEG - 1) / SEG;
  const bool vin = (u.flags & kUnitInVec) != 0;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  const int nk = (warp < R ? (R - warp + NW - 1) / NW : 0) * nseg;  // segments of this warp
  const uint64_t pol = l2_policy_drop();
  const uint32_t wsa = saddr(win), hsa = saddr(hist);
  uint4 cur[NQ], nxt[NQ];
  uint32_t below = 0;
  // the warp's k-th segment: segment s = k % nseg of row warp + kr * NW,
  // kr = k / nseg (the pair advanced step by step, no division)
  auto load_seg = [&](int k, int kr, int s, uint4 (&v)[NQ]) {
    const uint8_t* grow =
        gin + static_cast<int64_t>(row0 + min(warp + kr * NW, R - 1)) * u.in_stride * TR::kBytes;
    if (k < nk && vin && s * SEG + SEG <= T) {  // a whole segment: plain vector loads
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        v[q] = ldg_policy(grow + static_cast<size_t>(s * SEG + q * 32 * VS + lane * VS) * TR::kBytes, pol);
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int x = s * SEG + q * 32 * VS + lane * VS;
        v[q] = (k < nk && x < T) ? gload_raw<DT>(grow, x, T, vin, pol) : make_uint4(0u, 0u, 0u, 0u);
      }
    }
  };
  Acc sum = 0;
  load_seg(0, 0, 0, cur);
  int kr = 0, s = 0;
  for (int k = 0; k < nk; ++k) {
    const int sn = s + 1 == nseg ? 0 : s + 1, krn = s + 1 == nseg ? kr + 1 : kr;
    load_seg(k + 1, krn, sn, nxt);
    {  // the segment after that toward L2, one 128-byte line a lane
      const int s2 = sn + 1 == nseg ? 0 : sn + 1, kr2 = sn + 1 == nseg ? krn + 1 : krn;
      constexpr int LINES = SEG * TR::kBytes / 128;
      if (k + 2 < nk && s2 * SEG + SEG <= T && lane < LINES) {
        const uint8_t* g2 = gin + static_cast<int64_t>(row0 + warp + kr2 * NW) * u.in_stride * TR::kBytes +
                            static_cast<size_t>(s2) * SEG * TR::kBytes + lane * 128;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(g2));
      }
    }
    auto count = [&](uint32_t val) {
      sum += val;
      if constexpr (WIN) {
        const int t = static_cast<int>(val - wlo);
        below += static_cast<uint32_t>(t) >> 31;
        red_shared_inc_below(static_cast<uint32_t>(t), kWinVals, wsa);
      } else {
        // the value's counter inside a target bin (the bin's coarse count is
        // rebuilt from those below), else its bin
        const uint32_t key = coarse_key(val);
        const uint32_t si = val + moff[key];  // spec index, or >= nsc off the targets
        red_shared_inc(si < nsc ? wsa + 4u * si : hsa + 4u * key);
      }
    };
    if (s * SEG + SEG <= T) {  // a whole segment: no bound per vector
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int j = 0; j < VS; ++j) count(raw_pw<DT>(cur[q], j));
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int x = s * SEG + q * 32 * VS + lane * VS;
#pragma unroll
        for (int j = 0; j < VS; ++j)
          if (x + j < T) count(raw_pw<DT>(cur[q], j));
      }
    }
    if (s == nseg - 1) {  // the warp leaves the row: its sum
      const unsigned long long rs = warp_sum64(static_cast<unsigned long long>(sum));
      if (lane == 0) f.rowS[warp + kr * NW] = rs;
      sum = 0;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) cur[q] = nxt[q];
    kr = krn;
    s = sn;
  }
  return below;
}

// Stats task: row power sums (spectrum) and the counts of its rows -- value
// window counts when the unit has one, else the coarse histogram with exact
// counts in the hinted bins.
template <int DT, int NT>
__device__ LOFK_TASK_FN void task_stats(const KParams& kp, const DevUnit& u, UnitState* us, const Task& tk,
                           uint8_t* ws, Fixed<NT>& f) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, NW = NT / kWarp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = u.T, R = tk.nrows, row0 = tk.row0;
  const bool vin = (u.flags & kUnitInVec) != 0;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws);                     // [0, 4.2K)
  uint32_t* spec = reinterpret_cast<uint32_t*>(ws + 6 * 1024);           // [6K, 22K)
  uint32_t* moff = reinterpret_cast<uint32_t*>(ws + 22 * 1024);          // [22K, 26.2K)
  const bool hinted = kp.hist.hint && u.hist_slot >= 0;
  if (tid == 0) {
    uint32_t wlo = 0;
    f.wmode = (hinted && !kp.sigma_std && (kp.schedule & LOF_SCHED_VALUE_WINDOW) &&
               hint_window(__ldcg(kp.hist.hint + 2 * u.hist_slot),
                           __ldcg(kp.hist.hint + 2 * u.hist_slot + 1), &wlo))
                  ? 1
                  : 0;
    f.wlo = wlo;
  }
  __syncthreads();
  const bool wmode = f.wmode != 0;
  if (tid < kWarp) {
    int nt = 0;
    if (hinted && !wmode)
      nt = spec_targets(__ldcg(kp.hist.hint + 2 * u.hist_slot),
                        __ldcg(kp.hist.hint + 2 * u.hist_slot + 1), f.tgt);
    if (tid == 0) f.n_tgt = nt;
  }
  if (!wmode) {
    for (int i = tid; i < kCoarseBins; i += NT) {
      hist[i] = 0u;
      moff[i] = kNoTarget;
    }
  }
  for (int i = tid; i < kMaxSpec; i += NT) spec[i] = 0u;
  for (int r = tid; r < R; r += NT) f.rowS[r] = 0;
  __syncthreads();
  const int nspec_t = f.n_tgt;
  if (tid < nspec_t) moff[coarse_key(f.tgt[tid].lo)] = f.tgt[tid].base - f.tgt[tid].lo;
  const uint32_t nsc = nspec_t ? f.tgt[nspec_t - 1].base + (f.tgt[nspec_t - 1].hi - f.tgt[nspec_t - 1].lo) + 1u : 0u;
  __syncthreads();
  const uint32_t below = wmode ? stats_rows<DT, NT, true>(u, row0, R, hist, spec, moff, nsc, f.wlo, f)
                               : stats_rows<DT, NT, false>(u, row0, R, hist, spec, moff, nsc, 0u, f);
  if (kp.sigma_std) {
    // exact 128-bit moments for the std estimator, in a pass of their own
    constexpr int SEG2 = 64 * VS;
    const int nseg2 = (T + SEG2 - 1) / SEG2;
    unsigned long long s1 = 0;
    unsigned __int128 s2 = 0;
    for (int task = warp; task < R * nseg2; task += NW) {
      const int r = task / nseg2, s = task - r * nseg2;
      const uint8_t* grow = gin + static_cast<int64_t>(row0 + r) * u.in_stride * TR::kBytes;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int x = s * SEG2 + q * 32 * VS + lane * VS;
        if (x < T) {
          uint32_t v[VS];
          gload_vec<DT>(grow, x, T, vin, v);
#pragma unroll
          for (int j = 0; j < VS; ++j) {
            s1 += v[j];
            s2 += static_cast<unsigned long long>(v[j]) * v[j];
          }
        }
      }
    }
    s1 = warp_sum64(s1);
    unsigned long long lo = static_cast<unsigned long long>(s2);
    unsigned long long hi = static_cast<unsigned long long>(s2 >> 64);
    warp_sum_u128(lo, hi);
    if (lane == 0) {
      f.red_a[warp] = s1;
      f.red_b[warp] = lo;
      f.red_c[warp] = hi;
    }
  }
  if (wmode) {
    const uint32_t b = warp_sum32(below);
    if (lane == 0 && b) atomicAdd(&us->win_below, static_cast<int>(b));
  }
  __syncthreads();
  // coarse counts of the target bins: the sums of their value counters (one
  // warp per bin)
  for (int t = warp; t < nspec_t; t += NW) {
    const Target g = f.tgt[t];
    uint32_t c = 0;
    for (uint32_t i = g.base + lane; i <= g.base + (g.hi - g.lo); i += kWarp) c += spec[i];
    c = warp_sum32(c);
    if (lane == 0) hist[coarse_key(g.lo)] += c;
  }
  __syncthreads();
  for (int r = tid; r < R; r += NT) kp.chan_S[u.chan_off + row0 + r] = f.rowS[r];
  if (!wmode) {
    for (int k = tid; k < kCoarseBins; k += NT) {
      const uint32_t h = hist[k];
      if (h) atomicAdd(us->coarse + k, h);
    }
  }
  const int nflush = wmode ? static_cast<int>(kWinVals) : static_cast<int>(nsc);
  for (int i = tid; i < nflush; i += NT) {
    const uint32_t h = spec[i];
    if (h) atomicAdd(us->spec + i, h);
  }
  if (tid == 0 && kp.sigma_std) {
    unsigned __int128 t1 = 0, t2 = 0;
    for (int w = 0; w < NW; ++w) {
      t1 += f.red_a[w];
      t2 += (static_cast<unsigned __int128>(f.red_c[w]) << 64) | f.red_b[w];
    }
    atomic_add_u128(us->mom + 0, t1);
    atomic_add_u128(us->mom + 2, t2);
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const int old = atomicAdd(&us->done_S, 1);
    f.last = (old + 1 == u.nS) ? 1 : 0;
    if (f.last) __threadfence();
  }
  __syncthreads();
  if (f.last) {
    unit_round1<DT, NT>(kp, u, us, ws, f);
    if (__ldcg(&us->state) == kStateFine) {
      // round 1 left bins to refine (no hint, or the data moved away from
      // it): this CTA counts them over every kept row of the unit, then
      // plans further rounds until the statistics are exact
      if (threadIdx.x == 0 && kp.counters) atomicAdd(kp.counters + 1, 1);
      count_fine_rows<DT, NT>(kp, u, us, 0, u.C, ws, f);
      unit_round2<DT, NT>(kp, u, us, ws, f);
    }
  }
}

// Fine task: exact counts in the refined bins for its kept rows (skipped when
// the first round already made the statistics exact).
template <int DT, int NT>
__device__ LOFK_TASK_FN void task_fine(const KParams& kp, const DevUnit& u, UnitState* us, const Task& tk,
                          uint8_t* ws, Fixed<NT>& f) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    if (!wait_geq(kp, &us->ready, 1, 300)) f.ok = 0;
    f.state = f.ok ? __ldcg(&us->ready) : 0;
  }
  __syncthreads();
  if (!f.ok || f.state == 2) return;
  count_fine_rows<DT, NT>(kp, u, us, tk.row0, tk.row0 + tk.nrows, ws, f);
  if (tid == 0) {
    if (kp.counters) atomicAdd(kp.counters + 1, 1);
    __threadfence();
    const int old = atomicAdd(&us->done_F, 1);
    f.last = (old + 1 == u.nF) ? 1 : 0;
    if (f.last) __threadfence();
  }
  __syncthreads();
  if (f.last) unit_round2<DT, NT>(kp, u, us, ws, f);
}

// A row flagged whole: mask all ones, data all zero.  One warp.
template <int DT>
__device__ void write_row_flagged(const DevUnit& u, int c, int T) {
  using TR = Traits<DT>;
  const int lane = threadIdx.x & 31;
  if (u.mask) {
    uint8_t* mr = u.mask + static_cast<int64_t>(c) * u.mask_stride;
    for (int x = lane; x < T; x += 32) mr[x] = 1;
  }
  if (u.out) {
    uint8_t* orow = static_cast<uint8_t*>(u.out) + static_cast<int64_t>(c) * u.out_stride * TR::kBytes;
    for (int x = lane; x < T; x += 32) TR::zero(orow, x);
  }
}

// Flag task: SumThreshold in time on its kept rows (Section 2.1), the history
// test (Section 4.1), the mask and the masked data.
template <int DT, int NT>
__device__ LOFK_TASK_FN void task_flag(const KParams& kp, const DevUnit& u, UnitState* us, const Task& tk,
                          uint8_t* ws, Fixed<NT>& f, uint32_t* s_Kp) {
  using TR = Traits<DT>;
  constexpr int VS = TR::kVec, SEG = 64 * VS, NW = NT / kWarp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = u.T, R = tk.nrows, row0 = tk.row0;
  const int nch = (T + 31) >> 5;
  const int MW = nch + 4;  // flag words per row, two zero words on each side
  const int nseg = (T + SEG - 1) / SEG;
  const StLayout L = st_layout(nch);
  // shared memory: the flag words of the task's R rows.  The general
  // (any-magnitude) path keeps Rb rows of prefix and of fire words in this
  // CTA's region of a global scratch (L2-resident; the path is rare).
  uint32_t* const smbits = reinterpret_cast<uint32_t*>(ws);
  uint32_t* const spfx = kp.gen_scratch + static_cast<int64_t>(blockIdx.x) * kp.gen_words;
  const int Rb = max(1, min(R, kp.gen_words / (L.per_row + MW)));
  uint32_t* const sfbits = spfx + Rb * L.per_row;
  const uint8_t* gin = static_cast<const uint8_t*>(u.in);
  if (tid == 0) {
    if (!wait_geq(kp, &us->ready, 2, 400)) f.ok = 0;
  }
  __syncthreads();
  if (!f.ok) return;
  for (int i = tid; i < kKTable; i += NT) f.K[i] = __ldcg(us->K + i);
  for (int r = tid; r < R; r += NT) {
    f.rowFc[r] = __ldcg(kp.chan_Fc + u.chan_off + row0 + r);
    f.rowS[r] = __ldcg(kp.chan_S + u.chan_off + row0 + r);
    f.rowFlagSum[r] = 0;
    f.rowNFlag[r] = 0;
    f.rowFh[r] = 0;
    // the history thresholds of the task's rows (Section 4.1), read once here
    const long long h = u.hist_slot >= 0 ? u.hist_slot + row0 + r : -1;
    uint8_t on = 0;
    double thr = 0.0;
    if (kp.enable_history && h >= 0) {
      const int cnt = kp.hist.count[h];
      if (cnt >= kp.history_min && cnt > 0) {
        on = 1;
        thr = kp.hist.thr[h];
      }
    }
    f.rowHon[r] = on;
    f.rowThr[r] = thr;
  }
  for (int i = tid; i < R * MW; i += NT) smbits[i] = 0u;
  if (tid == 0) {
    f.rows_done = 0;
    f.row_next = NW;
    f.time_on = __ldcg(&us->time_on);
    int kmax = 0;
    while (kmax < kp.max_log_window && (2 << kmax) <= T) ++kmax;
    f.kmax_t = kmax;
  }
  __syncthreads();
  if (tid == 0) {
    int nk = 0;
    for (int r = 0; r < R; ++r)
      if (!f.rowFc[r]) f.keep[nk++] = r;
    f.n_keep = nk;
  }
  // packed-path tables and guard (see the time pass helpers), one entry per thread
  bool bad = false;
  {
    const int total = koffset(f.kmax_t + 1);
    if (f.K[0] < 0 || f.K[0] >= (1ll << 20)) bad = true;
    for (int e = tid; e < total; e += NT) {
      int k = 0;
      while (koffset(k + 1) <= e) ++k;
      const int n = e - koffset(k);
      const long long* Kt = f.K + koffset(k);
      if (Kt[n] < 0 || Kt[n] >= static_cast<long long>(kZ)) bad = true;
      if (k == 0) {
        s_Kp[e] = static_cast<uint32_t>(Kt[n]);
      } else if (k <= 5) {
        if (Kt[n] >= (1ll << 25)) bad = true;  // 64 * Kt + 63 < 2^31
        s_Kp[e] = (static_cast<uint32_t>(Kt[n]) << kLowShift) + 63u;
      } else {
        s_Kp[e] = static_cast<uint32_t>(n) * kZ + static_cast<uint32_t>(Kt[n]);
      }
    }
    // prefilter bounds of the windows I >= 8 (see wr_fire_pf): c = Kt[I - 1] + 1,
    // Cb - 1 = min_n (Kt[n] + n * c).  The bound holds for any c >= 0; c = 0
    // (every nonzero union a candidate) where c > 2^21 (a factor that grows
    // with I), so that the union sums stay below 2^28.
    if (tid >= 3 && tid <= f.kmax_t) {
      const int k = tid, I = 1 << k;
      const long long* Kt = f.K + koffset(k);
      long long c = Kt[I - 1] + 1;
      if (c > (1ll << 21)) c = 0;
      long long m = Kt[0];
      for (int n = 1; n <= I; ++n) m = min(m, Kt[n] + n * c);
      s_Kp[kKbOff + 2 * k] = static_cast<uint32_t>(c);
      s_Kp[kKbOff + 2 * k + 1] = static_cast<uint32_t>(min(max(m, 0ll), (1ll << 30)));
    }
  }
  if (!(kp.schedule & LOF_SCHED_PACKED)) bad = true;  // schedule: the general path for every row
  bad = __syncthreads_or(bad);
  if (tid == 0) f.state = bad ? 0 : 1;
  __syncthreads();
  const int nkeep = f.n_keep;

  // ---- time pass over the kept rows of the task
  if (f.time_on && nkeep > 0) {
    if (f.state == 1) {
      // packed values: one warp per row (its segments one after the other,
      // each in registers, mask and data written as soon as they are final),
      // then the row's history test and, when it fires, the whole row flagged.
      // The warp's items (row, segment) are staged one ahead in its two
      // buffers, after the rows' flag words.
      using ST = WrStage<DT, kWrNpl>;
      const bool vin = (u.flags & kUnitInVec) != 0;
      const int nsg = wr_seg_count<kWrNpl>(T);
      uint8_t* const stage = ws + ((4 * R * MW + 15) & ~15) + warp * 2 * ST::kBufBytes;
      const uint64_t pol = l2_policy_drop();  // the input's last read
      // items (kept row k, segment) are claimed one at a time, item i being
      // segment i % nsg of kept row i / nsg (warp w starts with item w), so the
      // warps of a task finish within about one segment of each other.  The
      // segments of a row add their flagged counts and unflagged sums into
      // the row's accumulators (rowNFlag, rowFlagSum); the rows' history tests,
      // the rows it flags whole and the zeroes of in-place rows follow the
      // task's barrier below.
      // item / nsg as a multiply-high: m = ceil(2^32 / nsg) gives the exact
      // quotient for items below 2^32 / nsg (here below 64 * nsg)
      const uint32_t mq = nsg > 1 ? static_cast<uint32_t>((0x100000000ull + nsg - 1) / nsg) : 0u;
      auto item_row = [&](int it) {
        return nsg > 1 ? static_cast<int>(__umulhi(static_cast<uint32_t>(it), mq)) : it;
      };
      auto stage_item = [&](int it, int buf) {
        const int k = item_row(it);
        const WrSeg g = wr_seg<kWrNpl>(T, it - k * nsg);
        wr_stage<DT, kWrNpl>(stage + buf * ST::kBufBytes + lane * ST::kRowBytes,
                             gin + static_cast<int64_t>(row0 + f.keep[k]) * u.in_stride * TR::kBytes, g.xl, T,
                             vin, pol);
      };
      const int n_items = nkeep * nsg;
      int it = warp < n_items ? warp : -1, buf = 0;
      if (it >= 0) stage_item(it, 0);
      while (it >= 0) {
        int claim = 0;
        if (lane == 0) claim = atomicAdd(&f.row_next, 1);
        claim = __shfl_sync(kFull, claim, 0);
        const int in = claim < n_items ? claim : -1;
        const int kc = item_row(it), sg = it - kc * nsg;
        const int c = row0 + f.keep[kc], r = c - row0;
        uint8_t* const srow = stage + buf * ST::kBufBytes + lane * ST::kRowBytes;
        WrOut o;
        o.out = u.out ? static_cast<uint8_t*>(u.out) + static_cast<int64_t>(c) * u.out_stride * TR::kBytes
                      : nullptr;
        o.mask = u.mask ? u.mask + static_cast<int64_t>(c) * u.mask_stride : nullptr;
        o.inplace = (u.flags & kUnitInPlace) != 0;
        o.vout = (u.flags & kUnitOutVec) != 0;
        o.mask_vec = (u.flags & kUnitMaskVec) != 0;
        o.vin = vin;
        // out-of-place rows with 16-byte aligned output: the data goes out
        // with coalesced stores after the pass, and with it the mask bytes of
        // 16-byte aligned mask rows
        uint8_t* const coal_row =
            ((kp.schedule & LOF_SCHED_COALESCED) && o.out && !o.inplace && o.vout) ? o.out : nullptr;
        uint8_t* const coal_mask = (coal_row && o.mask && o.mask_vec) ? o.mask : nullptr;
        if (coal_row) o.out = nullptr;
        if (coal_mask) o.mask = nullptr;
        o.enabled = o.out != nullptr || o.mask != nullptr;
        const WrSeg g = wr_seg<kWrNpl>(T, sg);
        cp_async_wait_all();  // this item's samples (the only group in flight)
        WrRow<kWrNpl> Rw;
        wr_build<DT, kWrNpl>(Rw, srow, s_Kp[0]);
        if (in >= 0) {
          // the next item into the other buffer as early as possible (the
          // input comes from DRAM), once the bulk stores of its last item
          // have read it
          bulk_wait_read();
          stage_item(in, buf ^ 1);
        }
        wr_passes<kWrNpl>(Rw, g, 1, f.kmax_t, s_Kp, (kp.schedule & LOF_SCHED_BOUND64) != 0);
        int nfl = 0;
        unsigned long long su = 0;
        wr_finish<DT, kWrNpl>(Rw, g, T, srow, smbits + r * MW + 2, o, nfl, su);
        if (coal_row)
          wr_store_coalesced<DT, kWrNpl>(stage + buf * ST::kBufBytes, Rw.M[0], g, T, coal_row, coal_mask);
        // the row's counts: its history test and any whole-row flagging
        // follow the task's barrier, once every segment of the row is written
        if (lane == 0) {
          atomicAdd(&f.rowNFlag[r], nfl);
          atomicAdd(&f.rowFlagSum[r], su);
        }
        it = in;
        buf ^= 1;
      }
      bulk_wait_all();  // buffers free for the next task; data stored
      if (tid == 0) f.rows_done = 1;
      __syncthreads();
    } else {
      // any magnitudes: exact 64-bit window sums over a shared-memory prefix,
      // Rb rows at a time
      for (int kb = 0; kb < nkeep; kb += Rb) {
        const int* rows = f.keep + kb;
        const int nbb = min(Rb, nkeep - kb);
        st_build<DT, NT>(u, row0, T, nch, rows, nbb, spfx, L, smbits, MW, false, 0u);
        for (int i = tid; i < nbb * MW; i += NT) sfbits[i] = 0u;
        __syncthreads();
        st_bases<NT>(spfx, L, nch, nbb, nullptr);
        __syncthreads();
        for (int k = 0; k <= f.kmax_t; ++k) {
          const int I = 1 << k;
          const long long* Kt = f.K + koffset(k);
          for (int c = tid; c < nbb * nch; c += NT) {
            const int rb = c / nch, w = c - rb * nch, t0 = w << 5;
            uint32_t* F = sfbits + rb * MW + 2;
            const int nvalid = T - I + 1 - t0;
            if (nvalid <= 0) {
              F[w] = 0u;
              continue;
            }
            const uint32_t vm = nvalid >= 32 ? 0xFFFFFFFFu : ((1u << nvalid) - 1u);
            const uint32_t* pl = spfx + rb * L.per_row;
            const uint32_t* pb = pl + L.PLW;
            F[w] = general_fire(pl, pb, smbits + rows[rb] * MW + 2, t0, I, T, Kt) & vm;
          }
          __syncthreads();
          // new flags: windows that fired flag all their samples (snapshot)
          for (int c = tid; c < nbb * nch; c += NT) {
            const int rb = c / nch, w = c - rb * nch;
            const uint32_t* F = sfbits + rb * MW + 2;
            const uint32_t f0 = F[w], f1 = F[w - 1], f2 = F[w - 2];
            if ((f0 | f1 | f2) == 0u) continue;
            const uint32_t D = (I <= 32) ? dilate32(f0, f1, I)
                                         : (dilate32(f0, f1, 32) | dilate32(f1, f2, 32));
            smbits[rows[rb] * MW + 2 + w] |= D;
          }
          __syncthreads();
        }
        // flagged counts and flagged powers of the batch's rows (re-read)
        for (int c = tid; c < nbb * nch; c += NT) {
          const int kr = c / nch, w = c - kr * nch;
          const int r = rows[kr];
          uint32_t m = smbits[r * MW + 2 + w];
          if (m) {
            const uint8_t* grow = gin + static_cast<int64_t>(row0 + r) * u.in_stride * TR::kBytes;
            unsigned long long fs = 0;
            const int cnt = __popc(m);
            while (m) {
              const int j = __ffs(m) - 1;
              m &= m - 1u;
              fs += TR::at(grow, (w << 5) + j);
            }
            atomicAdd(&f.rowNFlag[r], cnt);
            atomicAdd(&f.rowFlagSum[r], fs);
          }
        }
        __syncthreads();
      }
    }
  }
  // ---- history flagger (Section 4.1) and per-row counts (rows the packed
  // time pass has not finished)
  const bool rows_done = f.rows_done != 0;
  for (int r = tid; r < R; r += NT) {
    const long long h = u.hist_slot >= 0 ? u.hist_slot + row0 + r : -1;
    unsigned long long add_total;
    if (f.rowFc[r]) {
      if (h >= 0) kp.hist.pend_flag[h] = 0;
      add_total = static_cast<unsigned long long>(T);
    } else {
      const int nfl = f.rowNFlag[r];
      const int n = T - nfl;
      uint8_t fh = 0;
      if (n > 0) {
        // the packed pass accumulates the unflagged sum, the general path the flagged one
        const unsigned long long su = rows_done ? f.rowFlagSum[r] : f.rowS[r] - f.rowFlagSum[r];
        const double cur = __ddiv_rn(__ull2double_rn(su), static_cast<double>(n));
        double staged = cur;
        if (f.rowHon[r]) {
          const double thr = f.rowThr[r];
          if (!(cur < thr)) {
            fh = 1;
            staged = thr;
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
      f.rowFh[r] = fh;
      atomicAdd(&f.cnt_time, static_cast<unsigned long long>(nfl));
      if (fh) atomicAdd(&f.cnt_hist, 1ull);
      add_total = fh ? static_cast<unsigned long long>(T) : static_cast<unsigned long long>(nfl);
    }
    atomicAdd(&f.cnt_total, add_total);
  }
  __syncthreads();

  // ---- apply: mask bytes and masked data, streamed row by row (Sections 3, 4)
  {
    const bool inplace = (u.flags & kUnitInPlace) != 0;
    const bool mask_vec = (u.flags & kUnitMaskVec) != 0;
    const bool vin = (u.flags & kUnitInVec) != 0;
    const bool vout = (u.flags & kUnitOutVec) != 0;
    constexpr uint32_t kVm = (1u << VS) - 1u;
    constexpr int NQO = 16 / VS, SEGO = 32 * NQO * VS;
    const int nsego = (T + SEGO - 1) / SEGO;
    const uint64_t pol_drop = l2_policy_drop();
    // rows of the packed time pass were written by the warps that flagged
    // them; only rows flagged whole (frequency pass, history test) and the
    // zeroes of in-place rows remain
    const bool fused = rows_done;
    // rows first (each warp reads the rows' flags; rows with nothing left
    // are skipped whole), their segments striped over the warps
    for (int r = 0; r < R; ++r) {
      const bool full = f.rowFc[r] || f.rowFh[r];
      if (fused && !full && !(inplace && u.out)) continue;
      for (int s = warp; s < nsego; s += NW) {
        const uint32_t* M = smbits + r * MW + 2;
        const int64_t grow_idx = static_cast<int64_t>(row0 + r);
        uint4 win[NQO];
        if (u.out && !inplace && vin && vout && !full) {
#pragma unroll
          for (int q = 0; q < NQO; ++q) {
            const int x = s * SEGO + q * 32 * VS + lane * VS;
            if (x + VS <= T)
              win[q] = ldg_policy(gin + grow_idx * u.in_stride * TR::kBytes +
                                      static_cast<size_t>(x) * TR::kBytes, pol_drop);
          }
        }
#pragma unroll
        for (int q = 0; q < NQO; ++q) {
          const int x = s * SEGO + q * 32 * VS + lane * VS;
          if (x >= T) continue;
          const int nv = min(VS, T - x);
          const uint32_t valid = nv >= VS ? kVm : ((1u << nv) - 1u);
          const uint32_t bits = full ? valid : ((M[x >> 5] >> (x & 31)) & valid);
          if (u.mask) {
            uint8_t* mrow = u.mask + grow_idx * u.mask_stride;
            if (mask_vec && nv == VS) {
              if constexpr (VS == 4) {
                st_stream_u32(mrow + x, (bits * 0x00204081u) & 0x01010101u);
              } else {
                const uint32_t lo = ((bits & 0xFu) * 0x00204081u) & 0x01010101u;
                const uint32_t hi = (((bits >> 4) & 0xFu) * 0x00204081u) & 0x01010101u;
                st_stream_u64(mrow + x, lo, hi);
              }
            } else {
              for (int j = 0; j < nv; ++j) mrow[x + j] = static_cast<uint8_t>((bits >> j) & 1u);
            }
          }
          if (u.out) {
            uint8_t* orow = static_cast<uint8_t*>(u.out) + grow_idx * u.out_stride * TR::kBytes;
            if (inplace) {
              uint32_t m = bits;
              while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1u;
                TR::zero(orow, x + j);
              }
            } else if (vin && vout && nv == VS) {
              uint4 w = make_uint4(0u, 0u, 0u, 0u);
              if (bits != kVm) {
                w = win[q];
                if (bits) {
                  uint32_t wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                  for (int j = 0; j < VS; ++j) {
                    if ((bits >> j) & 1u) {
                      if constexpr (VS == 4) wd[j] = 0u;
                      else wd[j >> 1] &= (j & 1) ? 0x0000FFFFu : 0xFFFF0000u;
                    }
                  }
                  w = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                }
              }
              __stcs(reinterpret_cast<uint4*>(orow + static_cast<size_t>(x) * TR::kBytes), w);
            } else {
              const uint8_t* irow = gin + grow_idx * u.in_stride * TR::kBytes;
              for (int j = 0; j < nv; ++j) {
                if ((bits >> j) & 1u) TR::zero(orow, x + j);
                else TR::copy(orow + static_cast<size_t>(x + j) * TR::kBytes,
                              irow + static_cast<size_t>(x + j) * TR::kBytes);
              }
            }
          }
        }
      }
    }
  }
  if (tid == 0 && u.stats) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&u.stats->n_flag_time), f.cnt_time);
    atomicAdd(reinterpret_cast<unsigned long long*>(&u.stats->n_chan_hist), f.cnt_hist);
    atomicAdd(reinterpret_cast<unsigned long long*>(&u.stats->n_flag_total), f.cnt_total);
  }
}

// ------------------------------------------------------------------ scheduling

__device__ __forceinline__ bool task_ready(const KParams& kp, int t) {
  const Task tk = kp.tasks[t];
  if (tk.kind == kTaskStats) return true;
  const int r = ld_acquire(&kp.ustate[tk.unit].ready);
  return tk.kind == kTaskFine ? r >= 1 : r >= 2;
}

// Thread 0: the next task to run, or -1 when the queue is drained.  A task
// whose unit is not ready yet (fine / flag tasks wait for the unit's
// statistics) is parked in a small per-CTA list and the next task is taken
// instead; parked tasks run as soon as they are ready.  Stats tasks never
// wait, fine tasks wait only on stats tasks and flag tasks only on fine
// tasks, and a CTA that polls always re-checks every task it holds, so the
// waits cannot form a cycle.  Gives up after kp.spin_limit ns without
// progress (error word set).
template <int NT>
__device__ int sched_next(const KParams& kp, Fixed<NT>& f) {
  constexpr int kDefer = 8;
  unsigned long long t0 = 0;
  for (;;) {
    for (int i = 0; i < f.n_def; ++i) {
      const int t = f.def[i];
      if (task_ready(kp, t)) {
        f.def[i] = f.def[--f.n_def];
        return t;
      }
    }
    if (!f.q_done && f.n_def <= kDefer) {
      const int t = atomicAdd(kp.queue, 1);
      if (t >= kp.n_tasks) {
        f.q_done = 1;
        continue;
      }
      if (task_ready(kp, t)) return t;
      f.def[f.n_def++] = t;
      continue;
    }
    if (f.n_def == 0) return -1;
    if (*reinterpret_cast<volatile int*>(kp.err) != 0) return -1;
    if (t0 == 0) t0 = global_ns();
    else if (global_ns() - t0 > static_cast<unsigned long long>(kp.spin_limit)) {
      set_error(kp, kErrTimeout, 500);
      return -1;
    }
    __nanosleep(256);
  }
}

// ------------------------------------------------------------------ the kernel
// Persistent loop over the task queue.  Tasks wait (bounded) only on tasks
// that precede them in the queue, so no CTA ever waits on work that has not
// been handed out.

// Compiled twice per input type and CTA size: PH = 0 runs the statistics
// launch (stats tasks and the unit-wide steps), PH = 1 the flag launch (flag
// tasks); each holds only its own code, so each launch's instruction
// footprint stays small.
template <int DT, int NT, int PH>
__global__ void __launch_bounds__(NT, NT == 128 ? 4 : 2) lof_block_kernel(const KParams kp) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ Fixed<NT> f;
  __shared__ uint32_t s_Kp[PH == 1 ? kKTable + 2 * 8 : 1];
  const int tid = threadIdx.x;
  if (tid == 0) {
    f.q_done = 0;
    f.n_def = 0;
  }
  for (;;) {
    if (tid == 0) {
      f.item = sched_next<NT>(kp, f);
      f.ok = 1;
      f.cnt_time = f.cnt_total = f.cnt_hist = 0;
    }
    __syncthreads();
    const int ti = f.item;
    if (ti < 0) break;
    const Task tk = kp.tasks[ti];
    const DevUnit u = kp.units[tk.unit];
    UnitState* const us = kp.ustate + tk.unit;
    if constexpr (PH == 0) {
      if (tk.kind == kTaskStats) task_stats<DT, NT>(kp, u, us, tk, smem, f);
      else if (tk.kind == kTaskFine) task_fine<DT, NT>(kp, u, us, tk, smem, f);
      else if (tid == 0) set_error(kp, kErrInternal, 60);  // a flag task in the statistics queue
    } else {
      if (tk.kind == kTaskFlag) task_flag<DT, NT>(kp, u, us, tk, smem, f, s_Kp);
      else if (tid == 0) set_error(kp, kErrInternal, 61);
    }
    __syncthreads();
    if (!f.ok) break;
  }
}

template <int DT, int NT>
void* kernel_ptr(int phase) {
  return phase ? reinterpret_cast<void*>(&lof_block_kernel<DT, NT, 1>)
               : reinterpret_cast<void*>(&lof_block_kernel<DT, NT, 0>);
}

}  // namespace
}  // namespace lofk

// This file is compiled once per input type (LOF_KERNEL_DT = LOF_CI16 or
// LOF_CI8) so that the two instantiations build in parallel; the CI16 object
// also holds the history commit kernel and the launchers.
#if !defined(LOF_KERNEL_DT) || (LOF_KERNEL_DT != 1 && LOF_KERNEL_DT != 2)
#error "compile with -DLOF_KERNEL_DT=2 (ci16) or -DLOF_KERNEL_DT=1 (ci8)"
#endif

#if LOF_KERNEL_DT == 2  // LOF_CI16
extern "C" void* lofk_block_kernel_ci16(int threads, int phase) {
  if (threads == 128) return lofk::kernel_ptr<LOF_CI16, 128>(phase);
  if (threads == 256) return lofk::kernel_ptr<LOF_CI16, 256>(phase);
  return nullptr;
}
#else  // LOF_CI8
extern "C" void* lofk_block_kernel_ci8(int threads, int phase) {
  if (threads == 128) return lofk::kernel_ptr<LOF_CI8, 128>(phase);
  if (threads == 256) return lofk::kernel_ptr<LOF_CI8, 256>(phase);
  return nullptr;
}
#endif

#if LOF_KERNEL_DT == 2
extern "C" void* lofk_block_kernel_ci8(int threads, int phase);

namespace lofk {
namespace {

// ------------------------------------------------------------------ history commit
// Section 4.1: add each staged value to its channel's ring and refresh the
// cached threshold mean + k * stddev (population, oldest -> newest, binary64
// without contraction).
__global__ void lof_commit_kernel(const CommitParams cp, int total, int refresh_only) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int a = 0, b = cp.n_units;  // unit with chan_off <= g
  while (b - a > 1) {
    const int m = (a + b) >> 1;
    if (cp.units[m].chan_off <= g) a = m;
    else b = m;
  }
  const DevUnit& u = cp.units[a];
  const int c = g - u.chan_off;
  if (c < 0 || c >= u.C || u.hist_slot < 0) return;
  const long long h = u.hist_slot + c;
  const HistoryDev& H = cp.hist;
  int cnt = H.count[h];
  int head = H.head[h];
  if (!refresh_only) {
    if (!H.pend_flag[h]) return;
    H.vals[h * H.H + head] = H.pend[h];
    head = (head + 1) % H.H;
    cnt = min(cnt + 1, H.H);
    H.head[h] = head;
    H.count[h] = cnt;
    H.pend_flag[h] = 0;
  }
  if (cnt <= 0) {
    H.thr[h] = 0.0;
    return;
  }
  const int oldest = (head - cnt + H.H) % H.H;
  double s = 0.0;
  for (int i = 0; i < cnt; ++i) s = __dadd_rn(s, H.vals[h * H.H + (oldest + i) % H.H]);
  const double mu = __ddiv_rn(s, static_cast<double>(cnt));
  double q = 0.0;
  for (int i = 0; i < cnt; ++i) {
    const double d = __dsub_rn(H.vals[h * H.H + (oldest + i) % H.H], mu);
    q = __dadd_rn(q, __dmul_rn(d, d));
  }
  const double sd = __dsqrt_rn(__ddiv_rn(q, static_cast<double>(cnt)));
  H.thr[h] = __dadd_rn(mu, __dmul_rn(cp.history_k, sd));
}

void* pick_kernel(int dtype, int threads, int phase) {
  if (dtype == LOF_CI16) return lofk_block_kernel_ci16(threads, phase);
  if (dtype == LOF_CI8) return lofk_block_kernel_ci8(threads, phase);
  return nullptr;
}

}  // namespace
}  // namespace lofk

using namespace lofk;

extern "C" int lofk_set_smem_limit(int dtype, int smem_bytes) {
  for (int t : {128, 256})
    for (int ph : {0, 1}) {
      void* k = pick_kernel(dtype, t, ph);
      if (!k) return -1;
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
          cudaSuccess)
        return -2;
    }
  return 0;
}

// Resident CTAs per SM of both launches of a block (the smaller).
extern "C" int lofk_max_blocks_per_sm(int dtype, int threads, int smem_bytes, int* out) {
  int best = 1 << 30;
  for (int ph : {0, 1}) {
    void* k = pick_kernel(dtype, threads, ph);
    if (!k) return -1;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
        cudaSuccess)
      return -2;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem_bytes) != cudaSuccess)
      return -3;
    best = std::min(best, n);
  }
  *out = best;
  return 0;
}

// The block kernel's entry of an input type, CTA size and launch (0 the
// statistics launch, 1 the flag launch), or NULL.
extern "C" void* lofk_block_kernel(int dtype, int threads, int phase) {
  return pick_kernel(dtype, threads, phase);
}

extern "C" int lofk_launch_block(int dtype, const KParams* kp, int grid, int threads,
                                 int smem_bytes, void* stream, int cooperative, int phase) {
  void* k = pick_kernel(dtype, threads, phase);
  if (!k) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(static_cast<unsigned>(threads));
  cfg.dynamicSmemBytes = static_cast<size_t>(smem_bytes);
  cfg.stream = static_cast<cudaStream_t>(stream);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = cooperative ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<KParams*>(kp)};
  const cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  return e == cudaSuccess ? 0 : static_cast<int>(e);
}

extern "C" int lofk_launch_commit(const CommitParams* cp, int total_channels, void* stream) {
  if (total_channels <= 0) return 0;
  const int bs = 256;
  const int grid = (total_channels + bs - 1) / bs;
  lof_commit_kernel<<<grid, bs, 0, static_cast<cudaStream_t>(stream)>>>(*cp, total_channels, 0);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : static_cast<int>(e);
}

extern "C" int lofk_launch_refresh(const CommitParams* cp, int total_channels, void* stream) {
  if (total_channels <= 0) return 0;
  const int bs = 256;
  const int grid = (total_channels + bs - 1) / bs;
  lof_commit_kernel<<<grid, bs, 0, static_cast<cudaStream_t>(stream)>>>(*cp, total_channels, 1);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : static_cast<int>(e);
}
#endif  // LOF_KERNEL_DT == 2
