// lof_sir.cu -- the scale-invariant rank (SIR) operator of Section 2.2 on the
// final mask of a block, along time on every channel and then along frequency
// on every time step (optional: lof_params.sir_percent > 0).
//
// Definition: with eta = percent / 100, a sample is flagged when some interval
// holding it has at least (1 - eta) of its samples flagged.  With integer
// weights w = +percent (flagged) and -(100 - percent) (unflagged) and prefix
// sums Q[0] = 0, Q[i + 1] = Q[i] + w[i], sample x qualifies exactly when
// max_{b > x} Q[b] >= min_{a <= x} Q[a].  Integer arithmetic throughout, so the
// result is exact.
//
// One warp runs the operator on one line (a channel's row, or one time step's
// column) in tiles of 32 lanes x NPT positions: a first pass gives each tile's
// weight sum and the extremes of its prefix sums (warp scans), lane 0 chains
// them along the line, and a second pass gives every lane the prefix minimum
// before it and the suffix maximum after it, from which its NPT decisions
// follow in registers.  Newly flagged samples get mask 1 and zero data, and
// are added to the unit's flag count.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "lof_internal.h"

namespace lofk {
namespace {

constexpr unsigned kFullS = 0xFFFFFFFFu;
constexpr int kSirMaxTiles = 128;   // per line: 128 tiles (time rows up to 131072 samples)
constexpr int kSirWarps = 8;        // warps per CTA
constexpr int kSirStrip = 32;       // time steps per CTA of the frequency pass

__device__ __forceinline__ int warp_excl_add(int v, int lane) {
  int s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFullS, s, o);
    if (lane >= o) s += y;
  }
  return s - v;
}
__device__ __forceinline__ int warp_excl_min(int v, int lane) {  // min over lanes < lane
  int s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFullS, s, o);
    if (lane >= o) s = min(s, y);
  }
  const int e = __shfl_up_sync(kFullS, s, 1);
  return lane == 0 ? INT32_MAX : e;
}
__device__ __forceinline__ int warp_excl_max_after(int v, int lane) {  // max over lanes > lane
  int s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_down_sync(kFullS, s, o);
    if (lane + o < 32) s = max(s, y);
  }
  const int e = __shfl_down_sync(kFullS, s, 1);
  return lane == 31 ? INT32_MIN : e;
}

// Per-line tile summaries of one warp: weight sum, min of the prefix sums over
// the tile's starts a (relative to the tile start), max over its ends b.
struct SirTiles {
  int sum[kSirMaxTiles], mn[kSirMaxTiles], mx[kSirMaxTiles];
};

// The operator on a line of L samples.  lt(k, f) fills f[0..NPT) with the
// 0/1 flags of the lane's samples k * 32 * NPT + lane * NPT + i (0 past L);
// st(x, g, f) receives the result g and the input flag f of sample x.
template <int NPT, class LT, class ST>
__device__ __forceinline__ void sir_line(int L, int percent, SirTiles& tl, LT lt, ST st) {
  const int lane = threadIdx.x & 31;
  constexpr int TILE = 32 * NPT;
  const int nt = (L + TILE - 1) / TILE;
  const int wp = percent, wn = -(100 - percent);
  // pass 1: tile summaries
  for (int k = 0; k < nt; ++k) {
    int f[NPT];
    lt(k, f);
    int q = 0, mn = 0, mx = INT32_MIN;
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
      const int x = k * TILE + lane * NPT + i;
      const int w = x < L ? (f[i] ? wp : wn) : 0;
      mn = min(mn, q);  // a = position i
      q += w;
      mx = max(mx, q);  // b = position i + 1
    }
    const int ex = warp_excl_add(q, lane);
    int tmn = ex + mn, tmx = ex + mx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tmn = min(tmn, __shfl_xor_sync(kFullS, tmn, o));
      tmx = max(tmx, __shfl_xor_sync(kFullS, tmx, o));
    }
    if (lane == 31) tl.sum[k] = ex + q;
    if (lane == 0) {
      tl.mn[k] = tmn;
      tl.mx[k] = tmx;
    }
  }
  __syncwarp();
  // along the line (lane 0): base of each tile, prefix minimum before it
  // (kept in mn) and suffix maximum after it (kept in mx)
  if (lane == 0) {
    int base = 0, pm = INT32_MAX;
    for (int k = 0; k < nt; ++k) {
      const int s = tl.sum[k], m = tl.mn[k];
      tl.sum[k] = base;
      tl.mn[k] = pm;
      pm = min(pm, base + m);
      tl.mx[k] += base;  // absolute max of the tile's ends
      base += s;
    }
    int sm = INT32_MIN;
    for (int k = nt - 1; k >= 0; --k) {
      const int m = tl.mx[k];
      tl.mx[k] = sm;
      sm = max(sm, m);
    }
  }
  __syncwarp();
  // pass 2: decisions
  for (int k = 0; k < nt; ++k) {
    int f[NPT], q[NPT + 1];
    lt(k, f);
    q[0] = 0;
    int mn = 0, mx = INT32_MIN;
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
      const int x = k * TILE + lane * NPT + i;
      const int w = x < L ? (f[i] ? wp : wn) : 0;
      mn = min(mn, q[i]);
      q[i + 1] = q[i] + w;
      mx = max(mx, q[i + 1]);
    }
    const int base = tl.sum[k] + warp_excl_add(q[NPT], lane);
    const int pm = min(tl.mn[k], warp_excl_min(base + mn, lane));
    const int sm = max(tl.mx[k], warp_excl_max_after(base + mx, lane));
    int suf[NPT];
    int s = sm;
#pragma unroll
    for (int i = NPT - 1; i >= 0; --i) {
      s = max(s, base + q[i + 1]);
      suf[i] = s;
    }
    int m = pm;
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
      const int x = k * TILE + lane * NPT + i;
      m = min(m, base + q[i]);
      if (x < L) st(x, suf[i] >= m ? 1 : 0, f[i]);
    }
  }
  __syncwarp();
}

// Unit of global channel g (units ordered by chan_off).
__device__ __forceinline__ int unit_of(const DevUnit* units, int n_units, int64_t g) {
  int a = 0, b = n_units;
  while (b - a > 1) {
    const int m = (a + b) >> 1;
    if (units[m].chan_off <= g) a = m;
    else b = m;
  }
  return a;
}

__device__ __forceinline__ void zero_sample(void* row, int64_t t, int es) {
  if (es == 8) reinterpret_cast<unsigned long long*>(row)[t] = 0ull;
  else if (es == 4) reinterpret_cast<uint32_t*>(row)[t] = 0u;
  else reinterpret_cast<uint16_t*>(row)[t] = 0;
}

// Time direction: one warp per channel row.
__global__ void __launch_bounds__(32 * kSirWarps) lof_sir_time_kernel(const DevUnit* units, int n_units,
                                                                      int64_t n_chan, int percent,
                                                                      int es, int skip_upto) {
  __shared__ SirTiles tiles[kSirWarps];
  const int warp = threadIdx.x >> 5;
  const int64_t g = static_cast<int64_t>(blockIdx.x) * kSirWarps + warp;
  if (g >= n_chan) return;
  const int ui = unit_of(units, n_units, g);
  const DevUnit& u = units[ui];
  const int c = static_cast<int>(g - u.chan_off);
  if (c < 0 || c >= u.C || !u.mask || u.T > 32 * 32 * kSirMaxTiles || u.T <= skip_upto) return;
  uint8_t* mrow = u.mask + static_cast<int64_t>(c) * u.mask_stride;
  uint8_t* orow = u.out ? static_cast<uint8_t*>(u.out) + static_cast<int64_t>(c) * u.out_stride * es
                        : nullptr;
  int added = 0;
  const int T = u.T, lane = threadIdx.x & 31;
  const bool vec = (u.flags & kUnitMaskVec) != 0;
  auto lt = [&](int k, int (&f)[32]) {
    const int x0 = k * 1024 + lane * 32;
    if (vec && x0 + 32 <= T) {
      const uint4 a = *reinterpret_cast<const uint4*>(mrow + x0);
      const uint4 b = *reinterpret_cast<const uint4*>(mrow + x0 + 16);
      const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 32; ++i) f[i] = ((w[i >> 2] >> (8 * (i & 3))) & 0xFFu) != 0u;
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) f[i] = x0 + i < T ? (mrow[x0 + i] != 0) : 0;
    }
  };
  sir_line<32>(
      u.T, percent, tiles[warp], lt,
      [&](int x, int gval, int fval) {
        if (gval && !fval) {
          mrow[x] = 1;
          if (orow) zero_sample(orow, x, es);
          ++added;
        }
      });
  added = __reduce_add_sync(kFullS, added);
  if ((threadIdx.x & 31) == 0 && added && u.stats)
    atomicAdd(reinterpret_cast<unsigned long long*>(&u.stats->n_flag_total),
              static_cast<unsigned long long>(added));
}

// Time direction for rows of up to 32 * kSirRowBlocks samples: one thread per
// row (a channel), the row taken in blocks of 32 samples.  A forward pass over
// the blocks keeps, per block, the prefix sum at its start and the least
// prefix sum over the starts of the blocks before it (in shared memory,
// [block][thread]); a backward pass then reloads each block's flags,
// recomputes its prefix minima in registers and decides its samples from
// the last one down against the running maximum of the prefix sums after
// them -- the same integer prefix sums as the line form, no shuffles and no
// barriers.
constexpr int kSirRowThreads = 64;
constexpr int kSirRowBlocks = 96;  // rows up to 3072 samples

// Flag bits of samples [x, x + 32) of a mask row (0 past T), as a word.
__device__ __forceinline__ uint32_t mask_bits32(const uint8_t* mrow, int x, int T, bool vec) {
  uint32_t b = 0u;
  if (vec && x + 32 <= T) {
    const uint4 p = *reinterpret_cast<const uint4*>(mrow + x);
    const uint4 q = *reinterpret_cast<const uint4*>(mrow + x + 16);
    const uint32_t w[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 32; ++i) b |= (((w[i >> 2] >> (8 * (i & 3))) & 0xFFu) != 0u ? 1u : 0u) << i;
  } else {
    for (int i = 0; i < 32 && x + i < T; ++i) b |= (mrow[x + i] != 0 ? 1u : 0u) << i;
  }
  return b;
}

__global__ void __launch_bounds__(kSirRowThreads) lof_sir_time_rows_kernel(const DevUnit* units, int n_units,
                                                                          int64_t n_chan, int percent, int es) {
  __shared__ int s_qs[kSirRowBlocks][kSirRowThreads], s_pl[kSirRowBlocks][kSirRowThreads];
  const int tid = threadIdx.x;
  const int64_t g = static_cast<int64_t>(blockIdx.x) * kSirRowThreads + tid;
  if (g >= n_chan) return;  // no warp-wide step follows
  const DevUnit& u = units[unit_of(units, n_units, g)];
  const int c = static_cast<int>(g - u.chan_off);
  const int T = u.T;
  if (c < 0 || c >= u.C || !u.mask || T > 32 * kSirRowBlocks) return;
  uint8_t* const mrow = u.mask + static_cast<int64_t>(c) * u.mask_stride;
  uint8_t* const orow =
      u.out ? static_cast<uint8_t*>(u.out) + static_cast<int64_t>(c) * u.out_stride * es : nullptr;
  const bool vec = (u.flags & kUnitMaskVec) != 0;
  const int wp = percent, wn = percent - 100;
  const int nb = (T + 31) / 32;
  int q = 0, m = INT32_MAX;
  for (int b = 0; b < nb; ++b) {
    const uint32_t bits = mask_bits32(mrow, 32 * b, T, vec);
    const int n = min(32, T - 32 * b);
    s_qs[b][tid] = q;
    s_pl[b][tid] = m;
    for (int i = 0; i < n; ++i) {
      m = min(m, q);
      q += ((bits >> i) & 1u) ? wp : wn;
    }
  }
  int R = INT32_MIN, added = 0;
  for (int b = nb - 1; b >= 0; --b) {
    const uint32_t bits = mask_bits32(mrow, 32 * b, T, vec);
    const int n = min(32, T - 32 * b);
    int L[32];
    int l = s_pl[b][tid], qq = s_qs[b][tid], qe = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      l = min(l, qq);  // a = 32 b + i
      L[i] = l;
      qq += ((bits >> i) & 1u) ? wp : wn;
      if (i + 1 == n) qe = qq;  // Q at the block's last sample + 1
    }
    uint32_t nw = 0u;
#pragma unroll
    for (int i = 31; i >= 0; --i) {
      if (i < n) {
        R = max(R, qe);
        nw |= (R >= L[i] ? 1u : 0u) << i;
        qe -= ((bits >> i) & 1u) ? wp : wn;
      }
    }
    nw &= ~bits;
    while (nw) {
      const int i = __ffs(nw) - 1;
      nw &= nw - 1u;
      mrow[32 * b + i] = 1;
      if (orow) zero_sample(orow, 32 * b + i, es);
      ++added;
    }
  }
  if (added && u.stats)
    atomicAdd(reinterpret_cast<unsigned long long*>(&u.stats->n_flag_total), static_cast<unsigned long long>(added));
}

// Frequency direction: a CTA stages a strip of 32 time steps of every
// channel in shared memory (rows of 33 bytes), one warp per time step runs
// the operator down the channels, then the strip is written back.  Marks:
// bit 0 = flagged, bit 1 = newly flagged here.
__global__ void __launch_bounds__(32 * kSirWarps) lof_sir_freq_kernel(const DevUnit* units, int percent,
                                                                      int es, int skip_upto) {
  extern __shared__ uint8_t strip[];
  __shared__ SirTiles tiles[kSirWarps];
  __shared__ int s_added;
  const DevUnit& u = units[blockIdx.y];
  if (!u.mask || u.C > 32 * 8 * kSirMaxTiles || u.C <= skip_upto) return;
  const int C = u.C, T = u.T, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int RS = kSirStrip + 1;
  for (int t0 = blockIdx.x * kSirStrip; t0 < T; t0 += gridDim.x * kSirStrip) {
    if (threadIdx.x == 0) s_added = 0;
    if ((u.flags & kUnitMaskVec) && t0 + kSirStrip <= T) {
      for (int i = threadIdx.x; i < C * (kSirStrip / 4); i += blockDim.x) {
        const int c = i / (kSirStrip / 4), j = 4 * (i - c * (kSirStrip / 4));
        const uint32_t w =
            *reinterpret_cast<const uint32_t*>(u.mask + static_cast<int64_t>(c) * u.mask_stride + t0 + j);
#pragma unroll
        for (int b = 0; b < 4; ++b) strip[c * RS + j + b] = ((w >> (8 * b)) & 0xFFu) ? 1 : 0;
      }
    } else {
      for (int i = threadIdx.x; i < C * kSirStrip; i += blockDim.x) {
        const int c = i / kSirStrip, j = i - c * kSirStrip;
        strip[c * RS + j] = t0 + j < T ? (u.mask[static_cast<int64_t>(c) * u.mask_stride + t0 + j] ? 1 : 0) : 0;
      }
    }
    __syncthreads();
    for (int j = warp; j < kSirStrip && t0 + j < T; j += kSirWarps) {
      auto lt = [&](int k, int (&f)[8]) {
        const int c0 = k * 256 + lane * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = c0 + i < C ? (strip[(c0 + i) * RS + j] & 1) : 0;
      };
      sir_line<8>(
          C, percent, tiles[warp], lt,
          [&](int c, int gval, int fval) {
            if (gval && !fval) strip[c * RS + j] = 3;
          });
    }
    __syncthreads();
    int added = 0;
    for (int i = threadIdx.x; i < C * kSirStrip; i += blockDim.x) {
      const int c = i / kSirStrip, j = i - c * kSirStrip;
      if (t0 + j >= T || strip[c * RS + j] != 3) continue;
      u.mask[static_cast<int64_t>(c) * u.mask_stride + t0 + j] = 1;
      if (u.out) zero_sample(static_cast<uint8_t*>(u.out) + static_cast<int64_t>(c) * u.out_stride * es, t0 + j, es);
      ++added;
    }
    added = __reduce_add_sync(kFullS, added);
    if (lane == 0 && added) atomicAdd(&s_added, added);
    __syncthreads();
    if (threadIdx.x == 0 && s_added && u.stats)
      atomicAdd(reinterpret_cast<unsigned long long*>(&u.stats->n_flag_total),
                static_cast<unsigned long long>(s_added));
    __syncthreads();
  }
}

// Frequency direction for units of at most 32 * NW channels: one thread per
// time step (a column of the unit), its flags held as bits in registers, so
// the columns run independently with no shuffles and no barriers.  A forward
// pass over the column loads its flags and gives, per block of 32 channels,
// the prefix sum at the block's start and the least prefix sum over the
// block's starts a.  A backward pass over the blocks then recomputes each
// block's prefix minima min_{a <= x} Q[a] in registers (from the least prefix
// sum over the blocks before it) and decides the block's channels from the
// last one down against the running maximum max_{b > x} Q[b].  The same
// integer prefix sums as the line form above, so the same decisions.
constexpr int kSirColThreads = 128;
constexpr int kSirColWords = 8;  // channels up to 256

template <int NW>
__global__ void __launch_bounds__(kSirColThreads) lof_sir_freq_cols_kernel(const DevUnit* units, int percent,
                                                                          int es) {
  const DevUnit& u = units[blockIdx.y];
  const int C = u.C, T = u.T;
  if (!u.mask || C > 32 * NW) return;  // the line form takes the unit
  const int t = blockIdx.x * kSirColThreads + threadIdx.x;
  const bool on = t < T;
  const int wp = percent, wn = percent - 100;
  const int64_t ms = u.mask_stride;
  uint8_t* const mcol = u.mask + (on ? t : 0);
  uint32_t bits[NW];
  int qs[NW], lmin[NW];
  int q = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const int n = on ? min(32, C - 32 * w) : 0;
    uint32_t b = 0u;
    int mn = INT32_MAX;
    qs[w] = q;
#pragma unroll 8
    for (int i = 0; i < n; ++i) {
      const uint32_t fl = mcol[static_cast<int64_t>(32 * w + i) * ms] != 0 ? 1u : 0u;
      b = __funnelshift_r(b, fl, 1);  // bit 31 <- this flag; bit i after the shift below
      mn = min(mn, q);
      q += fl ? wp : wn;
    }
    bits[w] = n > 0 ? b >> (32 - n) : 0u;
    lmin[w] = mn;
  }
  int pl[NW];  // least prefix sum over the starts of the blocks before w
  {
    int m = INT32_MAX;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      pl[w] = m;
      m = min(m, lmin[w]);
    }
  }
  uint8_t* const orow = static_cast<uint8_t*>(u.out);
  int added = 0, R = INT32_MIN;
  // the block's decisions: FULL blocks hold 32 channels, the last may hold fewer
  auto block = [&](int w, int n, auto full) {
    constexpr bool FULL = decltype(full)::value;
    const uint32_t bw = bits[w];
    int L[32];
    int l = pl[w], qq = qs[w], qe = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      l = min(l, qq);  // a = 32 w + i
      L[i] = l;
      qq += ((bw >> i) & 1u) ? wp : wn;
      if (!FULL && i + 1 == n) qe = qq;
    }
    if (FULL) qe = qq;  // Q at the block's end
    uint32_t nb = 0u;
#pragma unroll
    for (int i = 31; i >= 0; --i) {
      if (FULL || i < n) {
        R = max(R, qe);  // b = 32 w + i + 1
        nb |= (R >= L[i] ? 1u : 0u) << i;
        qe -= ((bw >> i) & 1u) ? wp : wn;
      }
    }
    nb &= ~bw;
    while (nb) {
      const int i = __ffs(nb) - 1;
      nb &= nb - 1u;
      const int64_t c = 32 * w + i;
      mcol[c * ms] = 1;
      if (orow) zero_sample(orow + c * u.out_stride * es, t, es);
      ++added;
    }
  };
#pragma unroll
  for (int w = NW - 1; w >= 0; --w) {
    const int n = on ? min(32, C - 32 * w) : 0;
    if (n == 32) block(w, 32, std::true_type{});
    else if (n > 0) block(w, n, std::false_type{});
  }
  added = __reduce_add_sync(kFullS, added);
  if ((threadIdx.x & 31) == 0 && added && u.stats)
    atomicAdd(reinterpret_cast<unsigned long long*>(&u.stats->n_flag_total),
              static_cast<unsigned long long>(added));
}

}  // namespace
}  // namespace lofk

// Limit of the SIR pass: rows up to 131072 samples (the channel limit of a
// unit, 2048, is far below the frequency pass's 32768).
extern "C" int lofk_sir_max_time() { return 32 * 32 * lofk::kSirMaxTiles; }

// Both directions of the SIR operator over n_units device units (es: bytes
// per data sample).  max_chan sizes the frequency pass's shared strip.
extern "C" int lofk_launch_sir(const lofk::DevUnit* units, int n_units, int64_t n_chan, int max_chan,
                               int max_time, int percent, int es, void* stream) {
  using namespace lofk;
  if (n_units <= 0 || percent <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // time: rows of up to 3072 samples one thread per row, longer ones by the
  // line form (which skips the others)
  const int64_t nr = (n_chan + kSirRowThreads - 1) / kSirRowThreads;
  lof_sir_time_rows_kernel<<<static_cast<unsigned>(nr), kSirRowThreads, 0, st>>>(units, n_units, n_chan, percent,
                                                                               es);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return static_cast<int>(e);
  if (max_time > 32 * kSirRowBlocks) {
    const int64_t nb = (n_chan + kSirWarps - 1) / kSirWarps;
    lof_sir_time_kernel<<<static_cast<unsigned>(nb), 32 * kSirWarps, 0, st>>>(units, n_units, n_chan, percent,
                                                                            es, 32 * kSirRowBlocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_cast<int>(e);
  }
  // frequency: units of up to 256 channels one thread per time step, larger
  // ones by the line form (which skips the others)
  const unsigned gx = static_cast<unsigned>((std::max(1, max_time) + kSirColThreads - 1) / kSirColThreads);
  lof_sir_freq_cols_kernel<kSirColWords><<<dim3(gx, static_cast<unsigned>(n_units)), kSirColThreads, 0, st>>>(
      units, percent, es);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_cast<int>(e);
  if (max_chan <= 32 * kSirColWords) return 0;
  const int smem = max_chan * (kSirStrip + 1);
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(&lof_sir_freq_kernel),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return -2;
  lof_sir_freq_kernel<<<dim3(16, static_cast<unsigned>(n_units)), 32 * kSirWarps, smem, st>>>(
      units, percent, es, 32 * kSirColWords);
  e = cudaGetLastError();
  return e == cudaSuccess ? 0 : static_cast<int>(e);
}
