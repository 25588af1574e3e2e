// Device-side building blocks of the conformal Hough path (sm_103a).
//
// Fixed-point conventions (shared by every kernel of this library):
//   hits       int32 micrometres, |x|, |y| <= 2^24
//   map        u_q = floor(2 x 2^32 / r^2)   (Eq. 1 with the factor 2 that makes Eq. 2 hold)
//   trig       c_j = round(2^14 cos th_j), s_j = round(2^14 sin th_j), th_j = (j + 1/2) pi / N_theta
//   rho        rho_q = u_q c_j + v_q s_j     (matrix R of Sec. 3), 2^46 units per um^-1
//   bin        k = clamp(floor((rho_q + H) N_rho / 2H), 0, N_rho - 1), H = 703687442
//              (rho range [-0.01, 0.01] mm^-1 of Sec. 2)
#pragma once

#include <cstdint>
#include <type_traits>

#include "hough.h"

namespace hgpu {

// Cells given as a sorted candidate list (kSorted: lower(j, k), end(j), key(p), rows ascending in
// a column) let the rounds walk a column instead of looking every cell up.
template <class C, class = void>
struct sorted_cells : std::false_type {};
template <class C>
struct sorted_cells<C, std::void_t<decltype(C::kSorted)>> : std::bool_constant<C::kSorted> {};

// Phase timers (builds with HOUGH_PHASE_TIMERS defined): thread 0 of a CTA adds the clock64()
// cycles since its previous mark to the counter of the phase that just ended (HOUGH_PHASE_*).
// The mark lives in shared memory; the counters are per translation unit, and the fused
// kernel's are the ones hough_phase_cycles reads. Without the define the marks compile away.
#ifdef HOUGH_PHASE_TIMERS
static __device__ unsigned long long g_phase_cycles[HOUGH_PHASE_COUNT];
__device__ __forceinline__ unsigned long long& phase_mark() {
  __shared__ unsigned long long t;
  return t;
}
#define HOUGH_PHASE_START()                                     \
  do {                                                          \
    if (threadIdx.x == 0) hgpu::phase_mark() = clock64();       \
  } while (0)
#define HOUGH_PHASE(p)                                                          \
  do {                                                                          \
    if (threadIdx.x == 0) {                                                     \
      const unsigned long long t_ = clock64();                                  \
      atomicAdd(&hgpu::g_phase_cycles[(p)], t_ - hgpu::phase_mark());           \
      hgpu::phase_mark() = t_;                                                  \
    }                                                                           \
  } while (0)
#else
#define HOUGH_PHASE_START() \
  do {                      \
  } while (0)
#define HOUGH_PHASE(p) \
  do {                 \
  } while (0)
#endif

constexpr long long kH = HOUGH_RHO_HALF_RANGE;
constexpr int kTwoHm1 = (int)(2 * kH - 1);  // 1407374883 < 2^31
// |u_q|, |v_q| <= kFast32 keeps u c + v s + H inside int32: 2 * 44061 * 2^14 + H < 2^31.
constexpr int kFast32 = 44061;
constexpr int kCoordMax = 1 << 24;
constexpr int kMaxNTheta = 1024;

// floor(t * N_rho / 2H) for t in [0, 2^31) by one 32x32 high product and one 32x32+64
// multiply-add: M = ceil(2^64 N_rho / 2H) (M < 2^44) is split into 32-bit halves and
// floor(t M / 2^64) is exact because t * (M - 2^64 N_rho/2H) / 2^64 < 2^-33 < 1/2H, the
// smallest distance of t N_rho / 2H to the next integer above it.
struct BinMagic {
  uint32_t lo, hi;
};

__device__ __forceinline__ int bin_of_t(uint32_t t, BinMagic m) {
  const uint32_t h = __umulhi(t, m.lo);
  const unsigned long long s = (unsigned long long)t * m.hi + h;
  return (int)(s >> 32);
}

// Clamped bin of t = rho + H given in int32 (fast path).
__device__ __forceinline__ int rho_bin32(int t, BinMagic m) {
  t = min(max(t, 0), kTwoHm1);
  return bin_of_t((uint32_t)t, m);
}

// Clamped bin of t = rho + H given in int64 (any mapped hit).
__device__ __forceinline__ int rho_bin64(long long t, BinMagic m) {
  t = min(max(t, 0LL), (long long)kTwoHm1);
  return bin_of_t((uint32_t)t, m);
}

// floor(a / b) for b > 0 given a float estimate q of a / b with relative error below
// 2^-21: for |q| < 2^20 the estimate is within one of the quotient and an exact remainder
// test fixes it; larger quotients take the 64-bit integer division.
__device__ __forceinline__ long long floor_div_est(long long a, long long b, float q) {
  if (fabsf(q) < 1048576.0f) {
    int q0 = (int)floorf(q);
    const long long r = a - (long long)q0 * b;
    if (r < 0) q0 -= 1;
    else if (r >= b) q0 += 1;
    return q0;
  }
  long long q0 = a / b;
  if ((a % b) != 0 && a < 0) q0 -= 1;
  return q0;
}

// Conformal map of one hit. Returns 0, or HOUGH_F_BAD_HIT for r = 0 or a coordinate beyond 2^24 um.
// The estimate uses x, y as floats (exact for |x|, |y| <= 2^24) and a rounded r^2.
__device__ __forceinline__ int map_hit(int x, int y, long long& u, long long& v) {
  if (x > kCoordMax || x < -kCoordMax || y > kCoordMax || y < -kCoordMax) return HOUGH_F_BAD_HIT;
  const long long r2 = (long long)x * x + (long long)y * y;
  if (r2 == 0) return HOUGH_F_BAD_HIT;
  const float fx = (float)x, fy = (float)y;
  const float s = 8589934592.0f / fmaf(fx, fx, fy * fy);  // 2^33 / r^2
  u = floor_div_est((long long)x * (1LL << 33), r2, fx * s);
  v = floor_div_est((long long)y * (1LL << 33), r2, fy * s);
  return 0;
}

__device__ __forceinline__ bool fits32(long long u, long long v) {
  return u <= kFast32 && u >= -kFast32 && v <= kFast32 && v >= -kFast32;
}

// SplitMix64 finaliser (Steele, Lea and Flood 2014), used for the accumulator fingerprint.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Trig table passed by value to kernels (bin-centre angles, computed on the host).
struct TrigTable {
  int16_t c[kMaxNTheta];
  int16_t s[kMaxNTheta];
};

__device__ __forceinline__ void red_add_shared(uint32_t* p, uint32_t v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Words of shared scratch the per-pass iterative finder takes (extract_iterative_passes's cm)
// for an n_theta x n_rho accumulator in slices of SH rows: an odd-padded stride of slice maxima
// per column, and one word per column.
__host__ __device__ inline int iter_slice_stride(int NR, int SH) { return ((NR + SH - 1) / SH) | 1; }
__host__ __device__ inline int iter_scratch_words(int NT, int NR, int SH) {
  return NT * iter_slice_stride(NR, SH) + NT;
}

// Iterative peak extraction (the paper's finder, Sec. 2), one pass per peak, over an
// accumulator behind `cells` (get(j, k) -> votes of a cell not yet suppressed, 0 once
// suppressed; clear(j, k) suppresses one cell without touching any other cell's value, so that
// other lanes may read and clear other cells meanwhile; with kPairs true, words() is the count of
// 32-bit words and word(w, k) the word of column w (low half) and column mirror_col(w) (high
// half) at row k). The general form of the finder, taken when the sorted form below does not
// apply.
// Cells are ordered by the packed word (votes << 16) | (n_rho - 1 - k): within a column the
// larger word is the cell with more votes and, on equal votes, the smaller k. Across columns
// the key (votes << 16) | (0xffff - j) orders by votes and, on equal votes, the smaller column
// (raster order). cm: iter_scratch_words(NT, NR, SH) words of shared scratch: the best packed
// word of every slice of SH rows (a power of two, at least 32) of every column (stride
// iter_slice_stride), then of every column. s: 1 int of shared scratch.
// The CTA builds the maxima; then warp 0 alone runs the passes, with no block barrier. Each
// pass takes the best column key; if that cell qualifies it is the next peak, its window is
// cleared, and the slices the window touches are re-scanned by groups of lanes, without the
// rows being cleared (they hold no votes any more, and a cell without votes never qualifies,
// since thr >= 1); then groups of lanes rebuild the window's column words. Every pass clears
// the extracted cell, so the loop ends. Records go to dst in extraction order (the first
// max_peaks); returns the true count.
template <class Cells>
__device__ int extract_iterative_passes(Cells& cells, int NT, int NR, int SH, int thr, int rel_num, int rel_den,
                                        int R, int maxp, uint32_t* cm, hough_peak* dst, int* s) {
  const int lane = threadIdx.x & 31, bd = blockDim.x;
  const int NS = (NR + SH - 1) / SH, NSP = iter_slice_stride(NR, SH);
  uint32_t* sl = cm;
  uint32_t* col = cm + NT * NSP;
  auto wrap = [&](int jj) { return jj < 0 ? jj + NT : (jj >= NT ? jj - NT : jj); };
  auto pack = [&](int j, int k) { return ((uint32_t)cells.get(j, k) << 16) | (uint32_t)(NR - 1 - k); };
  // slice maxima (a warp's lanes take consecutive columns of one slice), then column words
  for (int it = threadIdx.x; it < NT * NS; it += bd) {
    const int j = it % NT, q = it / NT;
    const int kb = min(NR, (q + 1) * SH);
    uint32_t b = 0;
#pragma unroll 8
    for (int k = q * SH; k < kb; ++k) b = max(b, pack(j, k));
    sl[j * NSP + q] = b;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < NT; j += bd) {
    uint32_t m = 0;
    for (int q = 0; q < NS; ++q) m = max(m, sl[j * NSP + q]);
    col[j] = m;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    auto best_key = [&]() {
      uint32_t b = 0;
#pragma unroll 8
      for (int j = lane; j < NT; j += 32) b = max(b, (col[j] & 0xffff0000u) | (uint32_t)(0xffff - j));
      return __reduce_max_sync(0xffffffffu, b);
    };
    auto log2_floor = [](int x) { return 31 - __clz(x); };
    const long long amax = (long long)(best_key() >> 16);
    // every per-pass index below is a shift or a multiply: SH is a power of two, lane groups
    // are powers of two, and item / W = (item * mW) >> 21, exact for W <= 129, item < 8192
    const int W = 2 * R + 1, LSH = log2_floor(SH);
    const uint32_t mW = ((1u << 21) + W - 1) / W;
    const int L1 = log2_floor(max(1, 32 / W));  // log2 lanes per window column
    int n = 0;
    for (;;) {
      const uint32_t best = best_key();
      const int v = (int)(best >> 16), j = 0xffff - (int)(best & 0xffffu);
      // thr >= 1, so a qualifying cell has a key and j is a column (ok is warp-uniform)
      if (!(v >= thr && (long long)v * rel_den >= (long long)rel_num * amax)) break;
      const int k = NR - 1 - (int)(col[j] & 0xffffu);
      if (lane == 0 && n < maxp) {
        hough_peak pk;
        pk.theta_bin = (int16_t)j;
        pk.rho_bin = (int16_t)k;
        pk.votes = (int16_t)v;
        pk.flags = 0;
        dst[n] = pk;
      }
      ++n;
      // the window: columns j - R .. j + R and rows r0 .. r1; a column past either end of the
      // theta range is taken from the other end with the rows mirrored
      const int r0 = max(0, k - R), r1 = min(NR - 1, k + R);
      for (int a = lane; a < W; a += 32) {  // clear: a lane per window column
        int jj = j - R + a, c0 = r0, c1 = r1;
        if (jj < 0 || jj >= NT) {
          jj = wrap(jj);
          c0 = NR - 1 - r1;
          c1 = NR - 1 - r0;
        }
        for (int kk = c0; kk <= c1; ++kk) cells.clear(jj, kk);
      }
      // re-scan the touched slices: item (q, a) is window column a, its q-th touched slice,
      // taken by a group of 2^LP lanes, each over SH >> LP rows
      const int span = max((r1 >> LSH) - (r0 >> LSH), ((NR - 1 - r0) >> LSH) - ((NR - 1 - r1) >> LSH)) + 1;
      const int cnt = span * W, LP = max(0, L1 - (span - 1)), RP = SH >> LP;
      for (int base = 0; base < cnt; base += 32 >> LP) {
        const int item = base + (lane >> LP), part = lane & ((1 << LP) - 1);
        uint32_t b = 0;
        int qs = -1, jj = 0;
        if (item < cnt) {
          const int q = (int)(((uint32_t)item * mW) >> 21), a = item - q * W;
          int x0 = r0, x1 = r1;
          jj = j - R + a;
          if (jj < 0 || jj >= NT) {
            jj = wrap(jj);
            x0 = NR - 1 - r1;
            x1 = NR - 1 - r0;
          }
          qs = (x0 >> LSH) + q;
          if (qs <= (x1 >> LSH)) {
            const int ka = (qs << LSH) + part * RP;
#pragma unroll 8
            for (int t = 0; t < RP; ++t) {
              const int kk = ka + t;
              if (kk < NR) {
                const uint32_t w = pack(jj, kk);
                if (kk < x0 || kk > x1) b = max(b, w);
              }
            }
          } else {
            qs = -1;
          }
        }
        for (int o = 1; o < (1 << LP); o <<= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        if (part == 0 && qs >= 0) sl[jj * NSP + qs] = b;
      }
      __syncwarp();
      // the window's column words, 2^L1 lanes per column
      for (int base = 0; base < W; base += 32 >> L1) {
        const int a = base + (lane >> L1), part = lane & ((1 << L1) - 1);
        uint32_t m = 0;
        int jj = 0;
        if (a < W) {
          jj = wrap(j - R + a);
#pragma unroll 4
          for (int q = part; q < NS; q += 1 << L1) m = max(m, sl[jj * NSP + q]);
        }
        for (int o = 1; o < (1 << L1); o <<= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (part == 0 && a < W) col[jj] = m;
      }
      __syncwarp();
    }
    if (lane == 0) s[0] = n;
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_IT_RESOLVE);
  const int n = s[0];
  __syncthreads();
  return n;
}

// Cell (j, k) lies in the suppression window of (ji, ki): columns ji - R .. ji + R and rows
// ki - R .. ki + R, a column past either end of the theta range taken from the other end with
// the rows mirrored (2R < n_theta, so at most one of the three column cases holds).
__device__ __forceinline__ bool in_window(int ji, int ki, int j, int k, int NT, int NR, int R) {
  const int d = j - ji;
  if (d >= -R && d <= R) return abs(k - ki) <= R;
  if (d - NT >= -R || d + NT <= R) return abs(NR - 1 - k - ki) <= R;
  return false;
}

// Sets bits b0 .. b1 of a shared bitmap.
__device__ __forceinline__ void or_bits(uint32_t* bm, int b0, int b1) {
  const int w0 = b0 >> 5, w1 = b1 >> 5;
  for (int w = w0; w <= w1; ++w) {
    uint32_t m = 0xffffffffu;
    if (w == w0) m &= 0xffffffffu << (b0 & 31);
    if (w == w1) m &= 0xffffffffu >> (31 - (b1 & 31));
    atomicOr(&bm[w], m);
  }
}

// Sorts n (a power of two) shared keys into descending order (bitonic); all threads call it.
__device__ __forceinline__ void bitonic_desc(uint32_t* keys, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        const int i = 2 * t - (t & (stride - 1)), l = i + stride;
        const uint32_t a = keys[i], b = keys[l];
        if (((i & size) == 0) == (a < b)) {
          keys[i] = b;
          keys[l] = a;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void store_peak(hough_peak* dst, uint32_t key) {
  hough_peak pk;
  pk.theta_bin = (int16_t)(1023 - (int)((key >> 10) & 1023u));
  pk.rho_bin = (int16_t)(1023 - (int)(key & 1023u));
  pk.votes = (int16_t)(key >> 20);
  pk.flags = 0;
  *dst = pk;
}

// The iterative finder (Sec. 2) in candidate form. Taking the unsuppressed cell with the most
// votes (raster order on ties) and suppressing its window, until the best cell fails the
// threshold, keeps exactly the candidates (cells with votes >= max(thr, ceil(rel_num amax /
// rel_den))) that no kept candidate ranked above them covers, in rank order: every cell ranked
// above the next peak is a peak or lies in a kept window. Candidates are keyed
// (votes << 20) | ((1023 - j) << 10) | (1023 - k), the larger key ranking first. The window
// relation is symmetric, so a candidate's dominators (higher-ranked candidates whose window
// covers it) are the higher-ranked candidates in its own window.
// Stage 1 (all threads): the maximum, then the candidate keys in any order (keys: cap words).
// Returns C, or -1 when the maximum exceeds 4095 votes or C exceeds cap. s[0], s[1] used.
template <class Cells>
__device__ int collect_candidates(Cells& cells, int NT, int NR, int thr, int rel_num, int rel_den, uint32_t* keys,
                                  int cap, int* s, int* tq_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    s[0] = 0;
    s[1] = 0;
  }
  __syncthreads();
  // the maximum (a warp takes rows, its lanes consecutive columns, or with Cells::kPairs
  // consecutive words of two columns each: w and NT - 1 - w)
  {
    int m = 0;
    if constexpr (Cells::kPairs) {  // four words a lane, both halves at once (16-bit SIMD maxima)
      const int W4 = (cells.words() + 3) >> 2, n4 = NR * W4;
      unsigned mm = 0u;
      for (int it = threadIdx.x; it < n4; it += blockDim.x) {
        const int k = it / W4;
        const uint4 x = cells.words4((it - k * W4) << 2, k);
        mm = __vmaxu2(mm, __vmaxu2(__vmaxu2(x.x, x.y), __vmaxu2(x.z, x.w)));
      }
      m = (int)max(mm & 0xffffu, mm >> 16);
    } else {
      for (int k = warp; k < NR; k += nwarps)
        for (int j = lane; j < NT; j += 32) m = max(m, cells.get(j, k));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0 && m) atomicMax(&s[0], m);
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_IT_MAX);
  const int amax = s[0];
  if (amax > 4095) return -1;  // uniform: every thread read the same value
  const long long need = ((long long)rel_num * amax + rel_den - 1) / rel_den;
  const int tq = (int)max((long long)thr, need);
  *tq_out = tq;
  auto key_of = [&](int v, int j, int k) {
    return ((uint32_t)v << 20) | ((uint32_t)(1023 - j) << 10) | (uint32_t)(1023 - k);
  };
  if constexpr (Cells::kPairs) {
    // four words (eight cells) a lane; a warp's candidates get consecutive positions (one
    // atomic a warp), each lane's in word order, low half first. (Two passes without atomics,
    // a warp counting its run of rows before writing, measured slower: 22.1 k against 12.7 k.)
    const int Wd = cells.words(), W4 = (Wd + 3) >> 2, n4 = NR * W4;
    const unsigned tq2 = (unsigned)tq * 0x10001u;
    for (int it0 = threadIdx.x - lane; it0 < n4; it0 += blockDim.x) {  // slots of a warp: uniform
      const int it = it0 + lane, k = it / W4, w4 = (it - k * W4) << 2;
      unsigned ge[4] = {0u, 0u, 0u, 0u};
      uint4 x = make_uint4(0u, 0u, 0u, 0u);
      if (it < n4) {
        x = cells.words4(w4, k);
        ge[0] = __vcmpgeu2(x.x, tq2);
        ge[1] = w4 + 1 < Wd ? __vcmpgeu2(x.y, tq2) : 0u;  // words past the tile's own: none
        ge[2] = w4 + 2 < Wd ? __vcmpgeu2(x.z, tq2) : 0u;
        ge[3] = w4 + 3 < Wd ? __vcmpgeu2(x.w, tq2) : 0u;
      }
      int n = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) n += (ge[q] & 1u) + (ge[q] >> 31);
      int pre = n;  // inclusive scan over the warp's lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += y;
      }
      const int total = __shfl_sync(0xffffffffu, pre, 31);
      int base = 0;
      if (lane == 31 && total) base = atomicAdd(&s[1], total);
      base = __shfl_sync(0xffffffffu, base, 31) + pre - n;
      if (n) {
        const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (ge[q] & 1u) {
            if (base < cap) keys[base] = key_of((int)(xs[q] & 0xffffu), w4 + q, k);
            ++base;
          }
          if (ge[q] >> 31) {
            if (base < cap) keys[base] = key_of((int)(xs[q] >> 16), cells.mirror_col(w4 + q), k);
            ++base;
          }
        }
      }
    }
  } else {
    for (int k = warp; k < NR; k += nwarps) {
      for (int j0 = 0; j0 < NT; j0 += 32) {
        const int j = j0 + lane;
        const int v = j < NT ? cells.get(j, k) : 0;
        const bool c = v >= tq;
        const uint32_t bal = __ballot_sync(0xffffffffu, c);
        if (bal) {
          int base = 0;
          if (lane == 0) base = atomicAdd(&s[1], __popc(bal));
          base = __shfl_sync(0xffffffffu, base, 0);
          const int pos = base + __popc(bal & ((1u << lane) - 1u));
          if (c && pos < cap) keys[pos] = key_of(v, j, k);
        }
      }
    }
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_IT_COLLECT);
  const int C = s[1];
  return C > cap ? -1 : C;
}

// Position of this lane's entry in a shared list counted by *cnt (-1 when p is false), one
// atomic a warp; every lane of the warp calls it.
__device__ __forceinline__ int warp_append(int* cnt, bool p) {
  const int lane = threadIdx.x & 31;
  const unsigned b = __ballot_sync(0xffffffffu, p);
  int base = 0;
  if (lane == 0 && b) base = atomicAdd(cnt, __popc(b));
  base = __shfl_sync(0xffffffffu, base, 0);
  return p ? base + __popc(b & ((1u << lane) - 1u)) : -1;
}

// Stage 2, in parallel rounds (all threads): st holds 2 bits per cell (cell (j, k) is pair
// j NR + k): 0 not a candidate or dropped, 1 undecided, 3 kept, each changed by one atomic, so
// readers see a whole state. Each round, an undecided candidate with no undecided higher-ranked
// cell in its window is kept, and the keeping thread at once drops every other candidate of
// that window (they all rank below it and none is kept: a kept one would have dropped it); one
// with a kept cell in its window (read before that cell's drops reached it) drops itself.
// Decisions are final, and each round keeps at least the highest-ranked undecided candidate;
// states read while others change are either the old or the final one, which only speeds this
// up. Pushing the drops halves the rounds against drops found by the dropped candidates' owners
// in the next round (8.1 -> 4.2 on the batched events).
// The kept keys are then gathered into st (as many as its st_words hold) and ordered by rank (by
// counting the kept keys above each, up to 1,024 of them; else bitonic). st_words: at least
// ceil(NT NR / 16) rounded up to a multiple of 32. act: two lists of act_cap 16-bit entries.
// Returns the count, or -1 (written nothing) past 64 rounds or st_words, or with more than 64
// candidates a thread. s[2] .. s[5] used.
template <class Cells>
__device__ int resolve_rounds(Cells& cells, int NT, int NR, int R, int tq, int maxp, const uint32_t* keys, int C,
                              uint32_t* st, int st_words, uint16_t* act, int act_cap, hough_peak* dst, int* s) {
  const int lane = threadIdx.x & 31, bd = blockDim.x;
  if (C > 64 * bd || C > 65536) return -1;
  // State word w lives at w ^ (w >> 5 & 31): the words of the same rows of neighbouring columns,
  // which the lanes of a warp read together, then fall in different banks (unswizzled, a column
  // of 256 rows is 16 words, and 32 columns would share 2 banks).
  const int nst = ((((NT * NR + 15) >> 4) + 31) & ~31);
  if (nst > st_words) return -1;
  auto swz = [](int w) { return w ^ ((w >> 5) & 31); };
  for (int i = threadIdx.x; i < nst; i += bd) st[i] = 0u;
  if (threadIdx.x < 4) s[2 + threadIdx.x] = 0;
  __syncthreads();
  auto cell_of = [&](uint32_t key) { return (1023 - (int)((key >> 10) & 1023u)) * NR + 1023 - (int)(key & 1023u); };
  // drops (1 -> 0) the candidates of column j + a of the window of the kept cell (j, k), except
  // the cell itself; a cleared low bit leaves a 0 as it was and cannot meet a kept cell
  auto push_column = [&](int j, int k, int a) {
    int jj = j + a, r0 = max(0, k - R), r1 = min(NR - 1, k + R);
    if (jj < 0 || jj >= NT) {  // across the theta wrap: the other end, rho mirrored
      jj = jj < 0 ? jj + NT : jj - NT;
      const int t0 = NR - 1 - r1;
      r1 = NR - 1 - r0;
      r0 = t0;
    }
    const int b0 = (jj * NR + r0) << 1, b1 = (jj * NR + r1) << 1, bc = a == 0 ? (j * NR + k) << 1 : -1;
    for (int w = b0 >> 5; w <= (b1 >> 5); ++w) {
      uint32_t m = 0x55555555u;
      if (w == (b0 >> 5)) m &= 0xffffffffu << (b0 & 31);
      if (w == (b1 >> 5)) m &= 0xffffffffu >> (31 - (b1 & 31));
      if (w == (bc >> 5)) m &= ~(1u << (bc & 31));
      atomicAnd(&st[swz(w)], ~m);
    }
  };
  for (int i = threadIdx.x; i < C; i += bd) {  // every candidate undecided
    const int c = cell_of(keys[i]);
    atomicOr(&st[swz(c >> 4)], 1u << ((c & 15) << 1));
  }
  __syncthreads();
  // The decision on undecided candidate (j, k) from the states of its window: 1 (drop) for a kept
  // cell in it, 2 (keep) for no undecided higher-ranked cell in it, else 0. The scan stops at the
  // first higher-ranked undecided cell: a kept cell it then misses drops the candidate by its push.
  auto decide = [&](int j, int k, uint32_t key) -> int {
    bool drop = false, all = true;
    const int k0 = max(0, k - R), k1 = min(NR - 1, k + R);
    for (int a = -R; a <= R && !drop && all; ++a) {
      int jj = j + a, r0 = k0, r1 = k1;
      if (jj < 0 || jj >= NT) {
        jj = jj < 0 ? jj + NT : jj - NT;
        r0 = NR - 1 - k1;
        r1 = NR - 1 - k0;
      }
      // the states of rows r0 .. r1 of column jj, 16 cells at a time
      const int b0 = (jj * NR + r0) << 1, nb = (r1 - r0 + 1) << 1;
      int p = 0, e_col = 0;  // sorted lists: a walk down column jj's list
      if constexpr (sorted_cells<Cells>::value) {
        p = cells.lower(jj, r0);
        e_col = cells.end(jj);
      }
      for (int off = 0; off < nb && !drop && all; off += 32) {
        const int bb = b0 + off, w = bb >> 5, sh = bb & 31, len = min(32, nb - off);
        uint32_t f = st[swz(w)] >> sh;
        if (sh && sh + len > 32) f |= st[swz(w + 1)] << (32 - sh);
        if (len < 32) f &= (1u << len) - 1u;
        if ((f & (f >> 1)) & 0x55555555u) {  // a kept cell
          drop = true;
          break;
        }
        uint32_t m = f & ~(f >> 1) & 0x55555555u;  // undecided cells
        while (m && all) {
          const int kr = r0 + ((off + __ffs(m) - 1) >> 1);
          uint32_t kd;
          if constexpr (sorted_cells<Cells>::value) {  // an undecided cell is in its column's list
            while (p < e_col && 1023 - (int)(cells.key(p) & 1023u) < kr) ++p;
            kd = p < e_col ? cells.key(p) : 0u;
          } else {
            kd = ((uint32_t)cells.get(jj, kr) << 20) | ((uint32_t)(1023 - jj) << 10) | (uint32_t)(1023 - kr);
          }
          if (kd > key) all = false;  // an undecided cell ranked above (the cell itself is equal)
          m &= m - 1u;
        }
      }
    }
    return drop ? 1 : all ? 2 : 0;
  };
  // Candidates kept in a slot of a warp (jk = j << 16 | k, else -1): the warp pushes their drops.
  auto push_slot = [&](int jk) {
    for (unsigned kb = __ballot_sync(0xffffffffu, jk >= 0); kb; kb &= kb - 1u) {
      const int x = __shfl_sync(0xffffffffu, jk, __ffs(kb) - 1);
      for (int a = lane - R; a <= R; a += 32) push_column(x >> 16, x & 0xffff, a);
    }
  };
  // The drops of the kept ones among candidates L[0 .. n) (candidates 0 .. n without a list),
  // pushed after the pass that kept them: a thread a (candidate, window column) pair. (Round 0's
  // survivors: 14 k cycles an event against 17 k pushed in the pass by their warps; in the later
  // rounds pushes in the pass are faster, since they drop candidates that the same round visits.)
  auto push_kept = [&](const uint16_t* L, int n) {
    const int W = 2 * R + 1;
    for (int it = threadIdx.x; it < n * W; it += bd) {
      const int e = it / W, a = it - e * W - R;
      const uint32_t key = keys[L ? (int)L[e] : e];
      const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u), c = j * NR + k;
      if (((st[swz(c >> 4)] >> ((c & 15) << 1)) & 3u) == 3u) push_column(j, k, a);
    }
  };
  // Round 0 in three passes, since most candidates are not local maxima and a warp's scans last
  // as long as its slowest lane's. (1) A candidate with a higher-ranked cell among its eight
  // neighbours (votes alone decide: cells below the threshold rank below every candidate) stays
  // undecided; the others are listed. (2) The listed ones that rank above their whole window are
  // kept, and push their drops. (3) The candidates still undecided are listed for round 1. Lists: act (the
  // survivors), then act + act_cap (round 1's); s[4] counts the survivors, s[2] the undecided.
  {
    for (int t0 = threadIdx.x - lane; t0 < C; t0 += bd) {  // slots of a warp: uniform
      const int t = t0 + lane;
      bool sv = t < C;
      if (sv && R > 0 && sorted_cells<Cells>::value) {  // three column walks
        const uint32_t key = keys[t];
        const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u);
        for (int da = -1; da <= 1; ++da) {
          int jj = j + da, r0 = max(0, k - 1), r1 = min(NR - 1, k + 1);
          if (jj < 0 || jj >= NT) {  // across the theta wrap: the other end, rho mirrored
            jj = jj < 0 ? jj + NT : jj - NT;
            const int t0 = NR - 1 - r1;
            r1 = NR - 1 - r0;
            r0 = t0;
          }
          if constexpr (sorted_cells<Cells>::value) {
            const int e_col = cells.end(jj);
            for (int p = cells.lower(jj, r0); p < e_col && 1023 - (int)(cells.key(p) & 1023u) <= r1; ++p)
              sv = sv && cells.key(p) <= key;
          }
        }
      } else if (sv && R > 0) {
        const uint32_t key = keys[t];
        const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          int jj = j + q / 3 - 1, kk = k + q % 3 - 1;
          if (q == 4 || kk < 0 || kk >= NR) continue;
          if (jj < 0 || jj >= NT) {  // across the theta wrap: the other end, rho mirrored
            jj = jj < 0 ? jj + NT : jj - NT;
            kk = NR - 1 - kk;
          }
          const uint32_t kd = ((uint32_t)cells.get(jj, kk) << 20) | ((uint32_t)(1023 - jj) << 10) |
                              (uint32_t)(1023 - kk);
          sv = sv && kd <= key;
        }
      }
      const int pos = warp_append(&s[4], sv);
      if (sv && pos < act_cap) act[pos] = (uint16_t)t;
    }
    __syncthreads();
    const int ns = s[4], n = ns <= act_cap ? ns : C;  // past the list's room: every candidate
    for (int t0 = threadIdx.x - lane; t0 < n; t0 += bd) {
      const int t = t0 + lane;
      const int i = t < n ? (ns <= act_cap ? (int)act[t] : t) : 0;
      const uint32_t key = keys[i];
      const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u);
      const int c = j * NR + k;
      // at the start of round 0 every candidate is undecided and none is kept, so the rules keep
      // exactly the candidates that rank above every other cell of their window: a test on the
      // votes alone, with independent reads (the state scan's reads depend on one another)
      if (t < n) {
        bool top = true;
        const int k0 = max(0, k - R), k1 = min(NR - 1, k + R);
        for (int a = -R; a <= R; ++a) {
          int jj = j + a, r0 = k0, r1 = k1;
          if (jj < 0 || jj >= NT) {  // across the theta wrap: the other end, rho mirrored
            jj = jj < 0 ? jj + NT : jj - NT;
            r0 = NR - 1 - k1;
            r1 = NR - 1 - k0;
          }
          if constexpr (sorted_cells<Cells>::value) {
            const int e_col = cells.end(jj);
            for (int p = cells.lower(jj, r0); p < e_col && 1023 - (int)(cells.key(p) & 1023u) <= r1; ++p)
              top &= cells.key(p) <= key;
          } else {
#pragma unroll 4
            for (int kr = r0; kr <= r1; ++kr)
              top &= (((uint32_t)cells.get(jj, kr) << 20) | ((uint32_t)(1023 - jj) << 10) | (uint32_t)(1023 - kr)) <= key;
          }
        }
        if (top) atomicOr(&st[swz(c >> 4)], 2u << ((c & 15) << 1));  // 1 -> 3
      }
    }
    __syncthreads();
    push_kept(ns <= act_cap ? act : nullptr, n);
    __syncthreads();
    for (int i0 = threadIdx.x - lane; i0 < C; i0 += bd) {  // slots of a warp: uniform
      const int i = i0 + lane, c = cell_of(keys[i < C ? i : 0]);
      const bool u = i < C && ((st[swz(c >> 4)] >> ((c & 15) << 1)) & 3u) == 1u;
      const int pos = warp_append(&s[2], u);
      if (u && pos < act_cap) act[act_cap + pos] = (uint16_t)i;
    }
    __syncthreads();
  }
  // Rounds 1, 2, ...: once at most act_cap candidates are undecided, a round visits only those:
  // the round before listed them (two lists of act_cap 16-bit indices, alternating). A candidate
  // takes a thread; at most half as many candidates as threads, a group of lanes, a window column a
  // lane (radius up to 7); at most four a warp, a whole warp with its lanes on the window's cells.
  bool listed = s[2] <= act_cap;  // uniform
  if (s[2] > 0)
  for (int round = 1;; ++round) {
    if (round == 64) return -1;  // uniform
    const int r3 = round % 3;
    const uint16_t* cur = act + (round & 1) * act_cap;
    uint16_t* nxt = act + ((round + 1) & 1) * act_cap;
    const int n_cur = listed ? s[2 + (round + 2) % 3] : C;  // the previous round's undecided
    if (listed && n_cur <= 4 * (bd >> 5) && R <= 7) {
      // Few left: a warp per undecided candidate, its lanes on the cells of the window, so that a
      // round costs one state read and at most one vote read per lane instead of one thread's walk
      // over the window's columns.
      const int W = 2 * R + 1, nc = W * W;
      const uint32_t mW = ((1u << 21) + W - 1) / W;  // q / W = (q mW) >> 21, exact for q < 2^10
      for (int t = threadIdx.x >> 5; t < n_cur; t += bd >> 5) {
        const int i = (int)cur[t];
        const uint32_t key = keys[i];
        const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u);
        const int c = j * NR + k;
        const uint32_t sw = __shfl_sync(0xffffffffu, st[swz(c >> 4)], 0);  // one reading for the warp
        if (((sw >> ((c & 15) << 1)) & 3u) != 1u) continue;  // dropped since it was listed
        bool kept_seen = false, above = false;
        for (int q = lane; q < nc; q += 32) {
          const int qa = (int)(((uint32_t)q * mW) >> 21);
          int jj = j + qa - R, kk = k + (q - qa * W) - R;
          if (kk < 0 || kk >= NR || (jj == j && kk == k)) continue;
          if (jj < 0 || jj >= NT) {  // across the theta wrap: the other end, rho mirrored
            jj = jj < 0 ? jj + NT : jj - NT;
            kk = NR - 1 - kk;
          }
          const int cc = jj * NR + kk;
          const uint32_t sv = (st[swz(cc >> 4)] >> ((cc & 15) << 1)) & 3u;
          if (sv == 3u) {
            kept_seen = true;
          } else if (sv == 1u) {
            const uint32_t kd = ((uint32_t)cells.get(jj, kk) << 20) | ((uint32_t)(1023 - jj) << 10) |
                                (uint32_t)(1023 - kk);
            above = above || kd > key;
          }
        }
        kept_seen = __any_sync(0xffffffffu, kept_seen);
        above = __any_sync(0xffffffffu, above);
        if (kept_seen) {
          if (lane == 0) atomicAnd(&st[swz(c >> 4)], ~(1u << ((c & 15) << 1)));  // 1 -> 0
        } else if (!above) {
          if (lane == 0) atomicOr(&st[swz(c >> 4)], 2u << ((c & 15) << 1));  // 1 -> 3
          if (lane < W) push_column(j, k, lane - R);
        } else if (lane == 0) {
          const int pos = atomicAdd(&s[2 + r3], 1);
          if (pos < act_cap) nxt[pos] = (uint16_t)i;
        }
      }
    } else if (listed && n_cur <= (bd >> 1) && R <= 7) {
      // A group of G lanes (8 up to radius 3, else 16) per candidate, a window column a lane: the
      // columns' scans run side by side instead of one after another in one thread. (With more
      // candidates than half the threads, a thread each measured faster: batched round 1 19.1 k
      // against 23.6 k cycles.)
      const int W = 2 * R + 1, G = W <= 8 ? 8 : 16, gpw = 32 / G;  // groups a warp
      const int grp = lane / G, sub = lane % G, a = sub - R;
      const unsigned gmask = ((1u << G) - 1u) << (grp * G);
      for (int t0 = (threadIdx.x >> 5) * gpw; t0 < n_cur; t0 += (bd >> 5) * gpw) {  // uniform a warp
        const int t = t0 + grp;
        const int i = t < n_cur ? (listed ? (int)cur[t] : t) : 0;
        const uint32_t key = keys[i];
        const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u), c = j * NR + k;
        const bool live = t < n_cur && ((st[swz(c >> 4)] >> ((c & 15) << 1)) & 3u) == 1u;  // uniform a group
        bool kept_seen = false, above = false;
        if (live && sub < W) {
          int jj = j + a, r0 = max(0, k - R), r1 = min(NR - 1, k + R);
          if (jj < 0 || jj >= NT) {  // across the theta wrap: the other end, rho mirrored
            jj = jj < 0 ? jj + NT : jj - NT;
            const int t1 = NR - 1 - r1;
            r1 = NR - 1 - r0;
            r0 = t1;
          }
          // the states of rows r0 .. r1 (at most 15 cells: one or two words)
          const int b0 = (jj * NR + r0) << 1, nb = (r1 - r0 + 1) << 1, w = b0 >> 5, sh = b0 & 31;
          uint32_t f = st[swz(w)] >> sh;
          if (sh && sh + nb > 32) f |= st[swz(w + 1)] << (32 - sh);
          if (nb < 32) f &= (1u << nb) - 1u;
          kept_seen = ((f & (f >> 1)) & 0x55555555u) != 0u;
          uint32_t m = f & ~(f >> 1) & 0x55555555u;  // undecided cells
          int p = 0, e_col = 0;
          if constexpr (sorted_cells<Cells>::value) {
            p = cells.lower(jj, r0);
            e_col = cells.end(jj);
          }
          while (m && !above) {
            const int kr = r0 + ((__ffs(m) - 1) >> 1);
            uint32_t kd;
            if constexpr (sorted_cells<Cells>::value) {
              while (p < e_col && 1023 - (int)(cells.key(p) & 1023u) < kr) ++p;
              kd = p < e_col ? cells.key(p) : 0u;
            } else {
              kd = ((uint32_t)cells.get(jj, kr) << 20) | ((uint32_t)(1023 - jj) << 10) | (uint32_t)(1023 - kr);
            }
            above = kd > key;  // an undecided cell ranked above (the cell itself is equal)
            m &= m - 1u;
          }
        }
        const bool gk = (__ballot_sync(0xffffffffu, kept_seen) & gmask) != 0u;
        const bool ga = (__ballot_sync(0xffffffffu, above) & gmask) != 0u;
        if (live && sub == 0 && gk) atomicAnd(&st[swz(c >> 4)], ~(1u << ((c & 15) << 1)));  // 1 -> 0
        if (live && sub == 0 && !gk && !ga) atomicOr(&st[swz(c >> 4)], 2u << ((c & 15) << 1));  // 1 -> 3
        if (live && !gk && !ga && sub < W) push_column(j, k, a);  // the kept one's drops
        // the undecided are counted, and listed for the next round while the list has room
        const bool und = live && sub == 0 && !gk && ga;
        const int pos = warp_append(&s[2 + r3], und);
        if (und && pos < act_cap) nxt[pos] = (uint16_t)i;
      }
    } else
    for (int t0 = threadIdx.x - lane; t0 < n_cur; t0 += bd) {  // slots of a warp: uniform
      const int t = t0 + lane;
      const int i = t < n_cur ? (listed ? (int)cur[t] : t) : 0;
      const uint32_t key = keys[i];
      const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u);
      const int c = j * NR + k;
      bool und = false;
      int jk = -1;
      if (t < n_cur && ((st[swz(c >> 4)] >> ((c & 15) << 1)) & 3u) == 1u) {
        const int d = decide(j, k, key);
        if (d == 1) {
          atomicAnd(&st[swz(c >> 4)], ~(1u << ((c & 15) << 1)));  // 1 -> 0
        } else if (d == 2) {
          atomicOr(&st[swz(c >> 4)], 2u << ((c & 15) << 1));  // 1 -> 3
          jk = (j << 16) | k;
        } else {
          und = true;
        }
      }
      // the undecided are counted, and listed for the next round while the list has room
      const int pos = warp_append(&s[2 + r3], und);
      if (und && pos < act_cap) nxt[pos] = (uint16_t)i;
      push_slot(jk);
    }
    // undecided count: three rotating counters, so that one barrier a round suffices
    if (threadIdx.x == 0) s[2 + (r3 + 1) % 3] = 0;
    __syncthreads();
    const int und = s[2 + r3];
    if (und == 0) break;
    listed = und <= act_cap;
  }
  HOUGH_PHASE(HOUGH_PHASE_IT_RESOLVE);
  // the kept keys, gathered into st once every state has been read
  unsigned long long flags = 0;
  {
    int t = 0;
    for (int i = threadIdx.x; i < C; i += bd, ++t) {
      const int c = cell_of(keys[i]);
      if (((st[swz(c >> 4)] >> ((c & 15) << 1)) & 3u) == 3u) flags |= 1ull << t;
    }
  }
  {
    const int kept = __reduce_add_sync(0xffffffffu, __popcll(flags));
    if (lane == 0 && kept) atomicAdd(&s[5], kept);
  }
  __syncthreads();
  const int nk = s[5];
  int N = 32;
  while (N < nk) N <<= 1;
  if (N > st_words) return -1;  // uniform; st is not needed by the other forms
  if (threadIdx.x == 0) s[4] = 0;
  __syncthreads();
  {
    int t = 0;
    for (int i0 = threadIdx.x - lane; i0 < C; i0 += bd, ++t) {  // slots of a warp: uniform
      const int i = i0 + lane;
      const bool kp = i < C && ((flags >> t) & 1ull);
      const int pos = warp_append(&s[4], kp);
      if (kp) st[pos] = keys[i];
    }
  }
  __syncthreads();
  if (nk <= 1024) {  // a kept key's rank is the count of kept keys above it (keys are distinct)
    for (int i = threadIdx.x; i < nk; i += bd) {
      const uint32_t key = st[i];
      int r = 0;
      for (int m = 0; m < nk; ++m) r += st[m] > key;
      if (r < maxp) store_peak(dst + r, key);
    }
  } else {
    for (int i = nk + threadIdx.x; i < N; i += bd) st[i] = 0u;
    __syncthreads();
    bitonic_desc(st, N);
    for (int i = threadIdx.x; i < min(nk, maxp); i += bd) store_peak(dst + i, st[i]);
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_IT_ORDER);
  return nk;
}

// Stage 2, as one walk (sup: a shared bitmap of NT NR bits, cell (j, k) bit j NR + k): the CTA
// sorts the keys (cap words, past C free), then warp 0 walks them 32 at a time: lanes drop
// candidates covered by earlier chunks' windows, then the lowest remaining lane is kept and the
// lanes its window covers drop out, until none remain; the kept windows go into the bitmap for
// the next chunks. Returns the count. s[0] used.
__device__ inline int resolve_walk(int NT, int NR, int R, int maxp, uint32_t* keys, int C, uint32_t* sup,
                                   hough_peak* dst, int* s) {
  const int lane = threadIdx.x & 31, bd = blockDim.x;
  int N = 32;
  while (N < C) N <<= 1;
  for (int i = C + threadIdx.x; i < N; i += bd) keys[i] = 0u;
  for (int i = threadIdx.x; i < (NT * NR + 31) >> 5; i += bd) sup[i] = 0u;
  __syncthreads();
  bitonic_desc(keys, N);
  if (threadIdx.x < 32) {
    const int W = 2 * R + 1;
    const uint32_t mW = ((1u << 21) + W - 1) / W;  // item / W = (item * mW) >> 21, exact here
    int n = 0;
    for (int base = 0; base < C; base += 32) {
      const int idx = base + lane;
      const uint32_t key = keys[idx];  // idx < N: zero past C
      const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u);
      const int cb = j * NR + k;
      const bool live = idx < C && !((sup[cb >> 5] >> (cb & 31)) & 1u);
      uint32_t L = __ballot_sync(0xffffffffu, live), A = 0;
      const int jk = (j << 16) | k;
      while (L) {
        const int i = __ffs(L) - 1;
        const int ji = __shfl_sync(0xffffffffu, jk, i);
        A |= 1u << i;
        L &= ~__ballot_sync(0xffffffffu, in_window(ji >> 16, ji & 0xffff, j, k, NT, NR, R));
      }
      const int na = __popc(A);
      if (na) {
        const bool kept = (A >> lane) & 1u;
        const int r = __popc(A & ((1u << lane) - 1u));
        if (kept && n + r < maxp) store_peak(dst + n + r, key);
        // this chunk's keys are in registers now: its words hold the kept cells
        __syncwarp();
        if (kept) keys[base + r] = (uint32_t)jk;
        __syncwarp();
        for (int it = lane; it < na * W; it += 32) {
          const int p = (int)(((uint32_t)it * mW) >> 21), a = it - p * W;
          const uint32_t c = keys[base + p];
          const int jp = (int)(c >> 16), kp = (int)(c & 0xffffu);
          int jj = jp - R + a, x0 = max(0, kp - R), x1 = min(NR - 1, kp + R);
          if (jj < 0 || jj >= NT) {
            jj = jj < 0 ? jj + NT : jj - NT;
            const int t0 = NR - 1 - x1;
            x1 = NR - 1 - x0;
            x0 = t0;
          }
          or_bits(sup, jj * NR + x0, jj * NR + x1);
        }
        __syncwarp();
        n += na;
      }
    }
    if (lane == 0) s[0] = n;
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_IT_RESOLVE);
  const int n = s[0];
  __syncthreads();
  return n;
}

// The iterative finder: the candidate form where it applies (cap > 0): resolved in rounds when
// st_words > 0, else (or when the rounds give up) by the walk; otherwise one pass per peak.
// scratch (shared): max(iter_scratch_words(NT, NR, SH), cap + max(ceil(NT NR / 32), st_words))
// words when sup is null: the candidate keys, then the walk's bitmap, or the rounds' states
// (st_words >= ceil(NT NR / 16) rounded up to 32 words). With sup given (a shared bitmap of NT NR
// bits, left set) the walk uses it, and scratch needs max(iter_scratch_words, cap + st_words).
template <class Cells>
__device__ int extract_iterative(Cells& cells, int NT, int NR, int SH, int thr, int rel_num, int rel_den, int R,
                                 int maxp, uint32_t* scratch, int cap, uint32_t* sup, int st_words,
                                 hough_peak* dst, int* s, uint16_t* act = nullptr, int act_cap = 0) {
  if (cap > 0) {
    int tq = 0;
    const int C = collect_candidates(cells, NT, NR, thr, rel_num, rel_den, scratch, cap, s, &tq);
    if (C >= 0) {
      if (st_words > 0) {
        const int n =
            resolve_rounds(cells, NT, NR, R, tq, maxp, scratch, C, scratch + cap, st_words, act, act_cap, dst, s);
        if (n >= 0) return n;
      }
      return resolve_walk(NT, NR, R, maxp, scratch, C, sup ? sup : scratch + cap, dst, s);
    }
  }
  return extract_iterative_passes(cells, NT, NR, SH, thr, rel_num, rel_den, R, maxp, scratch, dst, s);
}

__device__ __forceinline__ void flag_status(int* status, int f) {
  if (f) atomicOr(status, f);
}

}  // namespace hgpu
