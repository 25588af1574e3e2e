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

#include "hough.h"

namespace hgpu {

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

// Iterative peak extraction (the paper's finder, Sec. 2) over an accumulator behind `cells`
// (get(j, k) -> votes of a cell not yet suppressed, 0 once suppressed; clear(j, k) suppresses).
// cm: n_theta words of shared scratch holding each column's best cell packed as
// (votes << 16) | (n_rho - 1 - k): within a column the larger word is the cell with more votes
// and, on equal votes, the smaller k. s: 2 ints of shared scratch. Each pass: warp 0 takes the
// column with the most votes (equal votes: the smaller column, i.e. raster order); if that cell
// qualifies it is the next peak, the whole CTA clears its window and warps re-scan the 2R + 1
// columns it touches, one column per warp. Every pass clears the extracted cell, so the loop
// ends. Records go to dst in extraction order (the first max_peaks); returns the true count.
template <class Cells>
__device__ int extract_iterative(Cells& cells, int NT, int NR, int thr, int rel_num, int rel_den, int R, int maxp,
                                 uint32_t* cm, hough_peak* dst, int* s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  auto column_best = [&](int j) {
    uint32_t b = 0;
    for (int k = lane; k < NR; k += 32) {
      const uint32_t v = (uint32_t)cells.get(j, k);
      b = max(b, (v << 16) | (uint32_t)(NR - 1 - k));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    return b;
  };
  for (int j = warp; j < NT; j += nwarps) {
    const uint32_t b = column_best(j);
    if (lane == 0) cm[j] = b;
  }
  __syncthreads();
  long long amax = 0;
  {
    uint32_t m = 0;
    for (int j = lane; j < NT; j += 32) m = max(m, cm[j] >> 16);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    amax = m;  // every warp computes the same maximum
  }
  const int W = 2 * R + 1;
  int n = 0;
  for (;;) {
    if (warp == 0) {
      uint32_t bv = 0;
      int bj = NT;
      for (int j = lane; j < NT; j += 32) {
        const uint32_t c = cm[j];
        if ((c >> 16) > (bv >> 16) || bj == NT) {
          bv = c;
          bj = j;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint32_t ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if ((ov >> 16) > (bv >> 16) || ((ov >> 16) == (bv >> 16) && oj < bj)) {
          bv = ov;
          bj = oj;
        }
      }
      const int v = (int)(bv >> 16);
      const bool ok = bj < NT && v >= thr && (long long)v * rel_den >= (long long)rel_num * amax;
      if (lane == 0) {
        s[0] = ok ? bj : -1;
        s[1] = ok ? NR - 1 - (int)(bv & 0xffffu) : 0;
        if (ok && n < maxp) {
          hough_peak pk;
          pk.theta_bin = (int16_t)bj;
          pk.rho_bin = (int16_t)(NR - 1 - (int)(bv & 0xffffu));
          pk.votes = (int16_t)v;
          pk.flags = 0;
          dst[n] = pk;
        }
      }
    }
    __syncthreads();
    const int j = s[0], k = s[1];
    if (j < 0) break;
    ++n;
    for (int i = threadIdx.x; i < W * W; i += blockDim.x) {
      const int dj = i / W - R, dk = i % W - R;
      int jj = j + dj, kk = k + dk;
      if (kk < 0 || kk >= NR) continue;
      if (jj < 0 || jj >= NT) {
        jj = jj < 0 ? jj + NT : jj - NT;
        kk = NR - 1 - kk;
      }
      cells.clear(jj, kk);
    }
    __syncthreads();
    for (int dj = warp - R; dj <= R; dj += nwarps) {
      int jj = j + dj;
      jj = jj < 0 ? jj + NT : (jj >= NT ? jj - NT : jj);
      const uint32_t b = column_best(jj);
      if (lane == 0) cm[jj] = b;
    }
    __syncthreads();
  }
  return n;
}

__device__ __forceinline__ void flag_status(int* status, int f) {
  if (f) atomicOr(status, f);
}

}  // namespace hgpu
