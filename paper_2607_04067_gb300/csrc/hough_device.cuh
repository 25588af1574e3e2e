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

__device__ __forceinline__ void flag_status(int* status, int f) {
  if (f) atomicOr(status, f);
}

}  // namespace hgpu
