// Fused conformal-Hough kernel: map -> rho -> vote -> peaks -> select, one CTA per
// (event, theta tile) work item, the accumulator never leaving shared memory.
//
// Thread organisation (Sec. 3's event / angle-column / hit parallelism, redone for sm_103a):
//   - a work item is one event, or one theta tile of an event when its accumulator
//     does not fit one CTA's shared memory;
//   - every lane of a "worker" warp owns theta columns of the tile for the whole vote.
//     Lane l's cells live in shared-memory bank l only: word ((g * rows + row) * 32 + l),
//     rows = N_rho / 2 packed int16 pairs (or N_rho int32 cells), so the column-parallel
//     vote is free of bank conflicts whatever rho bins the hits hit; warps sharing
//     columns split the hits and add with red.shared. In mirror mode a lane owns
//     column j and its mirror N_theta-1-j (th -> pi - th: c -> -c, s -> s), so one pair
//     of products gives both rho values;
//   - for tiled events one extra warp votes the two neighbour columns of the tile
//     (halo), so the 3x3 peak test is exact on tile edges; the last tile CTA of an
//     event (ticket counter) merges the tiles' peak lists in tile order and selects.
#include <climits>
#include <map>
#include <mutex>
#include <utility>

#include "hough_internal.h"

namespace hgpu {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSelCap = 12;  // peak columns a lane tries alone before its hit goes to a whole warp

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

__device__ __forceinline__ uint32_t swap16(uint32_t x) { return __funnelshift_l(x, x, 16); }

template <bool A32>
__device__ __forceinline__ int acc_index(int c, int k, int nrp) {
  return A32 ? ((((c >> 5) * nrp + k) << 5) + (c & 31)) : ((((c >> 5) * (nrp >> 1) + (k >> 1)) << 5) + (c & 31));
}

template <bool A32>
__device__ __forceinline__ int acc_get(const uint32_t* acc, int c, int k, int nrp) {
  const uint32_t w = acc[acc_index<A32>(c, k, nrp)];
  return A32 ? (int)w : (int)((w >> ((k & 1) << 4)) & 0xffffu);
}

// One vote for row k of the column whose row-0 word is at shared address `colbase`.
// No memory clobber: the accumulator is only read after a barrier, and leaving the hit
// loads free to move above the atomics lets consecutive hits overlap.
template <bool A32>
__device__ __forceinline__ void vote_cell(uint32_t colbase, int k) {
  uint32_t addr, inc;
  if (A32) {
    addr = colbase + ((uint32_t)k << 7);
    inc = 1u;
  } else {
    addr = colbase + (((uint32_t)k >> 1) << 7);
    inc = 1u << (((uint32_t)k & 1u) << 4);
  }
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(inc));
}

// One vote for row k of a halo column: packed int16 pairs stored contiguously.
__device__ __forceinline__ void vote_halo(uint32_t colbase, int k) {
  const uint32_t addr = colbase + (((uint32_t)k >> 1) << 2);
  const uint32_t inc = 1u << (((uint32_t)k & 1u) << 4);
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(inc));
}

// In-place exclusive scan of arr[0, n) by the whole CTA; returns the total.
__device__ int block_exscan(int* arr, int n, int* s_tmp) {
  const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (n + nt - 1) / nt;
  const int lo = min(n, tid * per), hi = min(n, lo + per);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += arr[i];
  int x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_tmp[w] = x;
  __syncthreads();
  if (w == 0) {
    int z = (lane < (nt >> 5)) ? s_tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, z, o);
      if (lane >= o) z += y;
    }
    s_tmp[lane] = z;
  }
  __syncthreads();
  int excl = x - sum + (w > 0 ? s_tmp[w - 1] : 0);
  const int total = s_tmp[(nt >> 5) - 1];
  for (int i = lo; i < hi; ++i) {
    const int v = arr[i];
    arr[i] = excl;
    excl += v;
  }
  __syncthreads();
  return total;
}

__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* s_red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  if (lane == 0) s_red[w] = v;
  __syncthreads();
  unsigned long long t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_red[i];
  __syncthreads();
  return t;  // valid in thread 0
}

// ---- staging hits into shared memory ----

// Maps hits [base, base + cn) and appends those that fit the int32 fast path to hb
// (compacted, order not kept). Valid hits beyond int32 set bit 0 of *s_flags, bad
// hits bit 1.
__device__ void stage_vote32(const int2* __restrict__ xy, long long base, int cn, int2* hb, int* s_nv, int* s_flags,
                             bool as_float, long long lsq, uint16_t* idx) {
  const int lane = threadIdx.x & 31;
  // each thread's next hit is loaded one pass ahead, so the loads overlap the mapping
  int2 hn = threadIdx.x < cn ? xy[base + threadIdx.x] : make_int2(0, 0);
  for (int i0 = 0; i0 < cn; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const int2 h = hn;
    if (i + (int)blockDim.x < cn) hn = xy[base + i + blockDim.x];
    long long u = 0, v = 0;
    int st = 0;
    bool ok = false;
    if (i < cn) {
      st = map_hit(h.x, h.y, u, v);
      ok = (st == 0);
    }
    // fast path: int32 rho, and (mirror-pair layout) rho within one guard bin of the range
    const bool f = ok && fits32(u, v) && (lsq == 0 || u * u + v * v <= lsq);
    const unsigned bal = __ballot_sync(kFull, f);
    if (bal) {
      int slot = 0;
      if (lane == 0) slot = atomicAdd(s_nv, __popc(bal));
      slot = __shfl_sync(kFull, slot, 0);
      // float form for the float bin path: |u|, |v| <= 44061 are exact in float; the mirror-pair
      // layout (idx given) stores hits in pairs (u0, u1, v0, v1) for the vote's f32x2 arithmetic
      if (f) {
        const int at = slot + __popc(bal & lanemask_lt());
        if (idx) {
          float* fp = reinterpret_cast<float*>(hb) + 4 * (at >> 1) + (at & 1);
          fp[0] = (float)u;
          fp[2] = (float)v;
          idx[at] = (uint16_t)i;
        } else {
          hb[at] = as_float ? make_int2(__float_as_int((float)u), __float_as_int((float)v)) : make_int2((int)u, (int)v);
        }
      }
    }
    if (ok && !f) atomicOr(s_flags, 1);
    if (st) atomicOr(s_flags, 2);
  }
}

// Maps hits [base, base + cn) and appends every valid one as int64 to hw (compacted).
__device__ void stage_vote64(const int2* __restrict__ xy, long long base, int cn, longlong2* hw, int* s_nv) {
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < cn; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    long long u = 0, v = 0;
    bool ok = false;
    if (i < cn) {
      const int2 h = xy[base + i];
      ok = (map_hit(h.x, h.y, u, v) == 0);
    }
    const unsigned bal = __ballot_sync(kFull, ok);
    if (bal) {
      int slot = 0;
      if (lane == 0) slot = atomicAdd(s_nv, __popc(bal));
      slot = __shfl_sync(kFull, slot, 0);
      if (ok) hw[slot + __popc(bal & lanemask_lt())] = make_longlong2(u, v);
    }
  }
}

// Selection staging keeps hit order: hb[i] = (u, v), or (INT_MIN, 0) for a bad hit.
// A valid hit beyond int32 sets *s_wide.
__device__ void stage_sel32(const int2* __restrict__ xy, long long base, int cn, int2* hb, int* s_wide) {
  for (int i = threadIdx.x; i < cn; i += blockDim.x) {
    const int2 h = xy[base + i];
    long long u = 0, v = 0;
    const int st = map_hit(h.x, h.y, u, v);
    if (st) {
      hb[i] = make_int2(INT_MIN, 0);
    } else if (fits32(u, v)) {
      hb[i] = make_int2((int)u, (int)v);
    } else {
      hb[i] = make_int2(INT_MIN, 0);
      *s_wide = 1;
    }
  }
}

__device__ void stage_sel64(const int2* __restrict__ xy, long long base, int cn, longlong2* hw) {
  for (int i = threadIdx.x; i < cn; i += blockDim.x) {
    const int2 h = xy[base + i];
    long long u = 0, v = 0;
    const int st = map_hit(h.x, h.y, u, v);
    hw[i] = st ? make_longlong2(LLONG_MIN, 0) : make_longlong2(u, v);
  }
}

// ---- voting ----

// Which columns a worker lane owns, and where their row-0 words live.
struct VoteLane {
  bool on;          // lane votes
  bool halo;        // lane of the halo warp (tiles > 1)
  bool mirror;      // lane also votes the mirror column
  int p, P;         // hit partition of this warp, partitions per column set
  int cj, sj;       // trig of the (first) column
  uint32_t col1;    // shared address of column 1, row 0
  uint32_t col2;    // mirror column (mirror mode) or halo column
};

// Bin of the float estimate kf = u A + v B + N_rho/2 of k* = (u c + v s + H) N_rho / 2H, where
// A = c N_rho/2H, B = s N_rho/2H in float. |kf - k*| < N_rho 2^-21 (rounding of A, B and of
// the three float operations, each at most 2^-24 relative of a term below 1.6 N_rho), so
// floor(kf) = floor(k*) unless an integer lies within delta = N_rho 2^-20 of kf. y1 and y2
// round kc - 1/2 + delta and kc - 1/2 - delta to integers (adding 1.5 2^23 leaves no fraction
// bits); they differ exactly when such an integer exists, and then the exact integer path
// decides. Clamping kf to [1/2, N_rho - 1/2] first gives the edge bins for rho outside the
// range, as the integer clamp does.
struct FpBin {
  float khi, dlo, dhi;
};

__device__ __forceinline__ int bin_fp(float kf, const FpBin& K, float uf, float vf, int c, int s, BinMagic m) {
  const float kc = fminf(fmaxf(kf, 0.5f), K.khi);
  const float y1 = __fadd_rn(__fadd_rn(kc, K.dlo), 12582912.0f);
  const float y2 = __fadd_rn(__fadd_rn(kc, K.dhi), 12582912.0f);
  int r = __float_as_int(y1) - 0x4B400000;
  if (__float_as_int(y1) != __float_as_int(y2)) {
    const int u = __float2int_rn(uf), v = __float2int_rn(vf);
    r = rho_bin32(u * c + (v * s + (int)kH), m);
  }
  return r;
}

template <bool A32>
__device__ __forceinline__ void vote32_fp(const Plan& pl, const VoteLane& L, const int2* hb, int nv) {
  if (!L.on) return;
  const BinMagic m = pl.magic;
  const FpBin K{pl.fp_khi, pl.fp_dlo, pl.fp_dhi};
  const float c0 = pl.fp_c0;
  const int cj = L.cj, sj = L.sj;
  const float A = __fmul_rn((float)cj, pl.fp_scale), B = __fmul_rn((float)sj, pl.fp_scale);
  if (L.halo) {
    const int lane = threadIdx.x & 31;
    for (int i = lane & 15; i < nv; i += 16) {
      const float2 h = reinterpret_cast<const float2*>(hb)[i];
      vote_halo(L.col2, bin_fp(__fmaf_rn(h.x, A, __fmaf_rn(h.y, B, c0)), K, h.x, h.y, cj, sj, m));
    }
    return;
  }
  const float4* hb4 = reinterpret_cast<const float4*>(hb);
  const int np = nv >> 1, P = L.P;
  if (L.mirror) {
#pragma unroll 2
    for (int q = L.p; q < np; q += P) {
      const float4 h = hb4[q];
      const float v0 = __fmaf_rn(h.y, B, c0), v1 = __fmaf_rn(h.w, B, c0);
      vote_cell<A32>(L.col1, bin_fp(__fmaf_rn(h.x, A, v0), K, h.x, h.y, cj, sj, m));
      vote_cell<A32>(L.col2, bin_fp(__fmaf_rn(-h.x, A, v0), K, h.x, h.y, -cj, sj, m));
      vote_cell<A32>(L.col1, bin_fp(__fmaf_rn(h.z, A, v1), K, h.z, h.w, cj, sj, m));
      vote_cell<A32>(L.col2, bin_fp(__fmaf_rn(-h.z, A, v1), K, h.z, h.w, -cj, sj, m));
    }
    if ((nv & 1) && L.p == np % P) {
      const float2 h = reinterpret_cast<const float2*>(hb)[nv - 1];
      const float v0 = __fmaf_rn(h.y, B, c0);
      vote_cell<A32>(L.col1, bin_fp(__fmaf_rn(h.x, A, v0), K, h.x, h.y, cj, sj, m));
      vote_cell<A32>(L.col2, bin_fp(__fmaf_rn(-h.x, A, v0), K, h.x, h.y, -cj, sj, m));
    }
  } else {
#pragma unroll 4
    for (int q = L.p; q < np; q += P) {
      const float4 h = hb4[q];
      vote_cell<A32>(L.col1, bin_fp(__fmaf_rn(h.x, A, __fmaf_rn(h.y, B, c0)), K, h.x, h.y, cj, sj, m));
      vote_cell<A32>(L.col1, bin_fp(__fmaf_rn(h.z, A, __fmaf_rn(h.w, B, c0)), K, h.z, h.w, cj, sj, m));
    }
    if ((nv & 1) && L.p == np % P) {
      const float2 h = reinterpret_cast<const float2*>(hb)[nv - 1];
      vote_cell<A32>(L.col1, bin_fp(__fmaf_rn(h.x, A, __fmaf_rn(h.y, B, c0)), K, h.x, h.y, cj, sj, m));
    }
  }
}

template <bool A32>
__device__ __forceinline__ void vote32(const Plan& pl, const VoteLane& L, const int2* hb, int nv) {
  if (!L.on) return;
  const int Hh = (int)kH;
  const BinMagic m = pl.magic;
  const int cj = L.cj, sj = L.sj;
  if (L.halo) {
    const int lane = threadIdx.x & 31;
    for (int i = lane & 15; i < nv; i += 16) {
      const int2 h = hb[i];
      vote_halo(L.col2, rho_bin32(h.x * cj + (h.y * sj + Hh), m));
    }
    return;
  }
  const int4* hb4 = reinterpret_cast<const int4*>(hb);
  const int np = nv >> 1, P = L.P;
  if (L.mirror) {
#pragma unroll 2
    for (int q = L.p; q < np; q += P) {
      const int4 h = hb4[q];
      const int v0 = h.y * sj + Hh, u0 = h.x * cj;
      const int v1 = h.w * sj + Hh, u1 = h.z * cj;
      vote_cell<A32>(L.col1, rho_bin32(v0 + u0, m));
      vote_cell<A32>(L.col2, rho_bin32(v0 - u0, m));
      vote_cell<A32>(L.col1, rho_bin32(v1 + u1, m));
      vote_cell<A32>(L.col2, rho_bin32(v1 - u1, m));
    }
    if ((nv & 1) && L.p == np % P) {
      const int2 h = hb[nv - 1];
      const int v0 = h.y * sj + Hh, u0 = h.x * cj;
      vote_cell<A32>(L.col1, rho_bin32(v0 + u0, m));
      vote_cell<A32>(L.col2, rho_bin32(v0 - u0, m));
    }
  } else {
#pragma unroll 4
    for (int q = L.p; q < np; q += P) {
      const int4 h = hb4[q];
      vote_cell<A32>(L.col1, rho_bin32(h.x * cj + (h.y * sj + Hh), m));
      vote_cell<A32>(L.col1, rho_bin32(h.z * cj + (h.w * sj + Hh), m));
    }
    if ((nv & 1) && L.p == np % P) {
      const int2 h = hb[nv - 1];
      vote_cell<A32>(L.col1, rho_bin32(h.x * cj + (h.y * sj + Hh), m));
    }
  }
}

template <bool A32>
__device__ __forceinline__ void vote64(const Plan& pl, const VoteLane& L, const longlong2* hw, int nv) {
  if (!L.on) return;
  const BinMagic m = pl.magic;
  const long long cj = L.cj, sj = L.sj;
  if (L.halo) {
    const int lane = threadIdx.x & 31;
    for (int i = lane & 15; i < nv; i += 16) {
      const longlong2 h = hw[i];
      vote_halo(L.col2, rho_bin64(h.x * cj + h.y * sj + kH, m));
    }
    return;
  }
  for (int q = L.p; q < nv; q += L.P) {
    const longlong2 h = hw[q];
    const long long vs = h.y * sj + kH, uc = h.x * cj;
    vote_cell<A32>(L.col1, rho_bin64(vs + uc, m));
    if (L.mirror) vote_cell<A32>(L.col2, rho_bin64(vs - uc, m));
  }
}

// ---- mirror-pair word layout (untiled events, N_theta a multiple of 64) ----
// Word lane w in [0, N_theta/2) holds column w in its low half and column N_theta-1-w (its
// mirror) in its high half, one word per physical row p = k + 1. Rows p = 0 and p = N_rho + 1
// are guard rows: the fast path only takes hits whose rho stays within half a bin of the range,
// so its unclamped bins fall in [-1, N_rho]; the guard rows are folded into rows 0 and
// N_rho - 1 after the vote, which is what clamping would have done.

__device__ __forceinline__ int mp_word(int w, int p, int rows_phys) {
  return (((w >> 5) * rows_phys + p) << 5) + (w & 31);
}

// Cell (c, k) of a mirror-pair tile of Wd words; tile-local column c < Wd is word c's low half,
// c >= Wd word 2 Wd - 1 - c's high half.
__device__ __forceinline__ int mp_get(const uint32_t* acc, int c, int k, int Wd, const Plan& pl) {
  const bool hi = c >= Wd;
  const uint32_t x = acc[mp_word(hi ? 2 * Wd - 1 - c : c, k + 1, pl.rows_phys)];
  return hi ? (int)(x >> 16) : (int)(x & 0xffffu);
}

// Cells of the CTA's accumulator for the iterative finder (one tile): read, and suppress by a
// 16-bit store of zero into the cell's half of its word (a 32-bit store with int32 cells), which
// leaves the other half of the word alone.
template <bool A32, bool MP>
struct FusedCells {
  static constexpr bool kPairs = MP;  // word w holds columns w and 2 Wd - 1 - w
  uint32_t* acc;
  int Wd, nrp, rp;  // tile words, padded rows (other layouts), rows with guards (mirror-pair)
  __device__ int words() const { return Wd; }
  __device__ int mirror_col(int w) const { return 2 * Wd - 1 - w; }
  __device__ uint32_t word(int w, int k) const { return acc[mp_word(w, k + 1, rp)]; }
  // words w4 .. w4 + 3 of row k (w4 a multiple of 4: all four in one 32-word group, 16-byte aligned;
  // words past the tile's own are zero)
  __device__ uint4 words4(int w4, int k) const {
    return *reinterpret_cast<const uint4*>(acc + mp_word(w4, k + 1, rp));
  }
  __device__ int get(int j, int k) const {
    if (MP) {
      const bool hi = j >= Wd;
      const uint32_t x = acc[mp_word(hi ? 2 * Wd - 1 - j : j, k + 1, rp)];
      return hi ? (int)(x >> 16) : (int)(x & 0xffffu);
    }
    return acc_get<A32>(acc, j, k, nrp);
  }
  __device__ void clear(int j, int k) {
    if (MP) {
      const bool hi = j >= Wd;
      reinterpret_cast<uint16_t*>(acc)[2 * mp_word(hi ? 2 * Wd - 1 - j : j, k + 1, rp) + (hi ? 1 : 0)] = 0;
    } else if (A32) {
      acc[acc_index<true>(j, k, nrp)] = 0u;
    } else {
      reinterpret_cast<uint16_t*>(acc)[2 * acc_index<false>(j, k, nrp) + (k & 1)] = 0;
    }
  }
};

// Shared address of the vote whose float row estimate, shifted by 1 + 2^b + e (2^b > N_rho + 1,
// e = W/2 units of 2^-F, W a power of two), is kfp. In [2^b, 2^(b+1)) a float's low F = 23 - b
// bits are the fraction and the bits above them (127 + b) 2^b + integer part, so
// base2 + ((y >> F) << 7) with base2 = base - ((127 + b) 2^b << 7) is the row's word directly.
// The estimate is within N_rho 2^-21 + 2^-(F+1) <= e of the exact value; when the shifted
// fraction is below W (its bits above log2 W all zero: the exact value within e of an integer)
// the exact integer path (clamped) decides, otherwise the shift by e does not move the integer part.
__device__ __forceinline__ uint32_t mp_addr(float kfp, const Plan& pl, uint32_t base, uint32_t base2, float uf,
                                            float vf, int c, int s) {
  const uint32_t y = (uint32_t)__float_as_int(kfp);
  if ((y & (uint32_t)pl.mp_amask) == 0u) {
    const int u = __float2int_rn(uf), v = __float2int_rn(vf);
    return base + ((uint32_t)(rho_bin32(u * c + (v * s + (int)kH), pl.magic) + 1) << 7);
  }
  return base2 + ((y >> pl.mp_F) << 7);
}

__device__ __forceinline__ void red_u32(uint32_t addr, uint32_t inc) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(inc));
}

// d = a * b + c on pairs of floats (packed f32x2, each lane rounded as one fused multiply-add).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// Hit i of the mirror-pair staging: pairs of hits (u0, u1, v0, v1).
__device__ __forceinline__ float2 staged_hit(const float* f, int i) {
  const float* q = f + 4 * (i >> 1) + (i & 1);
  return make_float2(q[0], q[2]);
}

// The four votes of one staged pair of hits (u0, u1, v0, v1) into a word's two columns: row
// estimates of column j (+A) and of its mirror (-A), packed two hits at a time.
struct PairEst {
  float2 k02, k13;  // (hit 0, hit 1) in the low column, then in the high column
};

__device__ __forceinline__ PairEst pair_est(float4 h, float2 AA, float2 NAA, float2 BB, float2 CC) {
  const float2 V = fma2(make_float2(h.z, h.w), BB, CC);
  return PairEst{fma2(make_float2(h.x, h.y), AA, V), fma2(make_float2(h.x, h.y), NAA, V)};
}

__device__ __forceinline__ bool pair_clear(const PairEst& e, uint32_t am) {
  return ((__float_as_uint(e.k02.x) & am) != 0u) & ((__float_as_uint(e.k13.x) & am) != 0u) &
         ((__float_as_uint(e.k02.y) & am) != 0u) & ((__float_as_uint(e.k13.y) & am) != 0u);
}

__device__ __forceinline__ void pair_red_fast(const PairEst& e, uint32_t base2, int F) {
  red_u32(base2 + ((__float_as_uint(e.k02.x) >> F) << 7), 1u);
  red_u32(base2 + ((__float_as_uint(e.k13.x) >> F) << 7), 0x10000u);
  red_u32(base2 + ((__float_as_uint(e.k02.y) >> F) << 7), 1u);
  red_u32(base2 + ((__float_as_uint(e.k13.y) >> F) << 7), 0x10000u);
}

__device__ __forceinline__ void pair_red_exact(const PairEst& e, float4 h, const Plan& pl, uint32_t base,
                                               uint32_t base2, int cj, int sj) {
  red_u32(mp_addr(e.k02.x, pl, base, base2, h.x, h.z, cj, sj), 1u);
  red_u32(mp_addr(e.k13.x, pl, base, base2, h.x, h.z, -cj, sj), 0x10000u);
  red_u32(mp_addr(e.k02.y, pl, base, base2, h.y, h.w, cj, sj), 1u);
  red_u32(mp_addr(e.k13.y, pl, base, base2, h.y, h.w, -cj, sj), 0x10000u);
}

__device__ __forceinline__ void vote_mp32(const Plan& pl, const VoteLane& L, const int2* hb, int nv) {
  const int cj = L.cj, sj = L.sj;
  const float* hf = reinterpret_cast<const float*>(hb);
  if (L.halo) {
    // A halo word of a tile (columns j and N-1-j), 16 lanes: the same float row estimate as
    // the tile's own words, into a contiguous column (4 bytes per row, guard rows folded
    // like the accumulator's), exact bins when ambiguous.
    if (!L.on) return;
    const float A = __fmul_rn((float)cj, pl.fp_scale), B = __fmul_rn((float)sj, pl.fp_scale);
    const float c0 = pl.mp_c0;
    const uint32_t am = (uint32_t)pl.mp_amask, base2 = L.col2 - ((uint32_t)pl.mp_k7 >> 5);
    const int F = pl.mp_F;
#pragma unroll 2
    for (int i = L.p; i < nv; i += L.P) {
      const float2 h = staged_hit(hf, i);
      const float v0 = __fmaf_rn(h.y, B, c0);
      const uint32_t y0 = (uint32_t)__float_as_int(__fmaf_rn(h.x, A, v0));
      const uint32_t y1 = (uint32_t)__float_as_int(__fmaf_rn(-h.x, A, v0));
      if (((y0 & am) != 0u) & ((y1 & am) != 0u)) {
        red_u32(base2 + ((y0 >> F) << 2), 1u);
        red_u32(base2 + ((y1 >> F) << 2), 0x10000u);
      } else {
        const int u = __float2int_rn(h.x), vs = __float2int_rn(h.y) * sj + (int)kH;
        red_u32(L.col2 + ((uint32_t)(rho_bin32(u * cj + vs, pl.magic) + 1) << 2), 1u);
        red_u32(L.col2 + ((uint32_t)(rho_bin32(vs - u * cj, pl.magic) + 1) << 2), 0x10000u);
      }
    }
    return;
  }
  const float A = __fmul_rn((float)cj, pl.fp_scale), B = __fmul_rn((float)sj, pl.fp_scale);
  if (!L.on) return;
  const float2 AA = make_float2(A, A), NAA = make_float2(-A, -A), BB = make_float2(B, B);
  const float2 CC = make_float2(pl.mp_c0, pl.mp_c0);
  const uint32_t base = L.col1, base2 = L.col1 - (uint32_t)pl.mp_k7;
  const float4* hb4 = reinterpret_cast<const float4*>(hb);
  const int np = nv >> 1, P = L.P;
  const uint32_t am = (uint32_t)pl.mp_amask;
  const int F = pl.mp_F;
  // One pair of hits (4 votes) a step and one exactness test for the 4: the rare step with an
  // estimate in the ambiguous window takes the exact path vote by vote. (Two pairs a step with one
  // test for 8 votes measured slower inside this kernel: 43.4 k against 39.6 k cycles an event.)
#pragma unroll 4
  for (int q = L.p; q < np; q += P) {
    const float4 g = hb4[q];
    const PairEst eg = pair_est(g, AA, NAA, BB, CC);
    if (pair_clear(eg, am)) pair_red_fast(eg, base2, F);
    else pair_red_exact(eg, g, pl, base, base2, cj, sj);
  }
  if ((nv & 1) && L.p == np % P) {
    const float2 h = staged_hit(hf, nv - 1);
    const float v0 = __fmaf_rn(h.y, B, pl.mp_c0);
    red_u32(mp_addr(__fmaf_rn(h.x, A, v0), pl, base, base2, h.x, h.y, cj, sj), 1u);
    red_u32(mp_addr(__fmaf_rn(-h.x, A, v0), pl, base, base2, h.x, h.y, -cj, sj), 0x10000u);
  }
}

__device__ __forceinline__ void vote_mp64(const Plan& pl, const VoteLane& L, const longlong2* hw, int nv) {
  const BinMagic m = pl.magic;
  const long long cj = L.cj, sj = L.sj;
  if (L.halo) {
    if (!L.on) return;
    for (int i = L.p; i < nv; i += L.P) {
      const longlong2 h = hw[i];
      const long long vs = h.y * sj + kH, uc = h.x * cj;
      red_u32(L.col2 + ((uint32_t)(rho_bin64(vs + uc, m) + 1) << 2), 1u);
      red_u32(L.col2 + ((uint32_t)(rho_bin64(vs - uc, m) + 1) << 2), 0x10000u);
    }
    return;
  }
  if (!L.on) return;
  for (int q = L.p; q < nv; q += L.P) {
    const longlong2 h = hw[q];
    const long long vs = h.y * sj + kH, uc = h.x * cj;
    red_u32(L.col1 + ((uint32_t)(rho_bin64(vs + uc, m) + 1) << 7), 1u);
    red_u32(L.col1 + ((uint32_t)(rho_bin64(vs - uc, m) + 1) << 7), 0x10000u);
  }
}

// Guard rows into the edge rows (both halves at once: a column holds at most 32767 votes,
// so the packed add never carries across halves).
__device__ void mp_fold(const Plan& pl, uint32_t* acc, int n_words, uint32_t* halo) {
  const int rp = pl.rows_phys, NR = pl.n_rho;
  for (int w = threadIdx.x; w < n_words; w += blockDim.x) {
    uint32_t* col = acc + mp_word(w, 0, rp);
    col[32] += col[0];
    col[NR << 5] += col[(NR + 1) << 5];
    col[0] = 0u;  // zero guard rows now read as "no neighbour" in the scan
    col[(NR + 1) << 5] = 0u;
  }
  if (halo && threadIdx.x < 2) {  // the tile's two halo words (contiguous rows)
    uint32_t* col = halo + threadIdx.x * rp;
    col[1] += col[0];
    col[NR] += col[NR + 1];
    col[0] = 0u;
    col[NR + 1] = 0u;
  }
}

// Peak scan of the mirror-pair layout: one row per step, both columns of a word at once.
// For word lane w, lane w-1 holds the left neighbour of column w and the right neighbour of
// column N-1-w; lane w+1 the other two. Lane w = -1 supplies the theta wrap (word lane 0, rows
// mirrored, halves swapped) and lane w = N/2 the middle (word lane N/2-1, halves swapped).
// A tile owns words [aw, aw + half) (columns aw.. and their mirrors); its neighbour words
// aw - 1 and aw + half come from the halo (two contiguous columns of rows_phys words, no
// mirroring) unless the tile starts at word 0 (theta wrap) or ends at the middle word.
__device__ void scan_mp(const Plan& pl, const uint32_t* acc, const uint32_t* halo, int aw, int half,
                        uint32_t* pbits, bool do_cs, unsigned long long& csum) {
  const int NT = pl.n_theta, NR = pl.n_rho, R = pl.scan_ranges, rp = pl.rows_phys;
  const bool first = aw == 0, last = aw + half == (NT >> 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nblk = (half + 29) / 30;
  const uint32_t TT = (uint32_t)pl.threshold | ((uint32_t)pl.threshold << 16);
  for (int u = warp; u < nblk * R; u += nwarps) {
    const int b = u >> pl.scan_shift, r = u & (R - 1);
    const int k0 = (NR * r) >> pl.scan_shift, k1 = (NR * (r + 1)) >> pl.scan_shift;
    const int w = b * 30 + lane - 1;
    // Source word of this lane for logical row k: physical row k + 1 (or N_rho - k when the
    // rows are mirrored); the zeroed guard rows supply the missing rows -1 and N_rho.
    int sw = w, p0 = k0, step = 32;
    unsigned sel = 0x3210u;  // byte permutation: identity, or swap of the two halves
    const uint32_t* hcol = nullptr;
    if (w < 0) {
      if (first) {
        sw = 0;
        p0 = NR - (k0 - 1);
        step = -32;
        sel = 0x1032u;
      } else {
        hcol = halo;
      }
    } else if (w >= half) {
      if (w == half && last) {
        sw = half - 1;
        sel = 0x1032u;
      } else if (w == half) {
        hcol = halo + rp;
      } else {
        sw = 0;  // nothing: read guard row 0 (zero) throughout
        p0 = 0;
        step = 0;
      }
    }
    const uint32_t* ptr = hcol ? hcol + k0 : acc + mp_word(sw, p0, rp);  // row k0 - 1
    if (hcol) step = 1;
    const bool tested = lane >= 1 && lane <= 30 && w >= 0 && w < half;
    // Raster order runs over theta, then rho: the row above and the preceding column are
    // "before" a cell (strictly below it at a peak), the rest "after" (at most equal). The
    // preceding column of the low half (column aw+w) is lane w-1's low half (the wrapped
    // column N-1 at word 0: after, not before); of the high half (column N-1-aw-w) lane w+1's
    // high half; lane w-1's high half follows it (except at word 0: the wrapped column 0).
    // Strictness becomes +1 on that neighbour, so a cell is a peak iff C >= max(U + 1, D,
    // VU + addU, VD + 0x10000, T) per half; cells are at most 32767, so nothing carries.
    const uint32_t addU = (w != 0 || !first) ? 1u : 0x10000u;
    const int clo = w, chi = 2 * half - 1 - w;                // tile-local columns
    const int glo = aw + w, ghi = NT - 1 - aw - w;             // event columns
    uint32_t U = __byte_perm(ptr[0], 0u, sel);
    ptr += step;
    uint32_t C = __byte_perm(ptr[0], 0u, sel);
    ptr += step;
    for (int ks = k0; ks < k1;) {
      const int ke = min(k1, (ks | 31) + 1);  // rows of one bitmap word
      uint32_t bl = 0, bh = 0;                // peak flags, newest row in bit 0
      int k = ks;
      // Groups of four rows: the loads and the candidate test run straight through, and the
      // neighbour test only for a group where some tested cell reaches T (bit 15 of a half of
      // 0x8000 - (max(C, T) - C) is set iff C >= T); most groups have none.
      for (; k + 4 <= ke; k += 4) {
        uint32_t R4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          R4[i] = __byte_perm(ptr[0], 0u, sel);
          ptr += step;
        }
        const uint32_t c1 = R4[0], c2 = R4[1], c3 = R4[2];
        const uint32_t cand = ((0x80008000u - vmax2(C, TT) + C) | (0x80008000u - vmax2(c1, TT) + c1) |
                               (0x80008000u - vmax2(c2, TT) + c2) | (0x80008000u - vmax2(c3, TT) + c3)) &
                              0x80008000u;
        if (__any_sync(kFull, tested && cand != 0u)) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t Cc = i == 0 ? C : R4[i - 1], Uu = i == 0 ? U : (i == 1 ? C : R4[i - 2]), Dd = R4[i];
            const uint32_t VM = vmax2(vmax2(Uu, Cc), Dd);
            const uint32_t VU = __shfl_up_sync(kFull, VM, 1);
            const uint32_t VD = __shfl_down_sync(kFull, VM, 1);
            const uint32_t X = vmax2(vmax2(vmax2(Uu + 0x00010001u, Dd), vmax2(VU + addU, VD + 0x10000u)), TT);
            const uint32_t Z = 0x80008000u - vmax2(X, Cc) + Cc;
            bh = __funnelshift_l(Z, bh, 1);
            bl = __funnelshift_l(Z << 16, bl, 1);
          }
        } else {
          bh <<= 4;
          bl <<= 4;
        }
        if (do_cs && tested) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t Cc = i == 0 ? C : R4[i - 1];
            const unsigned a0 = Cc & 0xffffu, a1 = Cc >> 16;
            if (a0) csum += (unsigned long long)a0 * mix64((unsigned long long)glo * NR + k + i + 1);
            if (a1) csum += (unsigned long long)a1 * mix64((unsigned long long)ghi * NR + k + i + 1);
          }
        }
        U = R4[2];
        C = R4[3];
      }
#pragma unroll 4
      for (; k < ke; ++k) {
        const uint32_t D = __byte_perm(ptr[0], 0u, sel);
        ptr += step;
        const uint32_t VM = vmax2(vmax2(U, C), D);
        const uint32_t VU = __shfl_up_sync(kFull, VM, 1);
        const uint32_t VD = __shfl_down_sync(kFull, VM, 1);
        const uint32_t X = vmax2(vmax2(vmax2(U + 0x00010001u, D), vmax2(VU + addU, VD + 0x10000u)), TT);
        // half of Z has bit 15 set iff C >= X there: 0x8000 - (max(X, C) - C), no borrow
        const uint32_t Z = 0x80008000u - vmax2(X, C) + C;
        bh = __funnelshift_l(Z, bh, 1);
        bl = __funnelshift_l(Z << 16, bl, 1);
        if (do_cs && tested) {
          const unsigned a0 = C & 0xffffu, a1 = C >> 16;
          if (a0) csum += (unsigned long long)a0 * mix64((unsigned long long)glo * NR + k + 1);
          if (a1) csum += (unsigned long long)a1 * mix64((unsigned long long)ghi * NR + k + 1);
        }
        U = C;
        C = D;
      }
      if (tested) {
        const int sh = 32 - (ke - ks) - (ks & 31);  // row ks to bit ks & 31
        bl = __brev(bl) >> sh;
        bh = __brev(bh) >> sh;
        if (bl) atomicOr(&pbits[clo * pl.nrb + (ks >> 5)], bl);
        if (bh) atomicOr(&pbits[chi * pl.nrb + (ks >> 5)], bh);
      }
      ks = ke;
    }
  }
}

// ---- peak scan ----

// Row range [k0, k1) of scan range r (word aligned in the packed scan).
// (The number of ranges is a power of two, 2^scan_shift.)
__device__ __forceinline__ void scan_rows(const Plan& pl, bool packed, int r, int& k0, int& k1) {
  const int sh = pl.scan_shift;
  if (packed) {
    const int W2 = pl.n_rho >> 1;
    k0 = 2 * ((W2 * r) >> sh);
    k1 = 2 * ((W2 * (r + 1)) >> sh);
  } else {
    k0 = (pl.n_rho * r) >> sh;
    k1 = (pl.n_rho * (r + 1)) >> sh;
  }
}

// Column source of one scan lane: the tile column itself, a halo column, or the tile's own
// far column mirrored (theta wrap of an untiled event), or nothing.
struct ScanSrc {
  int kind;  // 0 tile column, 1 left halo, 2 right halo, 3 none
  int col;   // tile column for kind 0
  bool mir;  // rows mirrored (k -> N_rho - 1 - k)
};

__device__ __forceinline__ ScanSrc scan_src(int c, int wt, int T, int j0, int NT) {
  ScanSrc s{0, c, false};
  if (c < 0) {
    if (T == 1) {
      s.col = wt - 1;
      s.mir = true;
    } else {
      s.kind = 1;
      s.mir = (j0 == 0);
    }
  } else if (c >= wt) {
    if (c == wt) {
      if (T == 1) {
        s.col = 0;
        s.mir = true;
      } else {
        s.kind = 2;
        s.mir = (j0 + wt == NT);
      }
    } else {
      s.kind = 3;
    }
  }
  return s;
}

// Packed int16 scan (N_rho even): two rows per step, max.u16x2 for the 3-row column maxima,
// one shuffle each way for the neighbour columns, exact tie test only for candidates.
// Missing neighbours (rho edges, no column) read as 0, which never blocks a cell >= T >= 1.
__device__ void scan_packed(const Plan& pl, const uint32_t* acc, const uint32_t* halo, uint32_t* pbits,
                            int wt, int T, int j0, bool do_cs, unsigned long long& csum) {
  const int NT = pl.n_theta, NR = pl.n_rho, W2 = NR >> 1, R = pl.scan_ranges;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nblk = (wt + 29) / 30;
  const uint32_t TT = (uint32_t)pl.threshold | ((uint32_t)pl.threshold << 16);
  for (int u = warp; u < nblk * R; u += nwarps) {
    const int b = u >> pl.scan_shift, r = u & (R - 1);
    int k0, k1;
    scan_rows(pl, true, r, k0, k1);
    const int w0 = k0 >> 1, w1 = k1 >> 1;
    const int c = b * 30 + lane - 1;
    const ScanSrc s = scan_src(c, wt, T, j0, NT);
    const uint32_t* col = nullptr;
    int stride = 32;
    if (s.kind == 0) {
      col = acc + ((s.col >> 5) * W2 << 5) + (s.col & 31);
    } else if (s.kind < 3) {
      col = halo + (s.kind - 1) * W2;
      stride = 1;
    }
    auto fetch = [&](int w) -> uint32_t {
      if (!col || w < 0 || w >= W2) return 0u;
      const uint32_t x = col[(s.mir ? W2 - 1 - w : w) * stride];
      return s.mir ? swap16(x) : x;
    };
    const bool tested = lane >= 1 && lane <= 30 && c >= 0 && c < wt;
    const bool lstrict = !(c == 0 && j0 == 0);
    const bool rstrict = (c == wt - 1) && (j0 + wt == NT);
    // Both rows of a word at once: a cell is a peak iff C >= max(U + 1, D, VL (+1 when the
    // left column precedes it), VR (+1 when the right column is the wrapped column 0), T)
    // per half; cells are at most 32767, so nothing carries across halves.
    const uint32_t addL = lstrict ? 0x00010001u : 0u, addR = rstrict ? 0x00010001u : 0u;
    uint32_t P = fetch(w0 - 1), C = fetch(w0);
    const unsigned long long cell0 = (unsigned long long)(j0 + c) * NR;
    for (int ws = w0; ws < w1;) {
      const int we = min(w1, (ws | 15) + 1);  // row pairs of one bitmap word
      uint32_t bits = 0;                      // peak flags, row k in bit k & 31
      for (int w = ws; w < we; ++w) {
        const uint32_t N = fetch(w + 1);
        // the neighbour test only where some tested cell of the warp reaches T
        const uint32_t cand = (0x80008000u - vmax2(C, TT) + C) & 0x80008000u;
        if (__any_sync(kFull, tested && cand != 0u)) {
          const uint32_t U = __funnelshift_r(P, C, 16);   // rows 2w-1, 2w
          const uint32_t D = __funnelshift_r(C, N, 16);   // rows 2w+1, 2w+2
          const uint32_t VM = vmax2(vmax2(U, C), D);
          const uint32_t VL = __shfl_up_sync(kFull, VM, 1);
          const uint32_t VR = __shfl_down_sync(kFull, VM, 1);
          const uint32_t X = vmax2(vmax2(vmax2(U + 0x00010001u, D), vmax2(VL + addL, VR + addR)), TT);
          const uint32_t Z = 0x80008000u - vmax2(X, C) + C;  // bit 15 of a half: C >= X there
          bits |= (((Z >> 15) & 1u) | ((Z >> 30) & 2u)) << ((2 * w) & 31);  // rows 2w, 2w + 1
        }
        if (do_cs && tested) {
          const unsigned a0 = C & 0xffffu, a1 = C >> 16;
          if (a0) csum += (unsigned long long)a0 * mix64(cell0 + 2 * w + 1);
          if (a1) csum += (unsigned long long)a1 * mix64(cell0 + 2 * w + 2);
        }
        P = C;
        C = N;
      }
      if (tested && bits) atomicOr(&pbits[c * pl.nrb + (ws >> 4)], bits);
      ws = we;
    }
  }
}

// Scalar scan for the int32-cell layout or an odd N_rho: one row per step.
template <bool A32>
__device__ void scan_scalar(const Plan& pl, const uint32_t* acc, const uint32_t* halo, uint32_t* pbits,
                            int wt, int T, int j0, bool do_cs, unsigned long long& csum) {
  const int NT = pl.n_theta, NR = pl.n_rho, nrp = pl.nrho_pad, R = pl.scan_ranges;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nblk = (wt + 29) / 30;
  for (int u = warp; u < nblk * R; u += nwarps) {
    const int b = u >> pl.scan_shift, r = u & (R - 1);
    int k0, k1;
    scan_rows(pl, false, r, k0, k1);
    const int c = b * 30 + lane - 1;
    const ScanSrc s = scan_src(c, wt, T, j0, NT);
    auto fetch = [&](int kk) -> int {
      const int rr = s.mir ? NR - 1 - kk : kk;
      if (s.kind == 3 || rr < 0 || rr >= NR) return -1;
      if (s.kind == 0) return acc_get<A32>(acc, s.col, rr, nrp);
      return (int)((halo[(s.kind - 1) * (nrp >> 1) + (rr >> 1)] >> ((rr & 1) << 4)) & 0xffffu);
    };
    const bool tested = lane >= 1 && lane <= 30 && c >= 0 && c < wt;
    const bool lstrict = !(c == 0 && j0 == 0);
    const bool rstrict = (c == wt - 1) && (j0 + wt == NT);
    int vp = fetch(k0 - 1), vc = fetch(k0);
    const unsigned long long cell0 = (unsigned long long)(j0 + c) * NR;
    for (int k = k0; k < k1; ++k) {
      const int vn = fetch(k + 1);
      const int vm = max(max(vp, vc), vn);
      const int vmL = __shfl_up_sync(kFull, vm, 1);
      const int vmR = __shfl_down_sync(kFull, vm, 1);
      if (tested && vc >= pl.threshold && vc > vp && vc >= vn && (lstrict ? vc > vmL : vc >= vmL) &&
          (rstrict ? vc > vmR : vc >= vmR)) {
        atomicOr(&pbits[c * pl.nrb + (k >> 5)], 1u << (k & 31));
      }
      if (do_cs && tested && vc > 0) csum += (unsigned long long)vc * mix64(cell0 + k + 1);
      vp = vc;
      vc = vn;
    }
  }
}

// ---- selection: a lane tries the kSelCap most populated peak columns for its hit; hits
// still open go to a whole warp that tests 32 columns per step ----

template <bool WIDE>
__device__ __forceinline__ bool sel_test(const Plan& pl, long long u, long long v, int2 c2, const uint32_t* bmd) {
  const int k = WIDE ? rho_bin64(u * c2.x + v * c2.y + kH, pl.magic)
                     : rho_bin32((int)u * c2.x + ((int)v * c2.y + (int)kH), pl.magic);
  return (bmd[k >> 5] >> (k & 31)) & 1u;
}

template <bool WIDE>
__device__ int select_chunk(const Plan& pl, const void* buf, int cn, long long mbase, uint8_t* __restrict__ mask,
                            const int2* cs, const uint32_t* bm, int D, uint32_t* unres) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nrb = pl.nrb;
  const int cap = min(D, kSelCap);
  int kept = 0;
  for (int i0 = 0; i0 < cn; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    bool hard = false;
    if (i < cn) {
      long long u, v;
      bool bad;
      if (WIDE) {
        const longlong2 h = reinterpret_cast<const longlong2*>(buf)[i];
        u = h.x;
        v = h.y;
        bad = (h.x == LLONG_MIN);
      } else {
        const int2 h = reinterpret_cast<const int2*>(buf)[i];
        u = h.x;
        v = h.y;
        bad = (h.x == INT_MIN);
      }
      bool m = false;
      if (!bad)
        for (int d = 0; d < cap && !m; ++d) m = sel_test<WIDE>(pl, u, v, cs[d], bm + d * nrb);
      if (m) {
        mask[mbase + i] = 1;
        ++kept;
      } else if (bad || cap == D) {
        mask[mbase + i] = 0;
      } else {
        hard = true;
      }
    }
    const unsigned hb = __ballot_sync(kFull, hard);
    if (lane == 0) unres[(i0 >> 5) + warp] = hb;
  }
  __syncthreads();
  if (D > cap) {
    const int nw = (cn + 31) >> 5;
    for (int wi = warp; wi < nw; wi += nwarps) {
      uint32_t bits = unres[wi];
      while (bits) {
        const int i = (wi << 5) + __ffs(bits) - 1;
        bits &= bits - 1u;
        long long u, v;
        if (WIDE) {
          const longlong2 h = reinterpret_cast<const longlong2*>(buf)[i];
          u = h.x;
          v = h.y;
        } else {
          const int2 h = reinterpret_cast<const int2*>(buf)[i];
          u = h.x;
          v = h.y;
        }
        bool m = false;
        for (int d0 = cap; d0 < D && !m; d0 += 32) {
          const int d = d0 + lane;
          const bool t = d < D && sel_test<WIDE>(pl, u, v, cs[d], bm + d * nrb);
          m = __any_sync(kFull, t);
        }
        if (lane == 0) {
          mask[mbase + i] = m ? 1 : 0;
          kept += m;
        }
      }
    }
  }
  __syncthreads();
  return kept;
}

// Selection over the vote's staged hits (mirror-pair plan, one chunk, no wide hits): floats
// (u, v) in staging order with their original index. The bin comes from the vote's float
// estimate (physical row p = k + 1 read off the bit pattern, exact integer path when
// ambiguous); the dilated bitmaps carry guard bits 0 and N_rho + 1 equal to the edge bins'.
__device__ __forceinline__ bool sel_test_fp(const Plan& pl, float u, float v, int d, const float2* fab,
                                            const int2* cs, const uint32_t* bm) {
  const float2 ab = fab[d];
  const uint32_t y = (uint32_t)__float_as_int(__fmaf_rn(u, ab.x, __fmaf_rn(v, ab.y, pl.mp_c0)));
  int p;
  if ((y & (uint32_t)pl.mp_amask) == 0u) {
    const int2 c2 = cs[d];
    p = rho_bin32(__float2int_rn(u) * c2.x + (__float2int_rn(v) * c2.y + (int)kH), pl.magic) + 1;
  } else {
    p = (int)((y >> pl.mp_F) & (uint32_t)pl.mp_rmask);
  }
  return (bm[d * pl.nrb_g + (p >> 5)] >> (p & 31)) & 1u;
}

__device__ int select_staged(const Plan& pl, const int2* hb, const uint16_t* idx, int nv, long long a,
                             uint8_t* __restrict__ mask, const int2* cs, const float2* fab, const uint32_t* bm, int D,
                             uint32_t* unres) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int cap = min(D, kSelCap);
  const float* hf = reinterpret_cast<const float*>(hb);
  int kept = 0;
  for (int i0 = 0; i0 < nv; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    bool hard = false;
    if (i < nv) {
      const float2 h = staged_hit(hf, i);
      bool m = false;
      for (int d = 0; d < cap && !m; ++d) m = sel_test_fp(pl, h.x, h.y, d, fab, cs, bm);
      if (m) {
        mask[a + idx[i]] = 1;
        ++kept;
      } else {
        hard = cap < D;
      }
    }
    const unsigned hbits = __ballot_sync(kFull, hard);
    if (lane == 0) unres[(i0 >> 5) + warp] = hbits;
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_SEL_A);
  if (D > cap) {
    // Open hits come in runs (staging order follows the input), so warp w takes hit
    // 32 j + w of every word j, sweeping 32 words per ballot: runs spread over all warps.
    const int nw = (nv + 31) >> 5;
    for (int wi0 = 0; wi0 < nw; wi0 += 32) {
      for (int ws = warp; ws < 32; ws += nwarps) {
        const uint32_t word = (wi0 + lane < nw) ? unres[wi0 + lane] : 0u;
        uint32_t bits = __ballot_sync(kFull, (word >> ws) & 1u);
        while (bits) {
          const int i = ((wi0 + __ffs(bits) - 1) << 5) + ws;
          bits &= bits - 1u;
          const float2 h = staged_hit(hf, i);
          bool m = false;
          for (int d0 = cap; d0 < D && !m; d0 += 32) {
            const int d = d0 + lane;
            m = __any_sync(kFull, d < D && sel_test_fp(pl, h.x, h.y, d, fab, cs, bm));
          }
          if (lane == 0 && m) {
            mask[a + idx[i]] = 1;
            ++kept;
          }
        }
      }
    }
  }
  __syncthreads();
  return kept;
}

struct ItemShared {
  int nv, flags, wide, last, total, D, reuse;
  int kept_tot;
  long long tstart[128];  // segment starts of the tile merge (2 segments a mirror-pair tile)
  int tmp[32];
  unsigned long long red[32];
  int it_max, it_tq, it_ok, it_C, it_kept;  // iterative finder on theta tiles
};

// Word W of column P's peak rows dilated by +-hw (hw < 32) and cut to [0, N_rho): bit k is
// set iff a peak lies within hw rows of k (0 outside the column's nrb words).
__device__ __forceinline__ uint32_t dilated_word(const uint32_t* P, int W, int nrb, int NR, int hw) {
  if (W < 0 || W >= nrb) return 0u;
  const uint32_t pm = W > 0 ? P[W - 1] : 0u, p0 = P[W], pp = W + 1 < nrb ? P[W + 1] : 0u;
  uint32_t d = p0;
  for (int s = 1; s <= hw; ++s) d |= (p0 << s) | (pm >> (32 - s)) | (p0 >> s) | (pp << (32 - s));
  const int valid = NR - (W << 5);
  return valid < 32 ? d & ((1u << valid) - 1u) : d;
}

// Back-projection of every hit of event e against its stored peaks pk[0, S). With
// from_bits (one tile, every peak stored, keep_halfwidth < 32) the peak columns and the
// dilated bitmaps come straight from the scan's peak bitmap pbits, which then holds exactly
// the stored peaks.
__device__ int select_event(const Plan& pl, const FusedIO& io, unsigned char* smem, ItemShared& sh,
                            const int16_t* tc, const int16_t* ts, long long a, int n, const hough_peak* pk, int S,
                            bool from_bits) {
  const int NT = pl.n_theta, NR = pl.n_rho, tid = threadIdx.x, bd = blockDim.x;
  int* colcnt = reinterpret_cast<int*>(smem + pl.off_acc);
  int* colidx = colcnt + NT;
  int* hist = colidx + NT;
  int2* cs = reinterpret_cast<int2*>(hist + 64);
  float2* fab = reinterpret_cast<float2*>(cs + NT);
  uint32_t* bm = reinterpret_cast<uint32_t*>(fab + NT);
  uint32_t* unres = reinterpret_cast<uint32_t*>(smem + pl.off_unres);
  const bool staged = sh.reuse != 0;
  const int nrb = staged ? pl.nrb_g : pl.nrb;  // guard-bit bitmaps are one bit wider on each side
  const uint32_t* pbits = reinterpret_cast<const uint32_t*>(smem + pl.off_pbits);
  for (int i = tid; i < 64; i += bd) hist[i] = 0;
  if (from_bits) {
    for (int j = tid; j < NT; j += bd) {
      int cc = 0;
      for (int w = 0; w < pl.nrb; ++w) cc += __popc(pbits[j * pl.nrb + w]);
      colcnt[j] = cc;
    }
  } else {
    for (int i = tid; i < NT; i += bd) colcnt[i] = 0;
    __syncthreads();
    for (int q = tid; q < S; q += bd) atomicAdd(&colcnt[pk[q].theta_bin], 1);
  }
  __syncthreads();
  for (int j = tid; j < NT; j += bd)
    if (colcnt[j] > 0) atomicAdd(&hist[63 - min(colcnt[j], 63)], 1);
  __syncthreads();
  if (tid < 32) {
    const int x0 = hist[2 * tid], x1 = hist[2 * tid + 1];
    int x = x0 + x1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, x, o);
      if (tid >= o) x += y;
    }
    const int ex = x - x0 - x1;
    hist[2 * tid] = ex;
    hist[2 * tid + 1] = ex + x0;
    if (tid == 31) sh.D = x;
  }
  __syncthreads();
  for (int j = tid; j < NT; j += bd) {
    const int cc = colcnt[j];
    if (cc > 0) {
      const int pos = atomicAdd(&hist[63 - min(cc, 63)], 1);
      colidx[j] = pos;
      cs[pos] = make_int2(tc[j], ts[j]);
      fab[pos] = make_float2(__fmul_rn((float)tc[j], pl.fp_scale), __fmul_rn((float)ts[j], pl.fp_scale));
    }
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_SEL_COLUMNS);
  const int D = sh.D;
  const int hw = pl.keep_hw;
  if (from_bits) {
    for (int j = tid; j < NT; j += bd) {
      if (colcnt[j] == 0) continue;
      const uint32_t* P = pbits + j * pl.nrb;
      uint32_t* out = bm + colidx[j] * nrb;
      if (!staged) {
        for (int W = 0; W < nrb; ++W) out[W] = dilated_word(P, W, pl.nrb, NR, hw);
      } else {
        // bit k + 1 for row k; guard bits 0 and N_rho + 1 copy rows 0 and N_rho - 1
        const uint32_t last = (dilated_word(P, (NR - 1) >> 5, pl.nrb, NR, hw) >> ((NR - 1) & 31)) & 1u;
        uint32_t prev = 0u;
        for (int W = 0; W < nrb; ++W) {
          const uint32_t cur = dilated_word(P, W, pl.nrb, NR, hw);
          uint32_t g = (cur << 1) | (prev >> 31);
          if (W == 0) g |= cur & 1u;
          if (W == ((NR + 1) >> 5)) g |= last << ((NR + 1) & 31);
          out[W] = g;
          prev = cur;
        }
      }
    }
  } else {
  for (int i = tid; i < D * nrb; i += bd) bm[i] = 0;
  __syncthreads();
  for (int q = tid; q < S; q += bd) {
    const hough_peak pq = pk[q];
    const int d = colidx[pq.theta_bin];
    int lo = max(0, (int)pq.rho_bin - hw), hi = min(NR - 1, (int)pq.rho_bin + hw);
    if (staged) {  // bit k + 1 for row k; guard bits 0 and N_rho + 1 copy rows 0 and N_rho - 1
      lo = (lo == 0) ? 0 : lo + 1;
      hi = (hi == NR - 1) ? NR + 1 : hi + 1;
    }
    for (int w = lo >> 5; w <= (hi >> 5); ++w) {
      const int b0 = max(lo, w << 5) & 31, b1 = min(hi, (w << 5) + 31) & 31;
      const uint32_t bits = (b1 == 31 ? 0xffffffffu : ((1u << (b1 + 1)) - 1u)) & ~((1u << b0) - 1u);
      atomicOr(&bm[d * nrb + w], bits);
    }
  }
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_SEL_BITMAPS);
  int kept = 0;
  if (D == 0) {
    for (int i = tid; i < n; i += bd) io.mask[a + i] = 0;
    return 0;
  }
  if (staged) {
    for (int i = tid; i < n; i += bd) io.mask[a + i] = 0;
    __syncthreads();
    return select_staged(pl, reinterpret_cast<const int2*>(smem + pl.off_hits),
                         reinterpret_cast<const uint16_t*>(smem + pl.off_idx), sh.nv, a, io.mask, cs, fab, bm, D,
                         unres);
  }
  int2* hb = reinterpret_cast<int2*>(smem + pl.off_hits);
  longlong2* hw64 = reinterpret_cast<longlong2*>(smem + pl.off_hits);
  for (int h0 = 0; h0 < n; h0 += pl.hit_cap) {
    const int cn = min(pl.hit_cap, n - h0);
    if (tid == 0) sh.wide = 0;
    __syncthreads();
    stage_sel32(io.xy, a + h0, cn, hb, &sh.wide);
    __syncthreads();
    if (!sh.wide) {
      kept += select_chunk<false>(pl, hb, cn, a + h0, io.mask, cs, bm, D, unres);
    } else {
      const int half = pl.hit_cap >> 1;
      for (int s0 = 0; s0 < cn; s0 += half) {
        const int sn = min(half, cn - s0);
        stage_sel64(io.xy, a + h0 + s0, sn, hw64);
        __syncthreads();
        kept += select_chunk<true>(pl, hw64, sn, a + h0 + s0, io.mask, cs, bm, D, unres);
      }
    }
  }
  return kept;
}

// ---- the iterative finder (Sec. 2) on theta tiles ----

// Maximum (returned to every thread; *s_max must be 0 beforehand) and, with do_cs, this thread's
// part of the accumulator checksum over the tile's own cells.
template <bool A32>
__device__ int tile_max_cs(const Plan& pl, const uint32_t* acc, int Wd, int aw, int wt, int j0, bool do_cs,
                           int* s_max, unsigned long long& cs) {
  const int NT = pl.n_theta, NR = pl.n_rho, lane = threadIdx.x & 31, warp = threadIdx.x >> 5,
            nwarps = blockDim.x >> 5;
  int m = 0;
  if (pl.mp) {
    for (int k = warp; k < NR; k += nwarps)
      for (int w = lane; w < Wd; w += 32) {
        const uint32_t x = acc[mp_word(w, k + 1, pl.rows_phys)];
        const unsigned lo = x & 0xffffu, hi = x >> 16;
        m = max(m, (int)max(lo, hi));
        if (do_cs) {
          if (lo) cs += (unsigned long long)lo * mix64((unsigned long long)(aw + w) * NR + k + 1);
          if (hi) cs += (unsigned long long)hi * mix64((unsigned long long)(NT - 1 - aw - w) * NR + k + 1);
        }
      }
  } else {
    for (int k = warp; k < NR; k += nwarps)
      for (int c = lane; c < wt; c += 32) {
        const int v = acc_get<A32>(acc, c, k, pl.nrho_pad);
        m = max(m, v);
        if (do_cs && v) cs += (unsigned long long)v * mix64((unsigned long long)(j0 + c) * NR + k + 1);
      }
  }
  m = __reduce_max_sync(kFull, m);
  if (lane == 0 && m) atomicMax(s_max, m);
  __syncthreads();
  return *s_max;
}

// Bit k of word (c, k >> 5) of pbits for every tile-local column c whose cell k holds >= tq votes
// (tile-local columns as in the peak records: mirror-pair word w's low half is column w, its
// high half column 2 Wd - 1 - w).
template <bool A32>
__device__ void tile_candidate_bits(const Plan& pl, const uint32_t* acc, uint32_t* pbits, int Wd, int wt, int tq) {
  const int NR = pl.n_rho, nrb = pl.nrb, lane = threadIdx.x & 31, warp = threadIdx.x >> 5,
            nwarps = blockDim.x >> 5;
  if (pl.mp) {
    for (int k = warp; k < NR; k += nwarps)
      for (int w = lane; w < Wd; w += 32) {
        const uint32_t x = acc[mp_word(w, k + 1, pl.rows_phys)];
        if ((int)(x & 0xffffu) >= tq) atomicOr(&pbits[w * nrb + (k >> 5)], 1u << (k & 31));
        if ((int)(x >> 16) >= tq) atomicOr(&pbits[(2 * Wd - 1 - w) * nrb + (k >> 5)], 1u << (k & 31));
      }
  } else {
    for (int k = warp; k < NR; k += nwarps)
      for (int c = lane; c < wt; c += 32)
        if (acc_get<A32>(acc, c, k, pl.nrho_pad) >= tq) atomicOr(&pbits[c * nrb + (k >> 5)], 1u << (k & 31));
  }
}

__device__ __forceinline__ uint32_t cand_key(int v, int j, int k) {
  return ((uint32_t)v << 20) | ((uint32_t)(1023 - j) << 10) | (uint32_t)(1023 - k);
}

// Candidates of the iterative finder in sparse form: keys (cand_key) in raster order, colstart[j]
// the first candidate of column j and colstart[NT] = C.
struct SparseCands {
  uint32_t* keys;
  const int* colstart;
  int C;
};

// Votes of a cell that is a candidate of a sparse list (the dense rounds only ask for candidates):
// the row within its column's list by binary search.
struct ListCells {
  static constexpr bool kSorted = true;  // the rounds walk a column's list instead of searching each cell
  const uint32_t* keys;
  const int* colstart;
  // first candidate of column j at row k or below it in the list (rows ascend), else the column's end
  __device__ int lower(int j, int k) const {
    int lo = colstart[j], hi = colstart[j + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (1023 - (int)(keys[mid] & 1023u) < k) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  }
  __device__ int end(int j) const { return colstart[j + 1]; }
  __device__ uint32_t key(int p) const { return keys[p]; }
  __device__ int get(int j, int k) const {
    const int lo = lower(j, k);
    return (lo < colstart[j + 1] && 1023 - (int)(keys[lo] & 1023u) == k) ? (int)(keys[lo] >> 20) : 0;
  }
};

// Visits every other candidate in the suppression window of candidate i (columns j - R .. j + R
// and rows k - R .. k + R; a column past either end of the theta range is taken from the other end
// with the rows mirrored, rows beyond the rho edges do not exist), each column's rows found by a
// binary search; visit(m, key_m) returns false to stop.
template <class V>
__device__ __forceinline__ void visit_window(const SparseCands& s, int NT, int NR, int R, int i, V&& visit) {
  const uint32_t key = s.keys[i];
  const int j = 1023 - (int)((key >> 10) & 1023u), k = 1023 - (int)(key & 1023u);
  for (int d = -R; d <= R; ++d) {
    int jj = j + d, r0 = max(0, k - R), r1 = min(NR - 1, k + R);
    if (jj < 0 || jj >= NT) {
      jj = jj < 0 ? jj + NT : jj - NT;
      const int q0 = NR - 1 - r1;
      r1 = NR - 1 - r0;
      r0 = q0;
    }
    int lo = s.colstart[jj];
    const int end = s.colstart[jj + 1];
    int hi = end;
    while (lo < hi) {  // first candidate of column jj at a row >= r0
      const int mid = (lo + hi) >> 1;
      if (1023 - (int)(s.keys[mid] & 1023u) < r0) lo = mid + 1;
      else hi = mid;
    }
    for (int m = lo; m < end; ++m) {
      const uint32_t km = s.keys[m];
      if (1023 - (int)(km & 1023u) > r1) break;
      if (m != i && !visit(m, km)) return;
    }
  }
}

// The iterative finder's peaks from its candidates (Sec. 2: the best unsuppressed cell is the next
// peak and suppresses its window, until the best fails the threshold). The passes keep exactly the
// candidates that no kept higher-ranked candidate covers, listed by rank; the window relation is
// symmetric, so a candidate's dominators are the higher-ranked candidates in its own window. They
// are listed once per candidate (CSR, in work when it fits; else every round rescans the window).
// Rounds then settle the candidates in parallel: dropped once a dominator is kept, kept once every
// dominator is dropped; every round settles at least the best undecided one. The kept keys,
// compacted into the front of keys and ordered by rank (bitonic within keys_room, else by
// counting), are stored to dst (the first maxp); returns their count. All threads call it.
__device__ int resolve_sparse(const Plan& pl, const SparseCands& s, int keys_room, unsigned char* work,
                              int work_bytes, hough_peak* dst, ItemShared& sh) {
  const int NT = pl.n_theta, NR = pl.n_rho, R = pl.nms_radius, maxp = pl.max_peaks, C = s.C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, bd = blockDim.x, nwarps = bd >> 5;
  volatile uint8_t* st = work;  // 1 undecided, 2 dropped, 3 kept
  const int st_bytes = (C + 15) & ~15, doff_words = (C + 4) & ~3;
  int* doff = reinterpret_cast<int*>(work + st_bytes);
  uint16_t* dom = reinterpret_cast<uint16_t*>(doff + doff_words);  // candidate indices (C < 65536)
  const long long dom_cap = ((long long)work_bytes - st_bytes - 4LL * doff_words) / 2;
  bool csr = dom_cap >= 0;
  if (csr) {
    for (int i = tid; i < C; i += bd) {
      const uint32_t key = s.keys[i];
      int cnt = 0;
      visit_window(s, NT, NR, R, i, [&](int, uint32_t km) {
        cnt += km > key;
        return true;
      });
      doff[i] = cnt;
    }
    __syncthreads();
    const int E = block_exscan(doff, C, sh.tmp);
    if (tid == 0) doff[C] = E;
    csr = E <= dom_cap;  // uniform
    __syncthreads();
  }
  if (csr) {
    for (int i = tid; i < C; i += bd) {
      const uint32_t key = s.keys[i];
      int t = doff[i];
      visit_window(s, NT, NR, R, i, [&](int m, uint32_t km) {
        if (km > key) dom[t++] = (uint16_t)m;
        return true;
      });
      st[i] = doff[i + 1] == doff[i] ? 3 : 1;  // no dominator: kept at once
    }
  } else {
    for (int i = tid; i < C; i += bd) st[i] = 1;
  }
  if (tid < 3) sh.tmp[tid] = 0;
  __syncthreads();
  for (int round = 0;; ++round) {
    int und = 0;
    for (int i = tid; i < C; i += bd) {
      if (st[i] != 1) continue;
      bool drop = false, all = true;
      if (csr) {
        for (int t = doff[i], t1 = doff[i + 1]; t < t1; ++t) {
          const uint8_t sd = st[dom[t]];
          if (sd == 3) {
            drop = true;
            break;
          }
          all = all && sd != 1;
        }
      } else {
        const uint32_t key = s.keys[i];
        visit_window(s, NT, NR, R, i, [&](int m, uint32_t km) {
          const uint8_t sm = st[m];
          if (sm == 3) {  // a kept candidate in the window always ranks above this one
            drop = true;
            return false;
          }
          if (sm == 1 && km > key) all = false;
          return true;
        });
      }
      if (drop) st[i] = 2;
      else if (all) st[i] = 3;
      else ++und;
    }
    // undecided count: three rotating counters, so that one barrier a round suffices
    const int r3 = round % 3;
    und = __reduce_add_sync(kFull, und);
    if (lane == 0 && und) atomicAdd(&sh.tmp[r3], und);
    if (tid == 0) sh.tmp[(r3 + 1) % 3] = 0;
    __syncthreads();
    if (sh.tmp[r3] == 0) break;
  }
  HOUGH_PHASE(HOUGH_PHASE_IT_RESOLVE);
  // the kept keys, compacted in place into the front of keys
  if (tid == 0) sh.it_kept = 0;
  __syncthreads();
  for (int i0 = 0; i0 < C; i0 += bd) {
    const int i = i0 + tid;
    const bool kept = i < C && st[i] == 3;
    const uint32_t key = kept ? s.keys[i] : 0u;
    const unsigned bal = __ballot_sync(kFull, kept);
    if (lane == 0) sh.tmp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, chunk = 0;
    for (int w = 0; w < nwarps; ++w) {
      const int c = sh.tmp[w];
      before += w < warp ? c : 0;
      chunk += c;
    }
    if (kept) s.keys[sh.it_kept + before + __popc(bal & lanemask_lt())] = key;
    __syncthreads();
    if (tid == 0) sh.it_kept += chunk;
    __syncthreads();
  }
  const int nk = sh.it_kept;
  int N = 32;
  while (N < nk) N <<= 1;
  if (nk > 256 && N <= keys_room) {
    for (int i = nk + tid; i < N; i += bd) s.keys[i] = 0u;
    __syncthreads();
    bitonic_desc(s.keys, N);
    for (int i = tid; i < min(nk, maxp); i += bd) store_peak(dst + i, s.keys[i]);
  } else {  // rank = the kept keys above it (keys are distinct)
    for (int i = tid; i < nk; i += bd) {
      const uint32_t key = s.keys[i];
      int r = 0;
      for (int m = 0; m < nk; ++m) r += s.keys[m] > key;
      if (r < maxp) store_peak(dst + r, key);
    }
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_IT_ORDER);
  return nk;
}

// The event's peaks from its tiles' candidate lists, in the last tile CTA of the event. The
// event's threshold tq = max(T, ceil(rel max)) comes from the tiles' maxima. The candidates (cells
// >= tq) are gathered in raster order, with the first candidate of every column (colstart), into
// the CTA's free shared memory, and settled in rounds as in the untiled finder (a candidate is
// dropped once a kept candidate lies in its window, kept once every higher-ranked candidate in
// its window is dropped), each window looked up column by column by binary search over rows.
// The kept ones, sorted by rank, are the peaks in extraction order. Returns their count, or -1
// (nothing written) when a tile could not publish all its candidates or they exceed the room.
__device__ int merge_iterative(const Plan& pl, const FusedIO& io, unsigned char* smem, ItemShared& sh, long long e) {
  const int T = pl.tiles, NT = pl.n_theta, NR = pl.n_rho, R = pl.nms_radius, maxp = pl.max_peaks;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, bd = blockDim.x, nwarps = bd >> 5;
  const int nseg = pl.mp ? 2 * T : T, cap = pl.merge_cap;
  int* colstart = reinterpret_cast<int*>(smem + pl.off_acc);  // NT + 1
  uint32_t* keys = reinterpret_cast<uint32_t*>(colstart + ((NT + 4) & ~3));
  if (tid == 0) {
    int M = 0;
    bool ok = true;
    long long run = 0;
    for (int tt = 0; tt < T; ++tt) {
      M = max(M, __ldcg(io.tile_max + e * T + tt));
      ok = ok && __ldcg(io.tile_cnt + 2 * (e * T + tt)) <= maxp;
    }
    for (int sg = 0; sg < nseg; ++sg) {
      const int tt = sg < T ? sg : 2 * T - 1 - sg;
      const int all = __ldcg(io.tile_cnt + 2 * (e * T + tt)), lo = __ldcg(io.tile_cnt + 2 * (e * T + tt) + 1);
      sh.tstart[sg] = run;
      run += sg < T ? lo : all - lo;
    }
    const long long need = ((long long)pl.rel_num * M + pl.rel_den - 1) / pl.rel_den;
    sh.it_tq = (int)max((long long)pl.threshold, need);
    sh.it_ok = ok && M <= 4095 ? 1 : 0;  // a key holds votes in 12 bits
    sh.it_C = 0;
  }
  __syncthreads();
  if (!sh.it_ok) return -1;  // uniform
  const int tq = sh.it_tq;
  // gather the candidates >= tq, in order
  for (int sg = 0; sg < nseg; ++sg) {
    const int tt = sg < T ? sg : 2 * T - 1 - sg;
    const int all = __ldcg(io.tile_cnt + 2 * (e * T + tt)), lo = __ldcg(io.tile_cnt + 2 * (e * T + tt) + 1);
    const int from = sg < T ? 0 : lo, ct = sg < T ? lo : all - lo;
    const hough_peak* src = io.tile_peaks + (e * T + tt) * (long long)maxp + from;
    for (int i0 = 0; i0 < ct; i0 += bd) {
      const int i = i0 + tid;
      uint32_t key = 0;
      bool keep = false;
      if (i < ct) {
        const int2 r = __ldcg(reinterpret_cast<const int2*>(src) + i);
        const int j = r.x & 0xffff, k = (r.x >> 16) & 0xffff, v = r.y & 0xffff;
        keep = v >= tq;
        key = cand_key(v, j, k);
      }
      const unsigned bal = __ballot_sync(kFull, keep);
      if (lane == 0) sh.tmp[warp] = __popc(bal);
      __syncthreads();
      int before = 0, chunk = 0;
      for (int w = 0; w < nwarps; ++w) {
        const int c = sh.tmp[w];
        before += w < warp ? c : 0;
        chunk += c;
      }
      const int pos = sh.it_C + before + __popc(bal & lanemask_lt());
      if (keep && pos < cap) keys[pos] = key;
      __syncthreads();
      if (tid == 0) sh.it_C += chunk;
      __syncthreads();
    }
  }
  const int C = sh.it_C;
  if (C > cap) return -1;  // uniform
  // first candidate of every column (keys are in raster order)
  for (int j = tid; j <= NT; j += bd) colstart[j] = 0;
  __syncthreads();
  for (int i = tid; i < C; i += bd) atomicAdd(&colstart[1023 - (int)((keys[i] >> 10) & 1023u)], 1);
  __syncthreads();
  block_exscan(colstart, NT + 1, sh.tmp);
  const SparseCands sc{keys, colstart, C};
  unsigned char* work = reinterpret_cast<unsigned char*>(keys + C);
  const int work_bytes = (int)(smem + pl.off_unres - work);
  hough_peak* dst = io.peaks + e * (long long)maxp;
  // the rounds on a 2-bit state per cell of the event where that map fits (512 x 512: 64 KB);
  // the rank of an undecided neighbour comes from its key, found by binary search in its column
  int stw = 32;
  while (stw < ((NT * NR + 15) >> 4)) stw <<= 1;
  if (4LL * stw <= work_bytes) {
    ListCells lc{keys, colstart};
    const int act_cap = (int)min(2048LL, (work_bytes - 4LL * stw) / 4);  // two lists of 16-bit indices
    const int n = resolve_rounds(lc, NT, NR, R, 0, maxp, keys, C, reinterpret_cast<uint32_t*>(work), stw,
                                 reinterpret_cast<uint16_t*>(work + 4LL * stw), act_cap, dst, sh.tmp);
    if (n >= 0) return n;  // else (past 64 rounds) the sparse form, which needs only keys and colstart
  }
  return resolve_sparse(pl, sc, cap, work, work_bytes, dst, sh);
}

// Steps 1-2 of a work item: clears the CTA's accumulator of theta tile t (with the halo columns,
// the peak bitmap and the flags) and votes the event's hits [a, a + n) into it, chunk by chunk.
template <bool A32>
__device__ void vote_tile(const Plan& pl, const FusedIO& io, unsigned char* smem, ItemShared& sh, long long a, int n,
                          int t) {
  uint32_t* acc = reinterpret_cast<uint32_t*>(smem + pl.off_acc);
  uint32_t* halo = reinterpret_cast<uint32_t*>(smem + pl.off_halo);
  int2* hb = reinterpret_cast<int2*>(smem + pl.off_hits);
  longlong2* hw = reinterpret_cast<longlong2*>(smem + pl.off_hits);
  uint32_t* pbits = reinterpret_cast<uint32_t*>(smem + pl.off_pbits);
  const int16_t* tc = reinterpret_cast<const int16_t*>(smem + pl.off_trig);
  const int16_t* ts = tc + pl.n_theta;
  const int T = pl.tiles, NT = pl.n_theta, nrp = pl.nrho_pad;
  const int j0 = t * pl.tile_w;
  const int wt = min(pl.tile_w, NT - j0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, bd = blockDim.x;
  const int wpad = pl.groups * 32;
  const int rows_w = A32 ? nrp : (nrp >> 1);  // words per column
  // mirror-pair tiles: words [aw, aw + Wd), i.e. columns [aw, aw + Wd) and their mirrors
  // (full tiles own tile_w / 2 words, the last one possibly fewer)
  const int Wd = pl.mp ? (wt >> 1) : 0, aw = t * (pl.tile_w >> 1);

  // lane roles of the vote
  VoteLane L;
  L.mirror = pl.mirror != 0;
  L.halo = warp >= pl.groups * pl.split;
  L.on = false;
  L.cj = L.sj = 0;
  L.col1 = L.col2 = 0;
  const uint32_t acc_s = (uint32_t)__cvta_generic_to_shared(acc);
  const bool want_halo = pl.peak_mode != HOUGH_PEAK_ITERATIVE;  // only the 3x3 test reads the halo
  if (L.halo && pl.mp) {
    // lanes 0-15: word aw - 1, lanes 16-31: word aw + Wd (both of its columns), each lane
    // a sixteenth of the hits; none at the theta wrap or at the middle word
    const int hs = lane >> 4, wg = hs ? aw + Wd : aw - 1;
    L.on = want_halo && (hs ? (aw + Wd < (NT >> 1)) : (aw > 0));
    if (L.on) {
      L.cj = tc[wg];
      L.sj = ts[wg];
    }
    L.col2 = (uint32_t)__cvta_generic_to_shared(halo) + (uint32_t)(hs * pl.rows_phys) * 4u;
    L.p = lane & 15;
    L.P = 16;
  } else if (L.halo) {
    const int jh = lane < 16 ? (j0 - 1 + NT) % NT : (j0 + wt) % NT;
    L.on = want_halo;
    L.cj = tc[jh];
    L.sj = ts[jh];
    L.col2 = (uint32_t)__cvta_generic_to_shared(halo) + (uint32_t)((lane >> 4) * (nrp >> 1)) * 4u;
    L.p = 0;
    L.P = 1;
  } else if (L.mirror) {
    const int P2 = 2 * pl.split;
    const int gpair = warp / P2, g2 = pl.groups - 1 - gpair;
    L.p = warp % P2;
    L.P = P2;
    const int c1 = gpair * 32 + lane;
    L.on = !pl.mp || c1 < Wd;  // lanes past the tile's last word idle
    if (L.on) {
      L.cj = tc[(pl.mp ? aw : j0) + c1];
      L.sj = ts[(pl.mp ? aw : j0) + c1];
    }
    if (pl.mp) {
      L.col1 = acc_s + (uint32_t)mp_word(c1, 0, pl.rows_phys) * 4u;
    } else {
      L.col1 = acc_s + (uint32_t)(((gpair * rows_w) << 5) + lane) * 4u;
      L.col2 = acc_s + (uint32_t)(((g2 * rows_w) << 5) + (31 - lane)) * 4u;
    }
  } else {
    const int g = warp / pl.split;
    L.p = warp % pl.split;
    L.P = pl.split;
    const int c1 = g * 32 + lane;
    L.on = c1 < wt;
    if (L.on) {
      L.cj = tc[j0 + c1];
      L.sj = ts[j0 + c1];
    }
    L.col1 = acc_s + (uint32_t)(((g * rows_w) << 5) + lane) * 4u;
  }

  // 1. clear accumulator, halo columns, peak bitmap and counters
  __syncthreads();
  HOUGH_PHASE_START();
  {
    uint4* z = reinterpret_cast<uint4*>(smem + pl.off_acc);
    const int nz = pl.region_bytes >> 4;
    for (int i = tid; i < nz; i += bd) z[i] = make_uint4(0u, 0u, 0u, 0u);
    if (T > 1)
      for (int i = tid; i < (pl.mp ? 2 * pl.rows_phys : nrp); i += bd) halo[i] = 0u;
    for (int i = tid; i < wpad * pl.nrb; i += bd) pbits[i] = 0;
    if (tid == 0) {
      sh.flags = 0;
      sh.it_max = 0;
    }
  }

  // 2. map + vote, chunk by chunk
  if (tid == 0) sh.reuse = (pl.mp && n > 0 && n <= pl.hit_cap) ? 1 : 0;
  for (int h0 = 0; h0 < n; h0 += pl.hit_cap) {
    const int cn = min(pl.hit_cap, n - h0);
    __syncthreads();
    HOUGH_PHASE(h0 == 0 ? HOUGH_PHASE_CLEAR : HOUGH_PHASE_VOTE);
    if (tid == 0) {
      sh.nv = 0;
      sh.wide = 0;
    }
    __syncthreads();
    stage_vote32(io.xy, a + h0, cn, hb, &sh.nv, &sh.wide, pl.fpbin != 0, pl.mp ? pl.mp_lsq : 0,
                 pl.mp ? reinterpret_cast<uint16_t*>(smem + pl.off_idx) : nullptr);
    __syncthreads();
    HOUGH_PHASE(HOUGH_PHASE_STAGE);
    if (tid == 0) {
      if (sh.wide & 2) sh.flags |= HOUGH_F_BAD_HIT;
      if (sh.wide & 1) sh.reuse = 0;  // wide hits are not in the staged list
    }
    if (!(sh.wide & 1)) {
      if (pl.mp)
        vote_mp32(pl, L, hb, sh.nv);
      else if (pl.fpbin)
        vote32_fp<A32>(pl, L, hb, sh.nv);
      else
        vote32<A32>(pl, L, hb, sh.nv);
    } else {
      const int half = pl.hit_cap >> 1;
      for (int s0 = 0; s0 < cn; s0 += half) {
        const int sn = min(half, cn - s0);
        __syncthreads();
        if (tid == 0) sh.nv = 0;
        __syncthreads();
        stage_vote64(io.xy, a + h0 + s0, sn, hw, &sh.nv);
        __syncthreads();
        if (pl.mp)
          vote_mp64(pl, L, hw, sh.nv);
        else
          vote64<A32>(pl, L, hw, sh.nv);
      }
    }
  }
  __syncthreads();
  HOUGH_PHASE(n > 0 ? HOUGH_PHASE_VOTE : HOUGH_PHASE_CLEAR);

}

template <bool A32>
__device__ void run_item(const Plan& pl, const FusedIO& io, unsigned char* smem, ItemShared& sh, long long item,
                         bool do_cs) {
  uint32_t* acc = reinterpret_cast<uint32_t*>(smem + pl.off_acc);
  uint32_t* halo = reinterpret_cast<uint32_t*>(smem + pl.off_halo);
  uint32_t* pbits = reinterpret_cast<uint32_t*>(smem + pl.off_pbits);
  int* cnt = reinterpret_cast<int*>(smem + pl.off_cnt);
  const int16_t* tc = reinterpret_cast<const int16_t*>(smem + pl.off_trig);
  const int16_t* ts = tc + pl.n_theta;

  const int T = pl.tiles, NT = pl.n_theta, NR = pl.n_rho, nrp = pl.nrho_pad;
  const long long e = io.order ? (long long)io.order[item / T] : item / T;
  const int t = (int)(item % T);
  const long long a = io.off[e];
  const long long nll = io.off[e + 1] - a;
  const bool too_large = nll > HOUGH_MAX_EVENT_HITS;
  const int n = too_large ? 0 : (int)nll;
  const int j0 = t * pl.tile_w;
  const int wt = min(pl.tile_w, NT - j0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, bd = blockDim.x;
  const int Wd = pl.mp ? (wt >> 1) : 0, aw = t * (pl.tile_w >> 1);

  vote_tile<A32>(pl, io, smem, sh, a, n, t);

  // 3-4. peaks
  const int maxp = pl.max_peaks;
  int total = 0, n_low = 0;
  unsigned long long cs_tile = 0;
  int tmax = 0;
  if (pl.peak_mode == HOUGH_PEAK_ITERATIVE && T == 1) {
    // the paper's iterative finder on a whole accumulator: the checksum first, then the
    // extraction, which clears the cells it suppresses; records in extraction order
    if (pl.mp) {
      mp_fold(pl, acc, Wd, nullptr);
      __syncthreads();
      HOUGH_PHASE(HOUGH_PHASE_FOLD);
    }
    auto iterative = [&](auto cells) {
      if (do_cs) {
        unsigned long long cs = 0;
        for (int c = tid; c < NT * NR; c += bd) {
          const int v = cells.get(c / NR, c % NR);
          if (v) cs += (unsigned long long)v * mix64((unsigned long long)c + 1);
        }
        cs_tile = block_sum_u64(cs, sh.red);
      }
      __syncthreads();
      HOUGH_PHASE(HOUGH_PHASE_SCAN);
      HOUGH_PHASE(HOUGH_PHASE_SCAN);
      const int st_words = (((NT * NR + 15) >> 4) + 31) & ~31;  // 2 bits a cell, whole 32-word blocks
      return extract_iterative(cells, NT, NR, kIterSliceRows, pl.threshold, pl.rel_num, pl.rel_den, pl.nms_radius,
                               maxp, pbits, pl.iter_cap, nullptr, st_words, io.peaks + e * (long long)maxp, sh.tmp,
                               reinterpret_cast<uint16_t*>(pbits + pl.iter_cap + st_words), pl.iter_act);
    };
    total = pl.mp ? iterative(FusedCells<A32, true>{acc, Wd, nrp, pl.rows_phys})
                  : iterative(FusedCells<A32, false>{acc, Wd, nrp, pl.rows_phys});
    n_low = total;
  } else {
    // 3. peak scan, or (the iterative finder on theta tiles) the tile's candidates: every cell
    // at or above the tile's own relative threshold, a superset of the cells the event's
    // threshold admits (the event's maximum is at least the tile's)
    unsigned long long csum = 0;
    const bool packed = !pl.mp && !A32 && (NR & 1) == 0;
    if (pl.peak_mode == HOUGH_PEAK_ITERATIVE) {
      if (pl.mp) {
        mp_fold(pl, acc, Wd, nullptr);
        __syncthreads();
        HOUGH_PHASE(HOUGH_PHASE_FOLD);
      }
      tmax = tile_max_cs<A32>(pl, acc, Wd, aw, wt, j0, do_cs, &sh.it_max, csum);
      const long long need = ((long long)pl.rel_num * tmax + pl.rel_den - 1) / pl.rel_den;
      tile_candidate_bits<A32>(pl, acc, pbits, Wd, wt, (int)max((long long)pl.threshold, need));
    } else if (pl.mp) {
      mp_fold(pl, acc, Wd, T > 1 ? halo : nullptr);
      __syncthreads();
      HOUGH_PHASE(HOUGH_PHASE_FOLD);
      scan_mp(pl, acc, halo, aw, Wd, pbits, do_cs, csum);
    } else if (packed) {
      scan_packed(pl, acc, halo, pbits, wt, T, j0, do_cs, csum);
    } else {
      scan_scalar<A32>(pl, acc, halo, pbits, wt, T, j0, do_cs, csum);
    }
    __syncthreads();
    HOUGH_PHASE(HOUGH_PHASE_SCAN);

    // 4. raster-order positions and peak records: keys (column, group of key_words bitmap words)
    // in raster order, counted from the peak bitmap
    const int KG = pl.key_groups, G = pl.key_words, nkeys = wt * KG;
    for (int key = tid; key < nkeys; key += bd) {
      const int c = key >> pl.key_shift, w0 = (key & (KG - 1)) * G, w1 = min(pl.nrb, w0 + G);
      int np = 0;
      for (int w = w0; w < w1; ++w) np += __popc(pbits[c * pl.nrb + w]);
      cnt[key] = np;
    }
    __syncthreads();
    total = block_exscan(cnt, nkeys, sh.tmp);
    HOUGH_PHASE(HOUGH_PHASE_EXSCAN);
    // peaks of the tile's low columns (mirror-pair tiles: the high columns follow them)
    n_low = (pl.mp && Wd < wt) ? cnt[Wd << pl.key_shift] : total;
    // event column of tile-local column c: mirror-pair tiles hold [aw, aw + Wd) then
    // [N - aw - Wd, N - aw), both ascending; other tiles [j0, j0 + wt)
    const int hi0 = NT - aw - 2 * Wd;
    hough_peak* dst = (T == 1) ? io.peaks + e * (long long)maxp : io.tile_peaks + (e * T + t) * (long long)maxp;
    uint2* dst2 = reinterpret_cast<uint2*>(dst);  // records are 8-byte aligned (checked on the host)
    const int nwarps = bd >> 5;
    if (G == 1) {
      // A warp takes 32 consecutive keys (one bitmap word each) and writes their peaks to
      // consecutive positions: lane i of a pass finds the key owning position P0 + i (the last
      // lane whose start is <= it) by a shuffle search and the bit by its rank in that word.
      for (int kb = warp * 32; kb < nkeys; kb += nwarps * 32) {
        const int key = kb + lane;
        uint32_t word = 0;
        int start = total;
        if (key < nkeys) {
          const int w = key & (KG - 1);
          word = (w < pl.nrb) ? pbits[(key >> pl.key_shift) * pl.nrb + w] : 0u;
          start = cnt[key];
        }
        const int P0 = __shfl_sync(kFull, start, 0);
        const int P1 = min(__shfl_sync(kFull, start + __popc(word), 31), maxp);
        for (int o0 = P0; o0 < P1; o0 += 32) {
          const int o = o0 + lane;
          int l = 0;
  #pragma unroll
          for (int st = 16; st > 0; st >>= 1) {
            const int sc = __shfl_sync(kFull, start, l + st);
            if (sc <= o) l += st;
          }
          const int r = o - __shfl_sync(kFull, start, l);
          const uint32_t wd = __shfl_sync(kFull, word, l);
          if (o < P1) {
            const int kl = kb + l, c = kl >> pl.key_shift;
            const int k = ((kl & (KG - 1)) << 5) + (int)__fns(wd, 0u, r + 1);
            const int votes = pl.mp ? mp_get(acc, c, k, Wd, pl) : acc_get<A32>(acc, c, k, nrp);
            const int col = pl.mp ? (c < Wd ? aw + c : hi0 + c) : j0 + c;
            dst2[o] = make_uint2((uint32_t)col | ((uint32_t)k << 16), (uint32_t)votes);
          }
        }
      }
    } else {
      for (int key = tid; key < nkeys; key += bd) {
        const int c = key >> pl.key_shift, w0 = (key & (KG - 1)) * G, w1 = min(pl.nrb, w0 + G);
        int pos = cnt[key];
        for (int w = w0; w < w1 && pos < maxp; ++w) {
          uint32_t bits = pbits[c * pl.nrb + w];
          while (bits && pos < maxp) {
            const int bb = __ffs(bits) - 1;
            bits &= bits - 1u;
            const int k = (w << 5) + bb;
            const int votes = pl.mp ? mp_get(acc, c, k, Wd, pl) : acc_get<A32>(acc, c, k, nrp);
            const int col = pl.mp ? (c < Wd ? aw + c : hi0 + c) : j0 + c;
            dst2[pos] = make_uint2((uint32_t)col | ((uint32_t)k << 16), (uint32_t)votes);
            ++pos;
          }
        }
      }
    }
    cs_tile = do_cs ? block_sum_u64(csum, sh.red) : 0ull;
    __syncthreads();
    HOUGH_PHASE(HOUGH_PHASE_RECORDS);
  }

  // 5. tiles: publish, and let the last tile of the event merge
  int ev_total = total;
  unsigned long long ev_cs = cs_tile;
  if (T > 1) {
    if (tid == 0) {
      io.tile_cnt[2 * (e * T + t)] = total;
      io.tile_cnt[2 * (e * T + t) + 1] = n_low;
      if (do_cs) io.tile_cs[e * T + t] = cs_tile;
      if (io.tile_max) io.tile_max[e * T + t] = tmax;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) sh.last = (atomicAdd(&io.tickets[e], 1) == T - 1);
    __syncthreads();
    if (!sh.last) {
      if (tid == 0 && sh.flags) atomicOr(io.status, sh.flags);
      return;
    }
    __threadfence();
    // Raster order of the event: the tiles' low segments in tile order, then (mirror-pair
    // tiles) their high segments in reverse tile order. Segment s < T is tile s's records
    // [0, lo); segment T + i is tile T-1-i's records [lo, all).
    const int nseg = pl.mp ? 2 * T : T;
    if (pl.peak_mode == HOUGH_PEAK_ITERATIVE) {
      ev_total = merge_iterative(pl, io, smem, sh, e);
      if (tid == 0) {
        unsigned long long csa = 0;
        if (do_cs)
          for (int tt = 0; tt < T; ++tt) csa += __ldcg(io.tile_cs + e * T + tt);
        sh.red[0] = csa;
      }
      __syncthreads();
      ev_cs = sh.red[0];
      if (ev_total < 0) {  // deferred: the fallback kernel writes this event's outputs
        if (tid == 0) {
          if (io.checksum) io.checksum[e] = ev_cs;
          io.defer_list[atomicAdd(io.defer_count, 1u)] = (int)e;
          if (sh.flags) atomicOr(io.status, sh.flags);
        }
        return;
      }
    } else {
    if (tid == 0) {
      long long run = 0;
      unsigned long long csa = 0;
      for (int sg = 0; sg < nseg; ++sg) {
        const int tt = sg < T ? sg : 2 * T - 1 - sg;
        const int all = __ldcg(io.tile_cnt + 2 * (e * T + tt)), lo = __ldcg(io.tile_cnt + 2 * (e * T + tt) + 1);
        sh.tstart[sg] = run;
        run += sg < T ? lo : all - lo;
        if (do_cs && sg < T) csa += __ldcg(io.tile_cs + e * T + tt);
      }
      sh.total = (int)run;
      sh.red[0] = csa;
    }
    __syncthreads();
    ev_total = sh.total;
    ev_cs = sh.red[0];
    hough_peak* out = io.peaks + e * (long long)maxp;
    for (int sg = 0; sg < nseg; ++sg) {
      const int tt = sg < T ? sg : 2 * T - 1 - sg;
      const int all = __ldcg(io.tile_cnt + 2 * (e * T + tt)), lo = __ldcg(io.tile_cnt + 2 * (e * T + tt) + 1);
      const int from = sg < T ? 0 : lo, ct = sg < T ? lo : all - lo;
      const long long st0 = sh.tstart[sg];
      const int ncopy = (int)max(0LL, min((long long)ct, (long long)maxp - st0));
      const hough_peak* src = io.tile_peaks + (e * T + tt) * (long long)maxp + from;
      for (int i = tid; i < ncopy; i += bd) {
        const int2 v = __ldcg(reinterpret_cast<const int2*>(src) + i);
        reinterpret_cast<int2*>(out)[st0 + i] = v;
      }
    }
    __syncthreads();
    }
  }

  // 6. event outputs and selection (single tile, or the last tile)
  if (tid == 0) {
    io.npeaks[e] = ev_total;
    if (io.checksum) io.checksum[e] = ev_cs;
    if (ev_total > maxp) sh.flags |= HOUGH_F_PEAK_OVERFLOW;
    if (too_large) sh.flags |= HOUGH_F_EVENT_TOO_LARGE;
  }
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_MERGE);
  int kept = 0;
  if (too_large) {
    for (long long i = tid; i < nll; i += bd) io.mask[a + i] = 0;
  } else {
    kept = select_event(pl, io, smem, sh, tc, ts, a, n, io.peaks + e * (long long)maxp, min(ev_total, maxp),
                        pl.peak_mode == HOUGH_PEAK_LOCAL_MAX && T == 1 && ev_total <= maxp && pl.keep_hw < 32);
  }
  if (tid == 0) sh.kept_tot = 0;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(kFull, kept, o);
  if (lane == 0 && kept) atomicAdd(&sh.kept_tot, kept);
  __syncthreads();
  HOUGH_PHASE(HOUGH_PHASE_SEL_B);
  if (tid == 0) {
    io.nkept[e] = sh.kept_tot;
    if (sh.flags) atomicOr(io.status, sh.flags);
  }
}

template <bool A32>
__global__ void __launch_bounds__(1024) fused_kernel(const Plan pl, const FusedIO io, const TrigTable trig) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ItemShared sh;
  __shared__ long long s_item;
  if (io.status[1] != 0) return;  // offsets of this call failed validation
  int16_t* tc = reinterpret_cast<int16_t*>(smem + pl.off_trig);
  for (int j = threadIdx.x; j < pl.n_theta; j += blockDim.x) {
    tc[j] = trig.c[j];
    tc[pl.n_theta + j] = trig.s[j];
  }
  __syncthreads();  // the table is read before run_item's first barrier
  const bool do_cs = io.checksum != nullptr;
  if (!io.persistent) {
    run_item<A32>(pl, io, smem, sh, blockIdx.x, do_cs);
    return;
  }
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(io.queue, (unsigned long long)pl.grab);
    __syncthreads();
    const long long base = s_item;
    if (base >= io.n_items) break;
    const long long end = min(base + pl.grab, io.n_items);
    for (long long it = base; it < end; ++it) run_item<A32>(pl, io, smem, sh, it, do_cs);
  }
}

// Accumulator of one deferred event in HBM (int32 cells, raster order) for the iterative finder;
// suppressed cells are kept in a shared bitmap.
struct SpillCells {
  static constexpr bool kPairs = false;
  const int* A;
  uint32_t* gone;
  int NR;
  __device__ int get(int j, int k) const {
    const int c = j * NR + k;
    return ((gone[c >> 5] >> (c & 31)) & 1u) ? 0 : A[c];
  }
  __device__ void clear(int j, int k) {
    const int c = j * NR + k;
    atomicOr(&gone[c >> 5], 1u << (c & 31));
  }
};

// Events the tiled iterative finder deferred (a tile's candidates beyond its record slots, more
// candidates than the merging CTA holds, or a maximum beyond the keys' 12-bit vote field): one
// CTA per HBM accumulator slot takes them in turn, votes every tile of the event in shared
// memory exactly as the fused kernel does and stores the cells to its slot, runs the iterative
// finder there (the stepwise form, any size) and selects the hits. Count and list were written
// by the fused kernel before this launch on the same stream.
template <bool A32>
__global__ void __launch_bounds__(1024) deferred_kernel(const Plan pl, const FusedIO io, const TrigTable trig) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ItemShared sh;
  if (io.status[1] != 0) return;
  const unsigned cnt = *io.defer_count;
  if (blockIdx.x >= cnt) return;
  int16_t* tc = reinterpret_cast<int16_t*>(smem + pl.off_trig);
  for (int j = threadIdx.x; j < pl.n_theta; j += blockDim.x) {
    tc[j] = trig.c[j];
    tc[pl.n_theta + j] = trig.s[j];
  }
  __syncthreads();
  const int T = pl.tiles, NT = pl.n_theta, NR = pl.n_rho, tid = threadIdx.x, bd = blockDim.x, lane = tid & 31;
  const uint32_t* acc = reinterpret_cast<const uint32_t*>(smem + pl.off_acc);
  int* A = io.spill + (long long)blockIdx.x * NT * NR;
  for (unsigned d = blockIdx.x; d < cnt; d += gridDim.x) {
    const long long e = io.defer_list[d];
    const long long a = io.off[e], nll = io.off[e + 1] - a;
    const int n = nll > HOUGH_MAX_EVENT_HITS ? 0 : (int)nll;  // a too-large event is never deferred
    int flags = 0;
    for (int t = 0; t < T; ++t) {
      vote_tile<A32>(pl, io, smem, sh, a, n, t);
      const int j0 = t * pl.tile_w, wt = min(pl.tile_w, NT - j0), Wd = pl.mp ? (wt >> 1) : 0,
                aw = t * (pl.tile_w >> 1);
      if (pl.mp) {
        mp_fold(pl, const_cast<uint32_t*>(acc), Wd, nullptr);
        __syncthreads();
        for (int i = tid; i < Wd * NR; i += bd) {
          const int w = i / NR, k = i - w * NR;
          const uint32_t x = acc[mp_word(w, k + 1, pl.rows_phys)];
          A[(aw + w) * NR + k] = (int)(x & 0xffffu);
          A[(NT - 1 - aw - w) * NR + k] = (int)(x >> 16);
        }
      } else {
        for (int i = tid; i < wt * NR; i += bd) {
          const int c = i / NR, k = i - c * NR;
          A[(j0 + c) * NR + k] = acc_get<A32>(acc, c, k, pl.nrho_pad);
        }
      }
      flags |= sh.flags;
      __syncthreads();
    }
    __threadfence_block();
    // the finder: its scratch first, then the suppression bitmap, below the trig table
    uint32_t* scratch = reinterpret_cast<uint32_t*>(smem);
    const int sw = iter_scratch_words(NT, NR, pl.def_sh);
    uint32_t* gone = scratch + (sw > pl.def_cap ? sw : pl.def_cap);
    for (int i = tid; i < (NT * NR + 31) >> 5; i += bd) gone[i] = 0u;
    __syncthreads();
    SpillCells cells{A, gone, NR};
    hough_peak* dst = io.peaks + e * (long long)pl.max_peaks;
    const int total = extract_iterative(cells, NT, NR, pl.def_sh, pl.threshold, pl.rel_num, pl.rel_den,
                                        pl.nms_radius, pl.max_peaks, scratch, pl.def_cap, gone, 0, dst, sh.tmp);
    if (tid == 0) {
      io.npeaks[e] = total;
      if (total > pl.max_peaks) flags |= HOUGH_F_PEAK_OVERFLOW;
      sh.reuse = 0;  // the staged hits were overwritten by the finder
    }
    __syncthreads();
    int kept = select_event(pl, io, smem, sh, tc, tc + NT, a, n, dst, min(total, pl.max_peaks), false);
    if (tid == 0) sh.kept_tot = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(kFull, kept, o);
    if (lane == 0 && kept) atomicAdd(&sh.kept_tot, kept);
    __syncthreads();
    if (tid == 0) {
      io.nkept[e] = sh.kept_tot;
      if (flags) atomicOr(io.status, flags);
    }
    __syncthreads();
  }
}

// Validates offsets (sets status word 1 for the following kernels), resets the persistent
// queue and the per-event tickets, and orders events by decreasing hit count.
__global__ void __launch_bounds__(1024) prep_kernel(const long long* off, long long ne, long long nh, int* status,
                                                    unsigned long long* queue, int* tickets, int* order) {
  __shared__ int hist[2048];
  __shared__ int s_tmp[32];
  int bad = 0;
  for (long long e = threadIdx.x; e < ne; e += blockDim.x) {
    const long long a = off[e], b = off[e + 1];
    if (b < a || a < 0 || b > nh) bad = 1;
  }
  if (threadIdx.x == 0 && (off[0] != 0 || off[ne] != nh)) bad = 1;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    status[1] = bad;
    if (bad) atomicOr(status, HOUGH_F_BAD_OFFSETS);
    if (queue) {
      queue[0] = 0ull;  // the persistent queue's item counter
      queue[1] = 0ull;  // the count of deferred events (tiled iterative finder)
    }
  }
  if (bad) return;
  if (tickets)
    for (long long e = threadIdx.x; e < ne; e += blockDim.x) tickets[e] = 0;
  if (!order) return;
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (long long e = threadIdx.x; e < ne; e += blockDim.x) {
    const long long c = off[e + 1] - off[e];
    atomicAdd(&hist[2047 - (int)min(c >> 4, 2047LL)], 1);
  }
  __syncthreads();
  block_exscan(hist, 2048, s_tmp);
  for (long long e = threadIdx.x; e < ne; e += blockDim.x) {
    const long long c = off[e + 1] - off[e];
    const int pos = atomicAdd(&hist[2047 - (int)min(c >> 4, 2047LL)], 1);
    order[pos] = (int)e;
  }
}

// Random (u, v, column) tuples in the int32 fast-path range: the float bin (with its exact
// fallback) against plain 64-bit floor division. Counts disagreements and fallbacks.
__global__ void selftest_fpbin_kernel(const Plan pl, const TrigTable trig, unsigned long long seed, long long n,
                                      unsigned long long* out) {
  unsigned long long bad = 0, amb = 0, bad_mp = 0, amb_mp = 0, n_mp = 0;
  const FpBin K{pl.fp_khi, pl.fp_dlo, pl.fp_dhi};
  const long long NR = pl.n_rho;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long z = mix64(seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1));
    const int u = (int)(z % (2ULL * kFast32 + 1)) - kFast32;
    const int v = (int)((z >> 20) % (2ULL * kFast32 + 1)) - kFast32;
    const int j = (int)((z >> 44) % (unsigned long long)pl.n_theta);
    const int c = trig.c[j], s = trig.s[j];
    const float uf = (float)u, vf = (float)v;
    const float A = __fmul_rn((float)c, pl.fp_scale), B = __fmul_rn((float)s, pl.fp_scale);
    const float kf = __fmaf_rn(uf, A, __fmaf_rn(vf, B, pl.fp_c0));
    const int k = bin_fp(kf, K, uf, vf, c, s, pl.magic);
    const float kc = fminf(fmaxf(kf, 0.5f), K.khi);
    amb += __fadd_rn(__fadd_rn(kc, K.dlo), 12582912.0f) != __fadd_rn(__fadd_rn(kc, K.dhi), 12582912.0f);
    const long long t = (long long)u * c + (long long)v * s + kH;
    const long long ref = t < 0 ? 0 : min(NR - 1, (t * NR) / (2 * kH));
    bad += (k != ref);
    // mirror-pair estimate: physical row from the bit pattern (guard rows 0 and N_rho + 1
    // stand for the clamped edge bins), exact path inside the ambiguous window
    if ((long long)u * u + (long long)v * v <= pl.mp_lsq) {
      ++n_mp;
      const uint32_t y = (uint32_t)__float_as_int(__fmaf_rn(uf, A, __fmaf_rn(vf, B, pl.mp_c0)));
      long long p;
      if ((y & (uint32_t)pl.mp_amask) == 0u) {
        ++amb_mp;
        p = rho_bin32(u * c + (v * s + (int)kH), pl.magic) + 1;
      } else {
        p = (long long)((y >> pl.mp_F) & (uint32_t)pl.mp_rmask);
        bad_mp += (((y >> pl.mp_F) << 7) - (uint32_t)pl.mp_k7) != ((uint32_t)p << 7);
      }
      bad_mp += (p < 0 || p > NR + 1 || min(max(p - 1, 0LL), NR - 1) != ref);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    bad += __shfl_down_sync(kFull, bad, o);
    amb += __shfl_down_sync(kFull, amb, o);
    bad_mp += __shfl_down_sync(kFull, bad_mp, o);
    amb_mp += __shfl_down_sync(kFull, amb_mp, o);
    n_mp += __shfl_down_sync(kFull, n_mp, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicAdd(out, bad);
    if (amb) atomicAdd(out + 1, amb);
    if (bad_mp) atomicAdd(out + 2, bad_mp);
    if (amb_mp) atomicAdd(out + 3, amb_mp);
    if (n_mp) atomicAdd(out + 4, n_mp);
  }
}

}  // namespace

cudaError_t launch_selftest_fpbin(const Plan& pl, const TrigTable& trig, unsigned long long seed, long long n,
                                  unsigned long long* out, cudaStream_t st) {
  selftest_fpbin_kernel<<<152 * 8, 256, 0, st>>>(pl, trig, seed, n, out);
  return cudaGetLastError();
}

cudaError_t launch_prep(const long long* off, long long n_events, long long n_hits, int* status,
                        unsigned long long* queue, int* tickets, int* order, cudaStream_t st) {
  prep_kernel<<<1, 1024, 0, st>>>(off, n_events, n_hits, status, queue, tickets, order);
  return cudaGetLastError();
}

// Raises the kernel's dynamic shared-memory limit to the largest size requested so far
// (per kernel and device; never lowers it), so that no attribute call happens while a
// stream is being captured into a graph once a shape has been used.
static cudaError_t set_smem(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> limit;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  int& cur = limit[std::make_pair(fn, dev)];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int fused_max_ctas_per_sm(const Plan& pl) {
  const void* fn = pl.acc32 ? (const void*)fused_kernel<true> : (const void*)fused_kernel<false>;
  if (set_smem(fn, pl.smem_bytes) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, pl.threads, pl.smem_bytes) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_fused(const Plan& pl, const FusedIO& io, const TrigTable& trig, int grid, cudaStream_t st) {
  cudaError_t err;
  const bool deferred = pl.peak_mode == HOUGH_PEAK_ITERATIVE && pl.tiles > 1;
  if (pl.acc32) {
    err = set_smem((const void*)fused_kernel<true>, pl.smem_bytes);
    if (err == cudaSuccess && deferred) err = set_smem((const void*)deferred_kernel<true>, pl.smem_bytes);
    if (err != cudaSuccess) return err;
    fused_kernel<true><<<grid, pl.threads, pl.smem_bytes, st>>>(pl, io, trig);
    if (deferred) deferred_kernel<true><<<io.n_spill, pl.threads, pl.smem_bytes, st>>>(pl, io, trig);
  } else {
    err = set_smem((const void*)fused_kernel<false>, pl.smem_bytes);
    if (err == cudaSuccess && deferred) err = set_smem((const void*)deferred_kernel<false>, pl.smem_bytes);
    if (err != cudaSuccess) return err;
    fused_kernel<false><<<grid, pl.threads, pl.smem_bytes, st>>>(pl, io, trig);
    if (deferred) deferred_kernel<false><<<io.n_spill, pl.threads, pl.smem_bytes, st>>>(pl, io, trig);
  }
  return cudaGetLastError();
}

}  // namespace hgpu

extern "C" int hough_phase_cycles(uint64_t* host_cycles, int32_t n, int32_t reset, int32_t* enabled) {
  if (!host_cycles || n < 0) return HOUGH_EINVAL;
  const int m = n < HOUGH_PHASE_COUNT ? n : HOUGH_PHASE_COUNT;
#ifdef HOUGH_PHASE_TIMERS
  if (enabled) *enabled = 1;
  unsigned long long buf[HOUGH_PHASE_COUNT];
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(buf, hgpu::g_phase_cycles, sizeof(buf));
  if (e == cudaSuccess && reset) {
    const unsigned long long zero[HOUGH_PHASE_COUNT] = {};
    e = cudaMemcpyToSymbol(hgpu::g_phase_cycles, zero, sizeof(zero));
  }
  if (e != cudaSuccess) {
    hgpu::note_cuda_error(e);
    return HOUGH_ECUDA;
  }
  for (int i = 0; i < m; ++i) host_cycles[i] = buf[i];
#else
  (void)reset;
  if (enabled) *enabled = 0;
  for (int i = 0; i < m; ++i) host_cycles[i] = 0;
#endif
  return HOUGH_OK;
}
