// Fused conformal-Hough kernel: map -> rho -> vote -> peaks -> select, one CTA per
// (event, theta tile) work item, the accumulator never leaving shared memory.
//
// Thread organisation (Sec. 3's event / angle-column / hit parallelism, redone for sm_103a):
//   - a work item is one event, or one theta tile of an event when its accumulator
//     does not fit one CTA's shared memory;
//   - every lane of a "worker" warp owns one theta column of the tile for the whole
//     vote: warp w votes column group g = w / split, hits i = p, p + split, ... with
//     p = w % split. Lane l's cells live in shared-memory bank l only: word
//     ((g * rows + row) * 32 + l), rows = N_rho / 2 packed int16 pairs (or N_rho
//     int32 cells), so the column-parallel vote is free of bank conflicts whatever
//     rho bins the hits hit, and warps sharing a column group add with red.shared;
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

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <bool A32>
__device__ __forceinline__ int acc_index(int c, int k, int nrp) {
  return A32 ? ((((c >> 5) * nrp + k) << 5) + (c & 31)) : ((((c >> 5) * (nrp >> 1) + (k >> 1)) << 5) + (c & 31));
}

template <bool A32>
__device__ __forceinline__ int acc_get(const uint32_t* acc, int c, int k, int nrp) {
  const uint32_t w = acc[acc_index<A32>(c, k, nrp)];
  return A32 ? (int)w : (int)((w >> ((k & 1) << 4)) & 0xffffu);
}

template <bool A32>
__device__ __forceinline__ void vote_cell(uint32_t* colbase, int k) {
  if (A32)
    red_add_shared(colbase + (k << 5), 1u);
  else
    red_add_shared(colbase + ((k >> 1) << 5), 1u << ((k & 1) << 4));
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
__device__ void stage_vote32(const int2* __restrict__ xy, long long base, int cn, int2* hb, int* s_nv, int* s_flags) {
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < cn; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    long long u = 0, v = 0;
    int st = 0;
    bool ok = false;
    if (i < cn) {
      const int2 h = xy[base + i];
      st = map_hit(h.x, h.y, u, v);
      ok = (st == 0);
    }
    const bool f = ok && fits32(u, v);
    const unsigned bal = __ballot_sync(kFull, f);
    if (bal) {
      int slot = 0;
      if (lane == 0) slot = atomicAdd(s_nv, __popc(bal));
      slot = __shfl_sync(kFull, slot, 0);
      if (f) hb[slot + __popc(bal & lanemask_lt())] = make_int2((int)u, (int)v);
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

template <bool A32>
__device__ __forceinline__ void vote32(const Plan& pl, uint32_t* acc, int* halo, const int2* hb, int nv, int cj,
                                       int sj, bool col_ok, bool halo_warp, int hc, int hs, int g, int p,
                                       int lane) {
  const int Hh = (int)kH;
  const BinMagic m = pl.magic;
  if (!halo_warp) {
    if (!col_ok) return;
    uint32_t* colbase = acc + ((A32 ? g * pl.nrho_pad : g * (pl.nrho_pad >> 1)) << 5) + lane;
    const int4* hb4 = reinterpret_cast<const int4*>(hb);
    const int np = nv >> 1, P = pl.split;
#pragma unroll 4
    for (int q = p; q < np; q += P) {
      const int4 h = hb4[q];
      const int k0 = rho_bin32(h.x * cj + (h.y * sj + Hh), m);
      const int k1 = rho_bin32(h.z * cj + (h.w * sj + Hh), m);
      vote_cell<A32>(colbase, k0);
      vote_cell<A32>(colbase, k1);
    }
    if ((nv & 1) && p == np % P) {
      const int2 h = hb[nv - 1];
      vote_cell<A32>(colbase, rho_bin32(h.x * cj + (h.y * sj + Hh), m));
    }
  } else {
    int* hcol = halo + (lane >> 4) * pl.nrho_pad;
    for (int i = lane & 15; i < nv; i += 16) {
      const int2 h = hb[i];
      red_add_shared(reinterpret_cast<uint32_t*>(hcol + rho_bin32(h.x * hc + (h.y * hs + Hh), m)), 1u);
    }
  }
}

template <bool A32>
__device__ __forceinline__ void vote64(const Plan& pl, uint32_t* acc, int* halo, const longlong2* hw, int nv, int cj,
                                       int sj, bool col_ok, bool halo_warp, int hc, int hs, int g, int p,
                                       int lane) {
  const BinMagic m = pl.magic;
  if (!halo_warp) {
    if (!col_ok) return;
    uint32_t* colbase = acc + ((A32 ? g * pl.nrho_pad : g * (pl.nrho_pad >> 1)) << 5) + lane;
    for (int q = p; q < nv; q += pl.split) {
      const longlong2 h = hw[q];
      vote_cell<A32>(colbase, rho_bin64(h.x * cj + h.y * sj + kH, m));
    }
  } else {
    int* hcol = halo + (lane >> 4) * pl.nrho_pad;
    for (int i = lane & 15; i < nv; i += 16) {
      const longlong2 h = hw[i];
      red_add_shared(reinterpret_cast<uint32_t*>(hcol + rho_bin64(h.x * hc + h.y * hs + kH, m)), 1u);
    }
  }
}

// ---- selection: one lane per hit, pulling hits dynamically, testing peak columns in
// decreasing order of peak count until one accepts the hit ----

template <bool WIDE>
__device__ int select_pull(const Plan& pl, const void* buf, int cn, long long mbase, uint8_t* __restrict__ mask,
                           const int2* cs, const uint32_t* bm, int D, int* s_next) {
  const int lane = threadIdx.x & 31;
  const BinMagic m = pl.magic;
  const int nrb = pl.nrb;
  int i = -1, d = 0, kept = 0;
  bool fin = false;
  long long u = 0, v = 0;
  for (;;) {
    const bool need = (i < 0) && !fin;
    const unsigned nb = __ballot_sync(kFull, need);
    if (nb) {
      const int leader = __ffs(nb) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(s_next, __popc(nb));
      base = __shfl_sync(kFull, base, leader);
      if (need) {
        const int ii = base + __popc(nb & lanemask_lt());
        if (ii < cn) {
          bool bad;
          if (WIDE) {
            const longlong2 h = reinterpret_cast<const longlong2*>(buf)[ii];
            u = h.x;
            v = h.y;
            bad = (h.x == LLONG_MIN);
          } else {
            const int2 h = reinterpret_cast<const int2*>(buf)[ii];
            u = h.x;
            v = h.y;
            bad = (h.x == INT_MIN);
          }
          if (bad)
            mask[mbase + ii] = 0;
          else {
            i = ii;
            d = 0;
          }
        } else {
          fin = true;
        }
      }
    }
    if (__all_sync(kFull, fin)) break;
    if (i >= 0) {
      const int2 c2 = cs[d];
      const int k = WIDE ? rho_bin64(u * c2.x + v * c2.y + kH, m)
                         : rho_bin32((int)u * c2.x + ((int)v * c2.y + (int)kH), m);
      if ((bm[d * nrb + (k >> 5)] >> (k & 31)) & 1u) {
        mask[mbase + i] = 1;
        ++kept;
        i = -1;
      } else if (++d == D) {
        mask[mbase + i] = 0;
        i = -1;
      }
    }
  }
  return kept;
}

struct ItemShared {
  int nv, flags, wide, next, last, total, D;
  int kept_tot;
  long long tstart[64];
  int tmp[32];
  unsigned long long red[32];
};

// Back-projection of every hit of event e against its stored peaks pk[0, S).
__device__ int select_event(const Plan& pl, const FusedIO& io, unsigned char* smem, ItemShared& sh,
                            const int16_t* tc, const int16_t* ts, long long a, int n, const hough_peak* pk, int S) {
  const int NT = pl.n_theta, NR = pl.n_rho, nrb = pl.nrb, tid = threadIdx.x, bd = blockDim.x;
  int* colcnt = reinterpret_cast<int*>(smem + pl.off_acc);
  int* colidx = colcnt + NT;
  int* hist = colidx + NT;
  int2* cs = reinterpret_cast<int2*>(hist + 64);
  uint32_t* bm = reinterpret_cast<uint32_t*>(cs + NT);
  for (int i = tid; i < NT; i += bd) colcnt[i] = 0;
  for (int i = tid; i < 64; i += bd) hist[i] = 0;
  __syncthreads();
  for (int q = tid; q < S; q += bd) atomicAdd(&colcnt[pk[q].theta_bin], 1);
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
    }
  }
  __syncthreads();
  const int D = sh.D;
  for (int i = tid; i < D * nrb; i += bd) bm[i] = 0;
  __syncthreads();
  const int hw = pl.keep_hw;
  for (int q = tid; q < S; q += bd) {
    const hough_peak pq = pk[q];
    const int d = colidx[pq.theta_bin];
    const int lo = max(0, (int)pq.rho_bin - hw), hi = min(NR - 1, (int)pq.rho_bin + hw);
    for (int w = lo >> 5; w <= (hi >> 5); ++w) {
      const int b0 = max(lo, w << 5) & 31, b1 = min(hi, (w << 5) + 31) & 31;
      const uint32_t bits = (b1 == 31 ? 0xffffffffu : ((1u << (b1 + 1)) - 1u)) & ~((1u << b0) - 1u);
      atomicOr(&bm[d * nrb + w], bits);
    }
  }
  __syncthreads();
  int kept = 0;
  if (D == 0) {
    for (int i = tid; i < n; i += bd) io.mask[a + i] = 0;
    return 0;
  }
  int2* hb = reinterpret_cast<int2*>(smem + pl.off_hits);
  longlong2* hw64 = reinterpret_cast<longlong2*>(smem + pl.off_hits);
  for (int h0 = 0; h0 < n; h0 += pl.hit_cap) {
    const int cn = min(pl.hit_cap, n - h0);
    if (tid == 0) {
      sh.wide = 0;
      sh.next = 0;
    }
    __syncthreads();
    stage_sel32(io.xy, a + h0, cn, hb, &sh.wide);
    __syncthreads();
    if (!sh.wide) {
      kept += select_pull<false>(pl, hb, cn, a + h0, io.mask, cs, bm, D, &sh.next);
    } else {
      const int half = pl.hit_cap >> 1;
      for (int s0 = 0; s0 < cn; s0 += half) {
        const int sn = min(half, cn - s0);
        __syncthreads();
        if (tid == 0) sh.next = 0;
        stage_sel64(io.xy, a + h0 + s0, sn, hw64);
        __syncthreads();
        kept += select_pull<true>(pl, hw64, sn, a + h0 + s0, io.mask, cs, bm, D, &sh.next);
      }
    }
    __syncthreads();
  }
  return kept;
}

template <bool A32>
__device__ void run_item(const Plan& pl, const FusedIO& io, unsigned char* smem, ItemShared& sh, long long item,
                         bool do_cs) {
  uint32_t* acc = reinterpret_cast<uint32_t*>(smem + pl.off_acc);
  int* halo = reinterpret_cast<int*>(smem + pl.off_halo);
  int2* hb = reinterpret_cast<int2*>(smem + pl.off_hits);
  longlong2* hw = reinterpret_cast<longlong2*>(smem + pl.off_hits);
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
  const int nwork = pl.groups * pl.split;
  const bool halo_warp = (warp >= nwork);
  const int g = warp / pl.split, p = warp % pl.split;
  const int cl = g * 32 + lane;
  const bool col_ok = !halo_warp && cl < wt;
  const int hl = (j0 - 1 + NT) % NT, hr = (j0 + wt) % NT;
  int cj = 0, sj = 0, hc = 0, hs = 0;
  if (col_ok) {
    cj = tc[j0 + cl];
    sj = ts[j0 + cl];
  }
  if (halo_warp) {
    const int jh = lane < 16 ? hl : hr;
    hc = tc[jh];
    hs = ts[jh];
  }
  const int R = pl.scan_ranges;
  const int wpad = pl.groups * 32;

  // 1. clear accumulator, halo columns, peak bitmap and counters
  __syncthreads();
  {
    uint4* z = reinterpret_cast<uint4*>(smem + pl.off_acc);
    const int nz = pl.region_bytes >> 4;
    for (int i = tid; i < nz; i += bd) z[i] = make_uint4(0u, 0u, 0u, 0u);
    if (T > 1)
      for (int i = tid; i < 2 * nrp; i += bd) halo[i] = 0;
    for (int i = tid; i < wpad * pl.nrb; i += bd) pbits[i] = 0;
    for (int i = tid; i < wpad * R; i += bd) cnt[i] = 0;
    if (tid == 0) sh.flags = 0;
  }

  // 2. map + vote, chunk by chunk
  for (int h0 = 0; h0 < n; h0 += pl.hit_cap) {
    const int cn = min(pl.hit_cap, n - h0);
    __syncthreads();
    if (tid == 0) {
      sh.nv = 0;
      sh.wide = 0;
    }
    __syncthreads();
    stage_vote32(io.xy, a + h0, cn, hb, &sh.nv, &sh.wide);
    __syncthreads();
    if (sh.wide & 2) {
      if (tid == 0) sh.flags |= HOUGH_F_BAD_HIT;
    }
    if (!(sh.wide & 1)) {
      vote32<A32>(pl, acc, halo, hb, sh.nv, cj, sj, col_ok, halo_warp, hc, hs, g, p, lane);
    } else {
      const int half = pl.hit_cap >> 1;
      for (int s0 = 0; s0 < cn; s0 += half) {
        const int sn = min(half, cn - s0);
        __syncthreads();
        if (tid == 0) sh.nv = 0;
        __syncthreads();
        stage_vote64(io.xy, a + h0 + s0, sn, hw, &sh.nv);
        __syncthreads();
        vote64<A32>(pl, acc, halo, hw, sh.nv, cj, sj, col_ok, halo_warp, hc, hs, g, p, lane);
      }
    }
  }
  __syncthreads();

  // 3. peak scan: warps sweep 30-column blocks (lanes 0 and 31 only supply neighbour
  // columns) over row ranges with a 3-row window; neighbour column maxima come by shuffle.
  unsigned long long csum = 0;
  {
    const int nwarps = bd >> 5;
    const int nblk = (wt + 29) / 30;
    const int nunits = nblk * R;
    for (int u = warp; u < nunits; u += nwarps) {
      const int b = u / R, r = u % R;
      const int k0 = (NR * r) / R, k1 = (NR * (r + 1)) / R;
      const int c = b * 30 + lane - 1;
      int kind = 0, scol = c;
      bool mir = false;
      if (c < 0) {
        if (T == 1) {
          scol = wt - 1;
          mir = true;
        } else {
          kind = 1;
          mir = (j0 == 0);
        }
      } else if (c >= wt) {
        if (c == wt) {
          if (T == 1) {
            scol = 0;
            mir = true;
          } else {
            kind = 2;
            mir = (j0 + wt == NT);
          }
        } else {
          kind = 3;
        }
      }
      const bool tested = lane >= 1 && lane <= 30 && c >= 0 && c < wt;
      const bool lstrict = !(c == 0 && j0 == 0);
      const bool rstrict = (c == wt - 1) && (j0 + wt == NT);
      auto fetch = [&](int kk) -> int {
        const int rr = mir ? NR - 1 - kk : kk;
        if (kind == 3 || rr < 0 || rr >= NR) return -1;
        if (kind == 0) return acc_get<A32>(acc, scol, rr, nrp);
        return halo[(kind - 1) * nrp + rr];
      };
      int vp = fetch(k0 - 1), vc = fetch(k0);
      int cnt_l = 0;
      const unsigned long long cell0 = (unsigned long long)(j0 + c) * NR;
      for (int k = k0; k < k1; ++k) {
        const int vn = fetch(k + 1);
        const int vm = max(max(vp, vc), vn);
        const int vmL = __shfl_up_sync(kFull, vm, 1);
        const int vmR = __shfl_down_sync(kFull, vm, 1);
        if (tested && vc >= pl.threshold && vc > vp && vc >= vn && (lstrict ? vc > vmL : vc >= vmL) &&
            (rstrict ? vc > vmR : vc >= vmR)) {
          atomicOr(&pbits[c * pl.nrb + (k >> 5)], 1u << (k & 31));
          ++cnt_l;
        }
        if (do_cs && tested && vc > 0) csum += (unsigned long long)vc * mix64(cell0 + k + 1);
        vp = vc;
        vc = vn;
      }
      if (tested) cnt[c * R + r] = cnt_l;
    }
  }
  __syncthreads();

  // 4. raster-order positions and peak records
  const int total = block_exscan(cnt, wt * R, sh.tmp);
  const int maxp = pl.max_peaks;
  hough_peak* dst = (T == 1) ? io.peaks + e * (long long)maxp : io.tile_peaks + (e * T + t) * (long long)maxp;
  for (int key = tid; key < wt * R; key += bd) {
    const int c = key / R, r = key % R;
    const int k0 = (NR * r) / R, k1 = (NR * (r + 1)) / R;
    if (k0 >= k1) continue;
    int pos = cnt[key];
    for (int w = k0 >> 5; w <= ((k1 - 1) >> 5); ++w) {
      uint32_t bits = pbits[c * pl.nrb + w];
      const int lo = max(k0 - (w << 5), 0), hi = min(k1 - (w << 5), 32);
      bits &= (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
      while (bits) {
        const int bb = __ffs(bits) - 1;
        bits &= bits - 1u;
        const int k = (w << 5) + bb;
        if (pos < maxp) {
          hough_peak pk;
          pk.theta_bin = (int16_t)(j0 + c);
          pk.rho_bin = (int16_t)k;
          pk.votes = (int16_t)acc_get<A32>(acc, c, k, nrp);
          pk.flags = 0;
          dst[pos] = pk;
        }
        ++pos;
      }
    }
  }
  const unsigned long long cs_tile = do_cs ? block_sum_u64(csum, sh.red) : 0ull;
  __syncthreads();

  // 5. tiles: publish, and let the last tile of the event merge
  int ev_total = total;
  unsigned long long ev_cs = cs_tile;
  if (T > 1) {
    if (tid == 0) {
      io.tile_cnt[e * T + t] = total;
      if (do_cs) io.tile_cs[e * T + t] = cs_tile;
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
    if (tid == 0) {
      long long run = 0;
      unsigned long long csa = 0;
      for (int tt = 0; tt < T; ++tt) {
        sh.tstart[tt] = run;
        run += __ldcg(io.tile_cnt + e * T + tt);
        if (do_cs) csa += __ldcg(io.tile_cs + e * T + tt);
      }
      sh.total = (int)run;
      sh.red[0] = csa;
    }
    __syncthreads();
    ev_total = sh.total;
    ev_cs = sh.red[0];
    hough_peak* out = io.peaks + e * (long long)maxp;
    for (int tt = 0; tt < T; ++tt) {
      const long long st0 = sh.tstart[tt];
      const int ct = __ldcg(io.tile_cnt + e * T + tt);
      const int ncopy = (int)max(0LL, min((long long)ct, (long long)maxp - st0));
      const hough_peak* src = io.tile_peaks + (e * T + tt) * (long long)maxp;
      for (int i = tid; i < ncopy; i += bd) {
        const int2 v = __ldcg(reinterpret_cast<const int2*>(src) + i);
        reinterpret_cast<int2*>(out)[st0 + i] = v;
      }
    }
    __syncthreads();
  }

  // 6. event outputs and selection (single tile, or the last tile)
  if (tid == 0) {
    io.npeaks[e] = ev_total;
    if (io.checksum) io.checksum[e] = ev_cs;
    if (ev_total > maxp) sh.flags |= HOUGH_F_PEAK_OVERFLOW;
    if (too_large) sh.flags |= HOUGH_F_EVENT_TOO_LARGE;
  }
  __syncthreads();
  int kept = 0;
  if (too_large) {
    for (long long i = tid; i < nll; i += bd) io.mask[a + i] = 0;
  } else {
    kept = select_event(pl, io, smem, sh, tc, ts, a, n, io.peaks + e * (long long)maxp, min(ev_total, maxp));
  }
  if (tid == 0) sh.kept_tot = 0;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(kFull, kept, o);
  if (lane == 0 && kept) atomicAdd(&sh.kept_tot, kept);
  __syncthreads();
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
    if (queue) *queue = 0ull;
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

}  // namespace

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
  if (pl.acc32) {
    err = set_smem((const void*)fused_kernel<true>, pl.smem_bytes);
    if (err != cudaSuccess) return err;
    fused_kernel<true><<<grid, pl.threads, pl.smem_bytes, st>>>(pl, io, trig);
  } else {
    err = set_smem((const void*)fused_kernel<false>, pl.smem_bytes);
    if (err != cudaSuccess) return err;
    fused_kernel<false><<<grid, pl.threads, pl.smem_bytes, st>>>(pl, io, trig);
  }
  return cudaGetLastError();
}

}  // namespace hgpu
